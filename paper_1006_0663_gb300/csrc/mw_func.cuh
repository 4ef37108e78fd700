// Elementary functions in FP64, double-double and quad-double for the one-time set-up of
// the Teukolsky step (tortoise inversion, Sec. 3.B; theta grid and initial pulse). They are
// this library's own implementations: argument reduction plus Taylor series, and Newton
// iterations seeded by the double-precision routine. Constants pi and ln 2 are summed from
// Machin's formula and the atanh series in the target precision. None of this runs in the
// time step.
#pragma once

#include "mw.cuh"

namespace mw {

// ---- uniform operator set over double / dd / qd -----------------------------------------
MW_HD double r_add(double a, double b) { return a + b; }
MW_HD double r_sub(double a, double b) { return a - b; }
MW_HD double r_mul(double a, double b) { return a * b; }
MW_HD double r_mul_d(double a, double b) { return a * b; }
MW_HD double r_div(double a, double b) { return a / b; }
MW_HD double r_sqrt(double a) { return std::sqrt(a); }
MW_HD double r_scale2(double a, double p) { return a * p; }
MW_HD double r_neg(double a) { return -a; }
MW_HD double lead(double a) { return a; }
MW_HD double ldexp_r(double a, int k) { return std::ldexp(a, k); }

MW_HD dd r_add(dd a, dd b) { return dd_add(a, b); }
MW_HD dd r_sub(dd a, dd b) { return dd_sub(a, b); }
MW_HD dd r_mul(dd a, dd b) { return dd_mul(a, b); }
MW_HD dd r_mul_d(dd a, double b) { return dd_mul_d(a, b); }
MW_HD_CALL dd r_div(dd a, dd b) { return dd_div(a, b); }
MW_HD dd r_sqrt(dd a) { return dd_sqrt(a); }
MW_HD dd r_scale2(dd a, double p) { return dd_scale2(a, p); }
MW_HD dd r_neg(dd a) { return dd_neg(a); }
MW_HD double lead(dd a) { return a.h; }
MW_HD dd ldexp_r(dd a, int k) { return dd{std::ldexp(a.h, k), std::ldexp(a.l, k)}; }

MW_HD_CALL qd r_add(qd a, qd b) { return qd_add(a, b); }
MW_HD_CALL qd r_sub(qd a, qd b) { return qd_sub(a, b); }
MW_HD_CALL qd r_mul(qd a, qd b) { return qd_mul(a, b); }
MW_HD_CALL qd r_mul_d(qd a, double b) { return qd_mul_d(a, b); }
MW_HD_CALL qd r_div(qd a, qd b) { return qd_div(a, b); }
MW_HD qd r_sqrt(qd a) { return qd_sqrt(a); }
MW_HD qd r_scale2(qd a, double p) { return qd_scale2(a, p); }
MW_HD qd r_neg(qd a) { return qd_neg(a); }
MW_HD double lead(qd a) { return a.x0; }
MW_HD qd ldexp_r(qd a, int k) {
  return qd{std::ldexp(a.x0, k), std::ldexp(a.x1, k), std::ldexp(a.x2, k), std::ldexp(a.x3, k)};
}

template <class R> MW_HD R r_from(double x);
template <> MW_HD double r_from<double>(double x) { return x; }
template <> MW_HD dd r_from<dd>(double x) { return dd_from(x); }
template <> MW_HD qd r_from<qd>(double x) { return qd_from(x); }

template <class R> struct prec_traits;
template <> struct prec_traits<double> { static constexpr int words = 1; static constexpr double eps = 1.2e-16; };
template <> struct prec_traits<dd> { static constexpr int words = 2; static constexpr double eps = 1e-33; };
template <> struct prec_traits<qd> { static constexpr int words = 4; static constexpr double eps = 1e-66; };

MW_HD double r_div_d(double a, double b) { return a / b; }
MW_HD_CALL dd r_div_d(dd a, double b) { return dd_div(a, dd_from(b)); }
MW_HD_CALL qd r_div_d(qd a, double b) { return qd_div(a, qd_from(b)); }

// ---- constants ----------------------------------------------------------------------------
// atan(1/n) = sum_k (-1)^k / ((2k+1) n^(2k+1))
template <class R> MW_HD R atan_inv(double n) {
  R pw = r_div_d(r_from<R>(1.0), n);  // 1/n^(2k+1)
  R sum = pw;
  const double n2 = n * n;
  for (int k = 1; k < 200; ++k) {
    pw = r_div_d(pw, n2);
    const R term = r_div_d(pw, double(2 * k + 1));
    sum = (k & 1) ? r_sub(sum, term) : r_add(sum, term);
    if (std::fabs(lead(term)) < prec_traits<R>::eps * 1e-3) break;
  }
  return sum;
}
// Machin: pi = 16 atan(1/5) - 4 atan(1/239).
template <class R> MW_HD R r_pi() {
  return r_sub(r_scale2(atan_inv<R>(5.0), 16.0), r_scale2(atan_inv<R>(239.0), 4.0));
}
template <> MW_HD double r_pi<double>() { return 3.141592653589793; }  // nearest double
// ln 2 = 2 atanh(1/3) = 2 sum_k (1/3)^(2k+1)/(2k+1).
template <class R> MW_HD R r_ln2() {
  R pw = r_div_d(r_from<R>(1.0), 3.0);
  R sum = pw;
  for (int k = 1; k < 200; ++k) {
    pw = r_div_d(pw, 9.0);
    const R term = r_div_d(pw, double(2 * k + 1));
    sum = r_add(sum, term);
    if (std::fabs(lead(term)) < prec_traits<R>::eps * 1e-3) break;
  }
  return r_scale2(sum, 2.0);
}
template <> MW_HD double r_ln2<double>() { return 0.6931471805599453; }  // nearest double

// ---- exp / log -------------------------------------------------------------------------------
// exp(x) = 2^k exp(r), x = k ln2 + r, |r| <= ln2/2; exp(r) from (1 + s)^(2^10) with
// s = exp(r/2^10) - 1 by Taylor, squared as s <- s (s + 2) to keep the small quantity.
template <class R> MW_HD_CALL R r_exp(R x, R ln2) {
  const double xd = lead(x);
  if (xd < -745.0) return r_from<R>(0.0);
  const double k = std::nearbyint(xd / lead(ln2));
  R r = r_sub(x, r_mul_d(ln2, k));
  r = r_scale2(r, 1.0 / 1024.0);
  // Taylor of exp(r) - 1 by Horner: r (1 + r/2 (1 + r/3 (1 + ...)))
  int nterms = prec_traits<R>::words == 1 ? 10 : (prec_traits<R>::words == 2 ? 14 : 24);
  R s = r_from<R>(1.0);
  for (int n = nterms; n >= 2; --n) s = r_add(r_from<R>(1.0), r_div_d(r_mul(r, s), double(n)));
  s = r_mul(r, s);
  for (int i = 0; i < 10; ++i) s = r_mul(s, r_add(s, r_from<R>(2.0)));
  return ldexp_r(r_add(s, r_from<R>(1.0)), int(k));
}
template <> MW_HD double r_exp<double>(double x, double) { return std::exp(x); }

// log(x) by Newton's method on exp: y <- y + x exp(-y) - 1, from the double logarithm.
template <class R> MW_HD_CALL R r_log(R x, R ln2) {
  R y = r_from<R>(std::log(lead(x)));
  const int iters = prec_traits<R>::words == 2 ? 2 : 3;
  for (int it = 0; it < iters; ++it) y = r_add(y, r_sub(r_mul(x, r_exp(r_neg(y), ln2)), r_from<R>(1.0)));
  return y;
}
template <> MW_HD double r_log<double>(double x, double) { return std::log(x); }

// ---- sin / cos on [0, pi] ------------------------------------------------------------------------
template <class R> MW_HD_CALL void taylor_sincos(R y, R& s, R& c) {
  // |y| <= pi/4: sin y = sum (-1)^k y^(2k+1)/(2k+1)!, cos y = sum (-1)^k y^(2k)/(2k)!
  const R y2 = r_mul(y, y);
  R term = y;
  s = y;
  R tc = r_from<R>(1.0);
  c = tc;
  for (int k = 1; k < 60; ++k) {
    tc = r_neg(r_div_d(r_mul(tc, y2), double((2 * k - 1) * (2 * k))));
    term = r_neg(r_div_d(r_mul(term, y2), double((2 * k) * (2 * k + 1))));
    c = r_add(c, tc);
    s = r_add(s, term);
    if (std::fabs(lead(tc)) < prec_traits<R>::eps * 1e-3) break;
  }
}
template <class R> MW_HD void r_sincos(R x, R pi, R& s, R& c) {
  const double xd = lead(x), pd = lead(pi);
  if (xd <= 0.25 * pd) {
    taylor_sincos(x, s, c);
  } else if (xd <= 0.75 * pd) {
    R ss, cc;  // x = pi/2 + y
    taylor_sincos(r_sub(x, r_scale2(pi, 0.5)), ss, cc);
    s = cc;
    c = r_neg(ss);
  } else {
    R ss, cc;  // x = pi - y
    taylor_sincos(r_sub(pi, x), ss, cc);
    s = ss;
    c = r_neg(cc);
  }
}
template <> MW_HD void r_sincos<double>(double x, double, double& s, double& c) {
  s = std::sin(x);
  c = std::cos(x);
}

}  // namespace mw
