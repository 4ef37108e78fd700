// Multi-word floating point for the Teukolsky step: double-double (dd, 2 x FP64) and
// quad-double (qd, 4 x FP64), the "quadruple" and "octal" precisions of arXiv:1006.0663
// (Sec. 3.D, Sec. 4), written from the published algorithms named at each function:
//   * TwoSum: Knuth, TAOCP vol. 2 (Moller 1965); 6 operations, no branch.
//   * Fast2Sum: Dekker 1971; 3 operations, requires |a| >= |b|.
//   * TwoProd with FMA: p = a*b, e = fma(a, b, -p).
//   * double-word add / multiply: Joldes, Muller, Popescu, "Tight and rigorous error bounds
//     for basic building blocks of double-word arithmetic", ACM TOMS 44 (2017),
//     Algorithms 5 (sloppy add), 6 (accurate add), 10 (times double), 12 (times double-word).
//   * quad-double: Hida, Li, Bailey, "Algorithms for quad-double precision floating point
//     arithmetic", ARITH-15 (2001): renormalisation, addition, multiplication, division.
// All operations are branch-free (the paper's conclusion, Sec. 6, blames the QD library's
// branches for poor GPU efficiency). The same header compiles for host and device; on the
// device every operation is an explicit round-to-nearest intrinsic so that the compiler
// cannot contract or reassociate the error-free transforms.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define MW_HD __host__ __device__ __forceinline__
// set-up-only routines: kept out of line so that the step kernels stay small to compile
#define MW_HD_CALL inline __host__ __device__ __noinline__
#else
#define MW_HD inline
#define MW_HD_CALL inline
#endif

namespace mw {

// ---------------------------------------------------------------------------------------
// Exactly rounded primitives (no contraction).
// ---------------------------------------------------------------------------------------
MW_HD double add_(double a, double b) {
#if defined(__CUDA_ARCH__)
  return __dadd_rn(a, b);
#else
  volatile double r = a + b;
  return r;
#endif
}
MW_HD double sub_(double a, double b) {
#if defined(__CUDA_ARCH__)
  return __dsub_rn(a, b);
#else
  volatile double r = a - b;
  return r;
#endif
}
MW_HD double mul_(double a, double b) {
#if defined(__CUDA_ARCH__)
  return __dmul_rn(a, b);
#else
  volatile double r = a * b;
  return r;
#endif
}
MW_HD double fma_(double a, double b, double c) {
#if defined(__CUDA_ARCH__)
  return __fma_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}

// ---------------------------------------------------------------------------------------
// Error-free transforms.
// ---------------------------------------------------------------------------------------
MW_HD void two_sum(double a, double b, double& s, double& e) {
  s = add_(a, b);
  const double bb = sub_(s, a);
  e = add_(sub_(a, sub_(s, bb)), sub_(b, bb));
}
MW_HD void fast_two_sum(double a, double b, double& s, double& e) {
  s = add_(a, b);
  e = sub_(b, sub_(s, a));
}
MW_HD void two_prod(double a, double b, double& p, double& e) {
  p = mul_(a, b);
  e = fma_(a, b, -p);
}

// TwoSum computed as a Fast2Sum after ordering the operands by magnitude. The order test
// runs on the integer pipe (IEEE magnitudes compare like their bit patterns), so the FP64
// pipe, the scarce resource on this GPU, sees 3 operations instead of 6. Results are
// identical to two_sum for finite operands. On the device the whole transform is one PTX
// block: written as separate C++ pieces, the compiler spent an extra FP64 instruction per
// call when the transforms were chained (measured with the FP64 instruction counters).
MW_HD void two_sum_ord(double a, double b, double& s, double& e) {
#if defined(__CUDA_ARCH__)
  asm("{\n\t.reg .pred p;\n\t.reg .b64 ia, ib;\n\t.reg .f64 hi, lo, d;\n\t"
      "mov.b64 ia, %2;\n\tmov.b64 ib, %3;\n\t"
      "and.b64 ia, ia, 0x7fffffffffffffff;\n\tand.b64 ib, ib, 0x7fffffffffffffff;\n\t"
      "setp.gt.u64 p, ib, ia;\n\t"
      "selp.f64 hi, %3, %2, p;\n\tselp.f64 lo, %2, %3, p;\n\t"
      "add.rn.f64 %0, hi, lo;\n\tsub.rn.f64 d, %0, hi;\n\tsub.rn.f64 %1, lo, d;\n\t}"
      : "=d"(s), "=d"(e)
      : "d"(a), "d"(b));
#else
  long long ia, ib;
  std::memcpy(&ia, &a, 8);
  std::memcpy(&ib, &b, 8);
  ia &= 0x7fffffffffffffffLL;
  ib &= 0x7fffffffffffffffLL;
  const bool swap = ib > ia;
  const double hi = swap ? b : a;
  const double lo = swap ? a : b;
  fast_two_sum(hi, lo, s, e);
#endif
}

// a - b as two_sum_ord(a, -b), with the sign of b flipped on the integer side so that the
// negation costs no FP64 operation.
MW_HD void two_diff_ord(double a, double b, double& s, double& e) {
#if defined(__CUDA_ARCH__)
  asm("{\n\t.reg .pred p;\n\t.reg .b64 ia, ib, nbb;\n\t.reg .f64 nb, hi, lo, d;\n\t"
      "mov.b64 ia, %2;\n\tmov.b64 nbb, %3;\n\t"
      "xor.b64 nbb, nbb, 0x8000000000000000;\n\tmov.b64 nb, nbb;\n\t"
      "and.b64 ia, ia, 0x7fffffffffffffff;\n\tand.b64 ib, nbb, 0x7fffffffffffffff;\n\t"
      "setp.gt.u64 p, ib, ia;\n\t"
      "selp.f64 hi, nb, %2, p;\n\tselp.f64 lo, %2, nb, p;\n\t"
      "add.rn.f64 %0, hi, lo;\n\tsub.rn.f64 d, %0, hi;\n\tsub.rn.f64 %1, lo, d;\n\t}"
      : "=d"(s), "=d"(e)
      : "d"(a), "d"(b));
#else
  two_sum_ord(a, -b, s, e);
#endif
}

// ---------------------------------------------------------------------------------------
// double-double
// ---------------------------------------------------------------------------------------
struct dd {
  double h, l;
};

MW_HD dd dd_from(double x) { return dd{x, 0.0}; }
MW_HD dd dd_neg(dd a) { return dd{-a.h, -a.l}; }
// Multiplication by a power of two: exact word by word.
MW_HD dd dd_scale2(dd a, double p2) { return dd{mul_(a.h, p2), mul_(a.l, p2)}; }

// JMP17 Algorithm 5 (SloppyDWPlusDW): error bounded relative to |a| + |b|.
MW_HD dd dd_add_sloppy(dd a, dd b) {
  double s, e;
  two_sum_ord(a.h, b.h, s, e);
  e = add_(e, add_(a.l, b.l));
  dd r;
  fast_two_sum(s, e, r.h, r.l);
  return r;
}
// JMP17 Algorithm 6 (AccurateDWPlusDW): relative error <= 3u^2 + 13u^3 of |a + b|.
MW_HD dd dd_add_accurate(dd a, dd b) {
  double sh, sl, th, tl;
  two_sum_ord(a.h, b.h, sh, sl);
  two_sum_ord(a.l, b.l, th, tl);
  const double c = add_(sl, th);
  double vh, vl;
  fast_two_sum(sh, c, vh, vl);
  const double w = add_(tl, vl);
  dd r;
  fast_two_sum(vh, w, r.h, r.l);
  return r;
}
// a - b by JMP17 Algorithm 6 with the subtractions folded into the ordered TwoSums.
MW_HD dd dd_sub_accurate(dd a, dd b) {
  double sh, sl, th, tl;
  two_diff_ord(a.h, b.h, sh, sl);
  two_diff_ord(a.l, b.l, th, tl);
  const double c = add_(sl, th);
  double vh, vl;
  fast_two_sum(sh, c, vh, vl);
  const double w = add_(tl, vl);
  dd r;
  fast_two_sum(vh, w, r.h, r.l);
  return r;
}
MW_HD dd dd_add(dd a, dd b) { return dd_add_accurate(a, b); }
MW_HD dd dd_sub(dd a, dd b) { return dd_add_accurate(a, dd_neg(b)); }
MW_HD dd dd_add_d(dd a, double b) { return dd_add_accurate(a, dd_from(b)); }

// JMP17 Algorithm 12 (DWTimesDW3, with FMA): relative error <= 4u^2.
MW_HD dd dd_mul(dd a, dd b) {
  double ch, cl1;
  two_prod(a.h, b.h, ch, cl1);
  const double tl0 = mul_(a.l, b.l);
  const double tl1 = fma_(a.h, b.l, tl0);
  const double cl2 = fma_(a.l, b.h, tl1);
  const double cl3 = add_(cl1, cl2);
  dd r;
  fast_two_sum(ch, cl3, r.h, r.l);
  return r;
}
// JMP17 Algorithm 10 (DWTimesFP3, with FMA): relative error <= 2u^2.
MW_HD dd dd_mul_d(dd a, double b) {
  double ch, cl1;
  two_prod(a.h, b, ch, cl1);
  const double cl3 = fma_(a.l, b, cl1);
  dd r;
  fast_two_sum(ch, cl3, r.h, r.l);
  return r;
}
// Long division: three quotient digits, then renormalised (used for set-up only).
MW_HD_CALL dd dd_div(dd a, dd b) {
  const double q1 = a.h / b.h;
  dd r = dd_sub(a, dd_mul_d(b, q1));
  const double q2 = r.h / b.h;
  r = dd_sub(r, dd_mul_d(b, q2));
  const double q3 = r.h / b.h;
  dd q;
  fast_two_sum(q1, q2, q.h, q.l);
  return dd_add_d(q, q3);
}
// One Newton step from the double square root: x + (a - x^2) / (2x).
MW_HD_CALL dd dd_sqrt(dd a) {
  if (a.h <= 0.0) return dd{0.0, 0.0};
  const double x = std::sqrt(a.h);
  const dd x2 = dd_mul(dd_from(x), dd_from(x));
  const dd r = dd_sub(a, x2);
  return dd_add_d(dd_from(x), r.h / (2.0 * x));
}

// ---------------------------------------------------------------------------------------
// quad-double: x0 + x1 + x2 + x3, nonoverlapping after renormalisation.
// ---------------------------------------------------------------------------------------
struct qd {
  double x0, x1, x2, x3;
};

MW_HD qd qd_from(double x) { return qd{x, 0.0, 0.0, 0.0}; }
MW_HD qd qd_from_dd(dd a) { return qd{a.h, a.l, 0.0, 0.0}; }
MW_HD qd qd_neg(qd a) { return qd{-a.x0, -a.x1, -a.x2, -a.x3}; }
MW_HD qd qd_scale2(qd a, double p2) {
  return qd{mul_(a.x0, p2), mul_(a.x1, p2), mul_(a.x2, p2), mul_(a.x3, p2)};
}

// Three-term error-free accumulation: (a, b, c) -> (a + b + c, err1, err2).
MW_HD void three_sum(double& a, double& b, double& c) {
  double t1, t2, t3;
  two_sum_ord(a, b, t1, t2);
  two_sum_ord(c, t1, a, t3);
  two_sum_ord(t2, t3, b, c);
}
// (a, b, c) -> (a + b + c, err) with the lower-order error dropped.
MW_HD void three_sum2(double& a, double& b, double c) {
  double t1, t2, t3;
  two_sum_ord(a, b, t1, t2);
  two_sum_ord(c, t1, a, t3);
  b = add_(t2, t3);
}

// Renormalisation of five overlapping terms (ordered by decreasing magnitude) into four
// (HLB01 Sec. 3.1, written branch-free): a bottom-up TwoSum sweep leaves the total in the
// leading word and exact remainders e1..e4; a top-down TwoSum sweep folds the remainders
// into three trailing words. Only the last addition rounds, so the value is kept to about
// one unit in the last place of the fourth word. The pair of sweeps is applied twice so
// that the words come out nonoverlapping.
MW_HD void renorm_pass(double& c0, double& c1, double& c2, double& c3, double c4) {
  double s, e1, e2, e3, e4, v;
  two_sum_ord(c3, c4, s, e4);
  two_sum_ord(c2, s, s, e3);
  two_sum_ord(c1, s, s, e2);
  two_sum_ord(c0, s, s, e1);
  c0 = s;
  two_sum_ord(e1, e2, c1, v);
  two_sum_ord(v, e3, c2, v);
  c3 = add_(v, e4);
}
MW_HD qd qd_renorm(double c0, double c1, double c2, double c3, double c4) {
  renorm_pass(c0, c1, c2, c3, c4);
  renorm_pass(c0, c1, c2, c3, 0.0);
  return qd{c0, c1, c2, c3};
}

// HLB01 quad-double addition ("sloppy" variant: errors relative to |a| + |b|).
MW_HD qd qd_add(qd a, qd b) {
  double s0, s1, s2, s3, t0, t1, t2, t3;
  two_sum_ord(a.x0, b.x0, s0, t0);
  two_sum_ord(a.x1, b.x1, s1, t1);
  two_sum_ord(a.x2, b.x2, s2, t2);
  two_sum_ord(a.x3, b.x3, s3, t3);
  two_sum_ord(s1, t0, s1, t0);
  three_sum(s2, t0, t1);
  three_sum2(s3, t0, t2);
  t0 = add_(add_(t0, t1), t3);
  return qd_renorm(s0, s1, s2, s3, t0);
}
// a - b: qd_add with the four leading subtractions done as ordered TwoDiffs (the sign of b is
// flipped on the integer side, no FP64 negations).
MW_HD qd qd_sub(qd a, qd b) {
  double s0, s1, s2, s3, t0, t1, t2, t3;
  two_diff_ord(a.x0, b.x0, s0, t0);
  two_diff_ord(a.x1, b.x1, s1, t1);
  two_diff_ord(a.x2, b.x2, s2, t2);
  two_diff_ord(a.x3, b.x3, s3, t3);
  two_sum_ord(s1, t0, s1, t0);
  three_sum(s2, t0, t1);
  three_sum2(s3, t0, t2);
  t0 = add_(add_(t0, t1), t3);
  return qd_renorm(s0, s1, s2, s3, t0);
}
MW_HD qd qd_add_d(qd a, double b) { return qd_add(a, qd_from(b)); }

// HLB01 quad-double multiplication: exact products of order 0..2 by TwoProd, order-3
// products rounded, order-4 terms dropped; sums by three-term accumulation.
MW_HD qd qd_mul(qd a, qd b) {
  double p0, q0, p1, q1, p2, q2, p3, q3, p4, q4, p5, q5;
  two_prod(a.x0, b.x0, p0, q0);
  two_prod(a.x0, b.x1, p1, q1);
  two_prod(a.x1, b.x0, p2, q2);
  two_prod(a.x0, b.x2, p3, q3);
  two_prod(a.x1, b.x1, p4, q4);
  two_prod(a.x2, b.x0, p5, q5);
  // order 1: p1 + p2 + q0
  three_sum(p1, p2, q0);
  // order 2: p2 + q1 + q2 + p3 + p4 + p5
  three_sum(p2, q1, q2);
  three_sum(p3, p4, p5);
  double s0, s1, s2, t0, t1;
  two_sum_ord(p2, p3, s0, t0);
  two_sum_ord(q1, p4, s1, t1);
  s2 = add_(q2, p5);
  two_sum_ord(s1, t0, s1, t0);
  s2 = add_(s2, add_(t0, t1));
  // order 3
  s1 = add_(s1, fma_(a.x0, b.x3, fma_(a.x1, b.x2, fma_(a.x2, b.x1, fma_(a.x3, b.x0, add_(add_(q0, q3), add_(q4, q5)))))));
  return qd_renorm(p0, p1, s0, s1, s2);
}
MW_HD qd qd_mul_d(qd a, double b) {
  double p0, q0, p1, q1, p2, q2;
  two_prod(a.x0, b, p0, q0);
  two_prod(a.x1, b, p1, q1);
  two_prod(a.x2, b, p2, q2);
  const double p3 = mul_(a.x3, b);
  double s0 = p0, s1, s2, s3;
  two_sum_ord(q0, p1, s1, s2);
  three_sum(s2, q1, p2);
  three_sum2(q1, q2, p3);
  s3 = q1;
  const double s4 = add_(q2, p2);
  return qd_renorm(s0, s1, s2, s3, s4);
}
// Long division (HLB01 Sec. 3.4): five quotient digits, renormalised. Set-up only.
MW_HD_CALL qd qd_div(qd a, qd b) {
  const double q0 = a.x0 / b.x0;
  qd r = qd_sub(a, qd_mul_d(b, q0));
  const double q1 = r.x0 / b.x0;
  r = qd_sub(r, qd_mul_d(b, q1));
  const double q2 = r.x0 / b.x0;
  r = qd_sub(r, qd_mul_d(b, q2));
  const double q3 = r.x0 / b.x0;
  r = qd_sub(r, qd_mul_d(b, q3));
  const double q4 = r.x0 / b.x0;
  return qd_renorm(q0, q1, q2, q3, q4);
}
// Newton iteration for 1/sqrt(a), then sqrt(a) = a * (1/sqrt(a)) corrected once.
MW_HD_CALL qd qd_sqrt(qd a) {
  if (a.x0 <= 0.0) return qd_from(0.0);
  qd x = qd_from(1.0 / std::sqrt(a.x0));
  const qd half_a = qd_scale2(a, 0.5);
  for (int it = 0; it < 3; ++it) {  // x <- x + x (1/2 - (a/2) x^2)
    const qd t = qd_sub(qd_from(0.5), qd_mul(half_a, qd_mul(x, x)));
    x = qd_add(x, qd_mul(x, t));
  }
  qd y = qd_mul(a, x);  // y ~ sqrt(a); one correction y + x (a - y^2)/2
  const qd corr = qd_mul(qd_scale2(x, 0.5), qd_sub(a, qd_mul(y, y)));
  return qd_add(y, corr);
}

MW_HD double qd_to_double(qd a) { return a.x0 + (a.x1 + (a.x2 + a.x3)); }

}  // namespace mw
