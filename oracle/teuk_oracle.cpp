// CPU oracle for the Lax-Wendroff Teukolsky step (Ginjupalli & Khanna, "High-Precision
// Numerical Simulations of Rotating Black Holes Accelerated by CUDA", arXiv:1006.0663).
//
// TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the CUDA path is
// checked against. It shares no code with the product library: it is compiled by itself,
// uses its own arithmetic (IEEE double with FMA contraction disabled, or GNU MPFR at a
// chosen precision, normally 256 bits), and is called only by the test suite, by the
// smoke check and by the CPU-baseline leg of the benchmark.
//
// What it computes, in the paper's order:
//   * tortoise coordinate r* (Sec. 3.B, dr*/dr = (r^2+a^2)/Delta) and its inversion r(r*);
//   * the first-order system u_t + D u_{r*} = S for u = {Phi_R, Phi_I, Pi_R, Pi_I}
//     (Sec. 3.B, Eqs. new_teu2 and d_matrix) obtained from the Teukolsky master equation
//     (Eq. 1) with the ansatz Psi = e^{i m phi~} r^3 Phi (Eq. psiphi) and
//     Pi = Phi_t + b Phi_{r*}, b = (r^2+a^2)/Sigma, Sigma^2 = (r^2+a^2)^2 - a^2 Delta sin^2(th);
//     the paper leaves M, L, A unprinted, the reduction used here is written out below and
//     pinned symbolically against Eq. 1 by the tests;
//   * the two-step Lax-Wendroff iteration (Eqs. lw1, lw2);
//   * 10th-order centred theta derivatives (Sec. 3.D; 2nd order as an option, Sec. 3.B);
//   * zero r* boundaries and axis parity for theta (Sec. 3.B, last paragraph).
//
// Parity status: every function here is pinned by tests (symbolic reduction from Eq. 1,
// theta operator on spin-weighted harmonics, tortoise closed form at a = 0, a -> -a
// conjugation symmetry, a = 0 separability and an independent radial solver, and a forced
// manufactured solution at a != 0: a smooth complex field whose forcing is derived from
// Eq. 1 itself, outside this file, converges at 2nd order, which pins how source()
// combines the complex coefficients). The optional dissipation and theta filter (not part
// of the paper's method) are pinned too: the dissipation through its linearity and its
// action on polynomials and the sawtooth, the filter against Legendre series and
// spin-weighted harmonics.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "mpfr_min.h"

namespace {

// ------------------------------------------------------------------------------------
// Scalar types. `double` is plain IEEE binary64 (the build disables FMA contraction).
// `mp` wraps an MPFR number at g_bits of precision, rounding to nearest.
// ------------------------------------------------------------------------------------
long g_bits = 256;

struct mp {
  mpfr_t v;
  mp() { mpfr_init2(v, g_bits); mpfr_set_si(v, 0, MPFR_RNDN); }
  mp(double d) { mpfr_init2(v, g_bits); mpfr_set_d(v, d, MPFR_RNDN); }
  mp(const mp& o) { mpfr_init2(v, g_bits); mpfr_set(v, o.v, MPFR_RNDN); }
  mp(mp&& o) noexcept { mpfr_init2(v, g_bits); mpfr_swap(v, o.v); }
  mp& operator=(const mp& o) { mpfr_set(v, o.v, MPFR_RNDN); return *this; }
  mp& operator=(mp&& o) noexcept { mpfr_swap(v, o.v); return *this; }
  ~mp() { mpfr_clear(v); }
};
inline mp operator+(const mp& a, const mp& b) { mp r; mpfr_add(r.v, a.v, b.v, MPFR_RNDN); return r; }
inline mp operator-(const mp& a, const mp& b) { mp r; mpfr_sub(r.v, a.v, b.v, MPFR_RNDN); return r; }
inline mp operator*(const mp& a, const mp& b) { mp r; mpfr_mul(r.v, a.v, b.v, MPFR_RNDN); return r; }
inline mp operator/(const mp& a, const mp& b) { mp r; mpfr_div(r.v, a.v, b.v, MPFR_RNDN); return r; }
inline mp operator-(const mp& a) { mp r; mpfr_neg(r.v, a.v, MPFR_RNDN); return r; }
inline bool operator<(const mp& a, const mp& b) { return mpfr_cmp(a.v, b.v) < 0; }

inline double sqrt_(double x) { return std::sqrt(x); }
inline double log_(double x) { return std::log(x); }
inline double exp_(double x) { return std::exp(x); }
inline double sin_(double x) { return std::sin(x); }
inline double cos_(double x) { return std::cos(x); }
inline double abs_(double x) { return std::fabs(x); }
inline double to_d(double x) { return x; }
template <class T> T pi_();
template <> double pi_<double>() { return 3.141592653589793; }  // nearest double to pi

inline mp sqrt_(const mp& x) { mp r; mpfr_sqrt(r.v, x.v, MPFR_RNDN); return r; }
inline mp log_(const mp& x) { mp r; mpfr_log(r.v, x.v, MPFR_RNDN); return r; }
inline mp exp_(const mp& x) { mp r; mpfr_exp(r.v, x.v, MPFR_RNDN); return r; }
inline mp sin_(const mp& x) { mp r; mpfr_sin(r.v, x.v, MPFR_RNDN); return r; }
inline mp cos_(const mp& x) { mp r; mpfr_cos(r.v, x.v, MPFR_RNDN); return r; }
inline mp abs_(const mp& x) { mp r; mpfr_abs(r.v, x.v, MPFR_RNDN); return r; }
inline double to_d(const mp& x) { return mpfr_get_d(x.v, MPFR_RNDN); }
template <> mp pi_<mp>() { mp r; mpfr_const_pi(r.v, MPFR_RNDN); return r; }

// A value as a sum of `n` doubles: w[0] = round(x), w[k] = round(x - w[0] - ... - w[k-1]).
inline void to_words(double x, double* w, int n, int64_t stride) {
  w[0] = x;
  for (int k = 1; k < n; ++k) w[k * stride] = 0.0;
}
inline void to_words(const mp& x, double* w, int n, int64_t stride) {
  mp rest = x;
  for (int k = 0; k < n; ++k) {
    double d = to_d(rest);
    w[k * stride] = d;
    rest = rest - mp(d);
  }
}
template <class T> T from_words(const double* w, int n, int64_t stride) {
  T s = T(w[0]);
  for (int k = 1; k < n; ++k) s = s + T(w[k * stride]);
  return s;
}

}  // namespace

extern "C" {

// Parameters of one problem, as plain IEEE doubles / ints (see teuk_oracle.h for meaning).
struct oracle_params {
  double M, a;
  int32_t s, m;
  double rstar_min, rstar_max;
  int32_t n_r, n_theta;
  double dt;            // outer step (0: 0.25 dr*); integrated with substeps of dt/substeps
  int32_t substeps;     // k >= 1
  int32_t theta_order;  // 10 (Sec. 3.D) or 2 (Sec. 3.B)
  int32_t parity;       // +1 or -1: sign of the reflection of Phi, Pi across each pole
  int32_t row_lo, row_hi;  // window of r* rows simulated (inclusive), 0 .. n_r-1 for all
  double ko_sigma;         // r* dissipation strength (not in the paper; 0 = off), see dissipate()
  double ko_theta;         // theta dissipation strength (not in the paper; 0 = off), see dissipate()
  int32_t theta_filter;    // theta filter (not in the paper; 0 = off): remove multipoles l >= this, see filter_rows()
  int32_t theta_filter_period;  // ... at the outer steps whose index is a multiple of this (0 = 1)
};

}  // extern "C"

namespace {

// 10th-order centred weights for an 11-point stencil on a uniform grid, q = -5..5,
// scaled to integers: d2 * 25200 (second derivative), d1 * 2520 (first derivative).
const double kD2_10[11] = {8, -125, 1000, -6000, 42000, -73766, 42000, -6000, 1000, -125, 8};
const double kD1_10[11] = {-2, 25, -150, 600, -2100, 0, 2100, -600, 150, -25, 2};

template <class T>
T fejer_weight(int N, int j);

template <class T>
struct Solver {
  oracle_params p;
  int nrow = 0, nth = 0;
  T M, a, rp, rm, tort_A, tort_B, rsmin, dr, dt, dts, dth;
  std::vector<T> th, sin_th, cos_th, cot_th;         // [nth]
  std::vector<T> rs_node, rs_half, x_node, x_half;   // [nrow], [nrow-1]
  std::vector<T> cn[8], ch[8];                       // coefficients [row*nth + j]
  std::vector<T> c_theta;                            // [nrow] max_j sqrt(Delta/Sigma^2) at the node
  std::vector<T> u[4], uh[4], un[4];                 // state, half state, next state
  int64_t substeps_done = 0;
  // Test-only forcing of the Pi rows (manufactured solutions): F(t) = e^{-i omega t} F^ at
  // nodes (fn) and half nodes (fh), real and imaginary parts; off unless set.
  bool forced = false;
  T f_omega;
  std::vector<T> fn[2], fh[2];

  // ---- Sec. 3.B: tortoise coordinate.  dr*/dr = (r^2+a^2)/Delta, Delta = (r-r+)(r-r-).
  // With x = r - r+, partial fractions give
  //   r*(x) = r+ + x + A ln(x/2M) + B ln((x + r+ - r-)/2M),
  //   A = 2M r+/(r+ - r-),  B = -2M r-/(r+ - r-),
  // the integration constant being fixed by the ln(./2M) terms (for a = 0 this is
  // r* = r + 2M ln(r/2M - 1)).
  T rstar_of_x(const T& x) const {
    return rp + x + tort_A * log_(x / (T(2.0) * M)) + tort_B * log_((x + rp - rm) / (T(2.0) * M));
  }
  // dr*/dx = (r^2+a^2)/Delta = 1 + A/x + B/(x + r+ - r-).
  T drstar_dx(const T& x) const { return T(1.0) + tort_A / x + tort_B / (x + rp - rm); }

  // Inverse: solve r*(x) = target for x > 0 by Newton's method in xi = ln x, started from a
  // bisection in double precision.
  T x_of_rstar(const T& target) const {
    const double td = to_d(target);
    const double Md = to_d(M), rpd = to_d(rp), rmd = to_d(rm), Ad = to_d(tort_A), Bd = to_d(tort_B);
    auto f = [&](double xi) {
      double x = std::exp(xi);
      return rpd + x + Ad * std::log(x / (2 * Md)) + Bd * std::log((x + rpd - rmd) / (2 * Md)) - td;
    };
    double lo = -740.0, hi = 40.0;  // r*(e^lo) < any target in range, r*(e^hi) > it
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (lo + hi);
      if (f(mid) < 0) lo = mid; else hi = mid;
    }
    T xi = T(0.5 * (lo + hi));
    for (int it = 0; it < 12; ++it) {
      T x = exp_(xi);
      T F = rstar_of_x(x) - target;
      T dF = x * drstar_dx(x);  // d r*/d xi
      xi = xi - F / dF;
    }
    return exp_(xi);
  }

  // ---- Coefficients of the first-order system at (x = r - r+, theta_j).
  // Derived from Eq. 1 (times Delta/r^3) with Psi = e^{i m phi~} r^3 Phi; ' = d/dr*:
  //   -Sigma^2 Phi_tt - B Phi_t + R^2 Phi'' + (6 R Delta/r + C) Phi'
  //       + Delta (Phi_thth + cot(th) Phi_th) + V Phi = 0,
  //   R = r^2 + a^2,
  //   B = 4 i M a m r + 2 s [Delta (r + i a cos th) - M (r^2 - a^2)],
  //   C = 2 r Delta + 2 s (r - M) R + 2 i m a R,
  //   V = R^2 f''/f + C f'/f + 4 i s m a (r - M) + Delta [s - (m + s cos th)^2 / sin^2 th],
  //   f = r^3:  f'/f = 3 Delta/(r R),  f''/f = 6 Delta [(r - M) r R + a^2 Delta]/(r^2 R^3).
  // With Pi = Phi_t + b Phi' this is  Phi_t + b Phi' = Pi  and
  //   Pi_t - b Pi' = -c Phi' - (B/Sigma^2) Pi + (Delta/Sigma^2) L_th Phi + (V/Sigma^2) Phi,
  //   c = b b' - (b B + 6 R Delta/r + C)/Sigma^2,
  //   b b' = a^2 Delta sin^2 th [R (r - M) - 2 r Delta]/Sigma^4,
  // so D = diag(b, b, -b, -b) as printed in Eq. d_matrix.
  // Output order: b, c_R, c_I, (B/S2)_R, (B/S2)_I, Delta/S2, (V/S2)_R, (V/S2)_I.
  void coeffs(const T& x, int j, T out[8]) const {
    const T s = T(double(p.s)), m = T(double(p.m));
    const T r = rp + x;
    const T Delta = x * (x + rp - rm);
    const T R = r * r + a * a;
    const T sn = sin_th[j], cs = cos_th[j];
    const T sn2 = sn * sn;
    const T Sig2 = R * R - a * a * Delta * sn2;
    const T b = R / sqrt_(Sig2);
    const T fp = T(3.0) * Delta / (r * R);
    const T fpp = T(6.0) * Delta * ((r - M) * r * R + a * a * Delta) / (r * r * R * R * R);
    const T B_R = T(2.0) * s * (Delta * r - M * (r * r - a * a));
    const T B_I = T(4.0) * M * a * m * r + T(2.0) * s * a * Delta * cs;
    const T C_R = T(2.0) * r * Delta + T(2.0) * s * (r - M) * R;
    const T C_I = T(2.0) * m * a * R;
    const T msc = m + s * cs;
    const T pot = Delta * (s - msc * msc / sn2);
    const T V_R = R * R * fpp + C_R * fp + pot;
    const T V_I = C_I * fp + T(4.0) * s * m * a * (r - M);
    const T bbp = a * a * Delta * sn2 * (R * (r - M) - T(2.0) * r * Delta) / (Sig2 * Sig2);
    const T c_R = bbp - (b * B_R + T(6.0) * R * Delta / r + C_R) / Sig2;
    const T c_I = -(b * B_I + C_I) / Sig2;
    out[0] = b;
    out[1] = c_R;
    out[2] = c_I;
    out[3] = B_R / Sig2;
    out[4] = B_I / Sig2;
    out[5] = Delta / Sig2;
    out[6] = V_R / Sig2;
    out[7] = V_I / Sig2;
  }

  int setup(const oracle_params& pp) {
    p = pp;
    if (!(p.M > 0) || !(std::fabs(p.a) < p.M)) return -1;
    if (p.n_r < 3 || p.n_theta < 6 || p.substeps < 1) return -1;
    if (p.theta_order != 10 && p.theta_order != 2) return -1;
    if (p.parity != 1 && p.parity != -1) return -1;
    if (p.row_lo < 0 || p.row_hi >= p.n_r || p.row_hi - p.row_lo < 2) return -1;
    if (!(p.rstar_max > p.rstar_min) || !(p.dt >= 0) || !(p.ko_sigma >= 0) || !(p.ko_theta >= 0)) return -1;
    const int l_low = std::max(std::abs(p.s), std::abs(p.m));
    if (p.theta_filter < 0 || (p.theta_filter > 0 && (p.theta_filter <= l_low || p.theta_filter - l_low > p.n_theta)))
      return -1;
    if (p.theta_filter_period < 0) return -1;
    nrow = p.row_hi - p.row_lo + 1;
    nth = p.n_theta;
    M = T(p.M);
    a = T(p.a);
    const T root = sqrt_(M * M - a * a);
    rp = M + root;
    rm = (a * a) / rp;  // r+ r- = a^2, avoids the cancellation in M - root
    tort_A = T(2.0) * M * rp / (rp - rm);
    tort_B = -(T(2.0) * M * rm) / (rp - rm);
    rsmin = T(p.rstar_min);
    dr = (T(p.rstar_max) - rsmin) / T(double(p.n_r - 1));
    dt = p.dt > 0 ? T(p.dt) : dr * T(0.25);  // dt = 0 selects 0.25 dr* in this precision
    dts = dt / T(double(p.substeps));
    const T pi = pi_<T>();
    dth = pi / T(double(nth));
    th.resize(nth); sin_th.resize(nth); cos_th.resize(nth); cot_th.resize(nth);
    for (int j = 0; j < nth; ++j) {
      th[j] = (T(double(j)) + T(0.5)) * dth;  // cell-centred theta grid
      sin_th[j] = sin_(th[j]);
      cos_th[j] = cos_(th[j]);
      cot_th[j] = cos_th[j] / sin_th[j];
    }
    rs_node.resize(nrow); x_node.resize(nrow);
    rs_half.resize(nrow - 1); x_half.resize(nrow - 1);
    for (int c = 0; c < 8; ++c) { cn[c].resize((size_t)nrow * nth); ch[c].resize((size_t)(nrow - 1) * nth); }
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < nrow; ++i) {
      const int gi = p.row_lo + i;
      rs_node[i] = rsmin + T(double(gi)) * dr;
      x_node[i] = x_of_rstar(rs_node[i]);
      T o[8];
      for (int j = 0; j < nth; ++j) {
        coeffs(x_node[i], j, o);
        for (int c = 0; c < 8; ++c) cn[c][(size_t)i * nth + j] = o[c];
      }
      if (i + 1 < nrow) {
        rs_half[i] = rsmin + (T(double(gi)) + T(0.5)) * dr;
        x_half[i] = x_of_rstar(rs_half[i]);
        for (int j = 0; j < nth; ++j) {
          coeffs(x_half[i], j, o);
          for (int c = 0; c < 8; ++c) ch[c][(size_t)i * nth + j] = o[c];
        }
      }
    }
    c_theta.assign(nrow, T(0.0));
    for (int i = 0; i < nrow; ++i)
      for (int j = 0; j < nth; ++j) {
        const T v = sqrt_(cn[5][(size_t)i * nth + j]);
        if (c_theta[i] < v) c_theta[i] = v;
      }
    for (int c = 0; c < 4; ++c) {
      u[c].assign((size_t)nrow * nth, T(0.0));
      un[c].assign((size_t)nrow * nth, T(0.0));
      uh[c].assign((size_t)(nrow - 1) * nth, T(0.0));
    }
    if (p.theta_filter > 0) setup_filter();
    return 0;
  }

  bool is_boundary_row(int i) const {
    const int gi = p.row_lo + i;
    return gi == 0 || gi == p.n_r - 1;
  }

  // Value of a theta row f at index jj, extended across the poles by reflection with sign P.
  const T& ext(const T* f, int jj) const {
    if (jj < 0) return f[-1 - jj];
    if (jj >= nth) return f[2 * nth - 1 - jj];
    return f[jj];
  }
  T ext_signed(const T* f, int jj) const {
    const bool ghost = jj < 0 || jj >= nth;
    if (ghost && p.parity < 0) return -ext(f, jj);
    return ext(f, jj);
  }

  // L_th f = f_thth + cot(th) f_th with centred differences (Sec. 3.D: 10th order;
  // Sec. 3.B: 2nd order), on the cell-centred grid with parity ghost cells.
  T theta_op(const T* f, int j) const {
    if (p.theta_order == 10) {
      T s2 = T(0.0), s1 = T(0.0);
      for (int q = -5; q <= 5; ++q) {
        const T fv = ext_signed(f, j + q);
        s2 = s2 + T(kD2_10[q + 5]) * fv;
        s1 = s1 + T(kD1_10[q + 5]) * fv;
      }
      const T d2 = s2 / (T(25200.0) * dth * dth);
      const T d1 = s1 / (T(2520.0) * dth);
      return d2 + cot_th[j] * d1;
    }
    const T fm = ext_signed(f, j - 1), f0 = f[j], fpl = ext_signed(f, j + 1);
    const T d2 = (fpl - T(2.0) * f0 + fm) / (dth * dth);
    const T d1 = (fpl - fm) / (T(2.0) * dth);
    return d2 + cot_th[j] * d1;
  }

  // S = -(M - D) u' - L u - A u at one point, from the averaged state ub[4], its r*
  // derivative du[4], L_th of the averaged Phi (LR, LI) and the 8 coefficients.
  //   S_Phi = Pi,
  //   S_Pi  = -c Phi' - (B/Sigma^2) Pi + (Delta/Sigma^2) L_th Phi + (V/Sigma^2) Phi,
  // complex products written out in real and imaginary parts.
  static void source(const T ub[4], const T du[4], const T& LR, const T& LI, const T cf[8], T S[4]) {
    const T &cR = cf[1], &cI = cf[2], &bR = cf[3], &bI = cf[4], &g = cf[5], &vR = cf[6], &vI = cf[7];
    S[0] = ub[2];
    S[1] = ub[3];
    S[2] = -(cR * du[0] - cI * du[1]) - (bR * ub[2] - bI * ub[3]) + g * LR + (vR * ub[0] - vI * ub[1]);
    S[3] = -(cR * du[1] + cI * du[0]) - (bR * ub[3] + bI * ub[2]) + g * LI + (vR * ub[1] + vI * ub[0]);
  }

  // Dissipation (NOT part of the paper's method; off unless ko_sigma > 0 or ko_theta > 0).
  // The two-step Lax-Wendroff iteration damps short r* wavelengths only at a rate
  // ~ (dt/dr*)^2 per iteration; with several iterations per dt = 0.25 dr* that damping is
  // too weak for the modes of near-zero numerical group velocity in the region where the
  // lower-order terms of the r^3-scaled system (c Phi' and V/Sigma^2 Phi) make a frozen
  // wave grow. And the theta terms sit in the source S, so for them the iteration is the
  // explicit midpoint rule, whose amplification exceeds 1 for every oscillatory mode; the
  // largest theta frequencies (grid-scale modes and the (m + s cos th)^2 / sin^2 th
  // potential of the pole cells) set how many iterations per dt that needs.
  // Once per outer step, before its first iteration, every component becomes
  //   u - eps_r d_r^4 u - eps_th(i) d_th^12 u,
  //   eps_r = ko_sigma dt / (16 dr*),  eps_th(i) = ko_theta c_th(i) dt / (4096 dth),
  // with the undivided differences d_r^4 (5 points in r*, rows 2 .. n_r - 3 only) and
  // d_th^12 = (d_th^2)^6 (13 points in theta with the parity ghosts, every interior row),
  // c_th(i) = max_j sqrt(Delta/Sigma^2) at node i. These are Kreiss-Oliger operators of
  // order 4 in r* and 12 in theta integrated over dt: changes of O(dr*^3) and O(dth^11)
  // for smooth fields, so the scheme keeps its 2nd order in (t, r*) and 10th in theta.
  // Both differences are taken from the same u. Window edges stay frozen as in substep().
  void dissipate() {
    const T eps_r = T(p.ko_sigma) * dt / (T(16.0) * dr);
    const bool do_r = p.ko_sigma > 0, do_th = p.ko_theta > 0;
    const int lo = std::max(2, 2 - p.row_lo), hi = std::min(nrow - 3, p.n_r - 3 - p.row_lo);
    // (d^2)^6 = sum_q (-1)^q C(12, 6 + q) f_{j+q}
    static const double kKO12[13] = {1, -12, 66, -220, 495, -792, 924, -792, 495, -220, 66, -12, 1};
    for (int c = 0; c < 4; ++c) {
      un[c] = u[c];
#pragma omp parallel for schedule(static)
      for (int i = 1; i < nrow - 1; ++i) {
        if (is_boundary_row(i)) continue;
        const T eps_th = T(p.ko_theta) * c_theta[i] * dt / (T(4096.0) * dth);
        const T* row = u[c].data() + (size_t)i * nth;
        for (int j = 0; j < nth; ++j) {
          const size_t k = (size_t)i * nth + j, n = (size_t)nth;
          T v = u[c][k];
          if (do_r && i >= lo && i <= hi) {
            const T d4 = u[c][k - 2 * n] - T(4.0) * u[c][k - n] + T(6.0) * u[c][k] - T(4.0) * u[c][k + n] +
                         u[c][k + 2 * n];
            v = v - eps_r * d4;
          }
          if (do_th) {
            T d12 = T(0.0);
            for (int q = -6; q <= 6; ++q) d12 = d12 + T(kKO12[q + 6]) * ext_signed(row, j + q);
            v = v - eps_th * d12;
          }
          un[c][k] = v;
        }
      }
      std::swap(u[c], un[c]);
    }
  }

  // Theta filter (NOT part of the paper's method; off unless theta_filter > 0). A multipole l
  // oscillates near the photon sphere at about (l + 1/2) / (3 sqrt(3) M); once that exceeds
  // what the central r* differences can carry (their frequencies stop at 1/dr*), the
  // multipole is trapped there by the grid, and the lower-order term c Phi' of the
  // r^3-scaled system makes it grow. The filter removes those multipoles once per outer step,
  // after dissipate(): every row of every component becomes its orthogonal projection onto
  //   span { y_l(theta_j) : max(|s|, |m|) <= l < theta_filter },
  // y_l the (unnormalised) spin-weighted harmonic of the problem's s and m, in the discrete
  // inner product <f, g> = sum_j w_j f_j g_j with Fejer's first-rule weights w_j. Written as
  // its definition: the coefficients solve the Gram system G c = b, G_ab = <y_a, y_b>,
  // b_a = <y_a, f>, and the row becomes sum_a c_a y_a.
  int n_keep = 0;
  std::vector<T> fy;     // [n_keep][nth]: y_l(theta_j), l = l_low .. theta_filter - 1
  std::vector<T> fw;     // [nth]: Fejer weights
  std::vector<T> fginv;  // [n_keep][n_keep]: G^-1

  void setup_filter() {
    const int l_low = std::max(std::abs(p.s), std::abs(p.m));
    n_keep = p.theta_filter - l_low;
    fy.assign((size_t)n_keep * nth, T(0.0));
    fw.assign(nth, T(0.0));
    for (int j = 0; j < nth; ++j) fw[j] = fejer_weight<T>(nth, j);
    for (int q = 0; q < n_keep; ++q)
      for (int j = 0; j < nth; ++j) fy[(size_t)q * nth + j] = spin_profile(l_low + q, th[j]);
    // G is symmetric positive definite: Gauss-Jordan elimination without pivoting, on [G | I].
    const int n = n_keep;
    std::vector<T> aug((size_t)n * 2 * n, T(0.0));
    for (int q = 0; q < n; ++q) {
      for (int r = 0; r < n; ++r) {
        T g = T(0.0);
        for (int j = 0; j < nth; ++j) g = g + fw[j] * fy[(size_t)q * nth + j] * fy[(size_t)r * nth + j];
        aug[(size_t)q * 2 * n + r] = g;
      }
      aug[(size_t)q * 2 * n + n + q] = T(1.0);
    }
    for (int c = 0; c < n; ++c) {
      const T piv = aug[(size_t)c * 2 * n + c];
      for (int r = 0; r < 2 * n; ++r) aug[(size_t)c * 2 * n + r] = aug[(size_t)c * 2 * n + r] / piv;
      for (int q = 0; q < n; ++q) {
        if (q == c) continue;
        const T f = aug[(size_t)q * 2 * n + c];
        for (int r = 0; r < 2 * n; ++r)
          aug[(size_t)q * 2 * n + r] = aug[(size_t)q * 2 * n + r] - f * aug[(size_t)c * 2 * n + r];
      }
    }
    fginv.assign((size_t)n * n, T(0.0));
    for (int q = 0; q < n; ++q)
      for (int r = 0; r < n; ++r) fginv[(size_t)q * n + r] = aug[(size_t)q * 2 * n + n + r];
  }

  // Projects every interior row (not the r* boundary rows, nor the frozen window edges).
  void filter_rows() {
    const int n = n_keep;
    for (int c = 0; c < 4; ++c) {
#pragma omp parallel for schedule(static)
      for (int i = 1; i < nrow - 1; ++i) {
        if (is_boundary_row(i)) continue;
        T* row = u[c].data() + (size_t)i * nth;
        std::vector<T> b(n, T(0.0)), coef(n, T(0.0));
        for (int q = 0; q < n; ++q)
          for (int j = 0; j < nth; ++j) b[q] = b[q] + fw[j] * fy[(size_t)q * nth + j] * row[j];
        for (int q = 0; q < n; ++q)
          for (int r = 0; r < n; ++r) coef[q] = coef[q] + fginv[(size_t)q * n + r] * b[r];
        for (int j = 0; j < nth; ++j) {
          T v = T(0.0);
          for (int q = 0; q < n; ++q) v = v + coef[q] * fy[(size_t)q * nth + j];
          row[j] = v;
        }
      }
    }
  }

  // The operators applied once per outer step, before its first iteration; the filter at the
  // outer steps whose index is a multiple of its period.
  void outer_step_ops() {
    if (p.ko_sigma > 0 || p.ko_theta > 0) dissipate();
    const int64_t period = p.theta_filter_period > 0 ? p.theta_filter_period : 1;
    if (p.theta_filter > 0 && (substeps_done / p.substeps) % period == 0) filter_rows();
  }

  // Forcing at time t: (Re, Im) of e^{-i omega t} F^ is (c F^_R + s F^_I, c F^_I - s F^_R).
  void forcing_phase(const T& t, T& c, T& sn) const {
    c = cos_(f_omega * t);
    sn = sin_(f_omega * t);
  }

  // One Lax-Wendroff iteration with step dts (Eqs. lw1, lw2), then the r* boundary rows.
  void substep() {
    if ((p.ko_sigma > 0 || p.ko_theta > 0 || p.theta_filter > 0) && substeps_done % p.substeps == 0)
      outer_step_ops();
    const T half = T(0.5);
    const T hdt = dts * half;
    // forcing phases at t_n (half step) and t_n + dts/2 (full step)
    T fc0 = T(0.0), fs0 = T(0.0), fc1 = T(0.0), fs1 = T(0.0);
    if (forced) {
      const T tn = T(double(substeps_done)) * dts;
      forcing_phase(tn, fc0, fs0);
      forcing_phase(tn + hdt, fc1, fs1);
    }
    // Eq. lw1: u^{n+1/2}_{i+1/2} = (u_{i+1} + u_i)/2 - dt/2 [D (u_{i+1} - u_i)/dr - S^n_{i+1/2}].
#pragma omp parallel for schedule(static)
    for (int h = 0; h < nrow - 1; ++h) {
      std::vector<T> barR(nth), barI(nth);
      for (int j = 0; j < nth; ++j) {
        const size_t k0 = (size_t)h * nth + j, k1 = (size_t)(h + 1) * nth + j;
        barR[j] = (u[0][k1] + u[0][k0]) * half;
        barI[j] = (u[1][k1] + u[1][k0]) * half;
      }
      for (int j = 0; j < nth; ++j) {
        const size_t k0 = (size_t)h * nth + j, k1 = (size_t)(h + 1) * nth + j;
        T ub[4], du[4], cf[8], S[4];
        for (int c = 0; c < 4; ++c) {
          ub[c] = (u[c][k1] + u[c][k0]) * half;
          du[c] = (u[c][k1] - u[c][k0]) / dr;
        }
        for (int c = 0; c < 8; ++c) cf[c] = ch[c][k0];
        const T LR = theta_op(barR.data(), j), LI = theta_op(barI.data(), j);
        source(ub, du, LR, LI, cf, S);
        if (forced) {
          S[2] = S[2] + (fc0 * fh[0][k0] + fs0 * fh[1][k0]);
          S[3] = S[3] + (fc0 * fh[1][k0] - fs0 * fh[0][k0]);
        }
        const T& b = cf[0];
        uh[0][k0] = ub[0] - hdt * (b * du[0] - S[0]);
        uh[1][k0] = ub[1] - hdt * (b * du[1] - S[1]);
        uh[2][k0] = ub[2] - hdt * (-b * du[2] - S[2]);
        uh[3][k0] = ub[3] - hdt * (-b * du[3] - S[3]);
      }
    }
    // Eq. lw2: u^{n+1}_i = u^n_i - dt [D (u_{i+1/2} - u_{i-1/2})/dr - S^{n+1/2}_i].
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nrow; ++i) {
      const bool interior = i > 0 && i < nrow - 1;
      if (!interior || is_boundary_row(i)) {
        for (int c = 0; c < 4; ++c)
          for (int j = 0; j < nth; ++j) {
            const size_t k = (size_t)i * nth + j;
            un[c][k] = is_boundary_row(i) ? T(0.0) : u[c][k];  // window edges stay frozen
          }
        continue;
      }
      std::vector<T> barR(nth), barI(nth);
      for (int j = 0; j < nth; ++j) {
        const size_t kp = (size_t)i * nth + j, km = (size_t)(i - 1) * nth + j;
        barR[j] = (uh[0][kp] + uh[0][km]) * half;
        barI[j] = (uh[1][kp] + uh[1][km]) * half;
      }
      for (int j = 0; j < nth; ++j) {
        const size_t k = (size_t)i * nth + j;
        const size_t kp = (size_t)i * nth + j, km = (size_t)(i - 1) * nth + j;  // i+1/2, i-1/2
        T ub[4], du[4], cf[8], S[4];
        for (int c = 0; c < 4; ++c) {
          ub[c] = (uh[c][kp] + uh[c][km]) * half;
          du[c] = (uh[c][kp] - uh[c][km]) / dr;
        }
        for (int c = 0; c < 8; ++c) cf[c] = cn[c][k];
        const T LR = theta_op(barR.data(), j), LI = theta_op(barI.data(), j);
        source(ub, du, LR, LI, cf, S);
        if (forced) {
          S[2] = S[2] + (fc1 * fn[0][k] + fs1 * fn[1][k]);
          S[3] = S[3] + (fc1 * fn[1][k] - fs1 * fn[0][k]);
        }
        const T& b = cf[0];
        un[0][k] = u[0][k] - dts * (b * du[0] - S[0]);
        un[1][k] = u[1][k] - dts * (b * du[1] - S[1]);
        un[2][k] = u[2][k] - dts * (-b * du[2] - S[2]);
        un[3][k] = u[3][k] - dts * (-b * du[3] - S[3]);
      }
    }
    for (int c = 0; c < 4; ++c) std::swap(u[c], un[c]);
    ++substeps_done;
  }

  // Unnormalised spin-weighted spherical harmonic sY_lm(theta) without e^{i m phi}: the
  // Goldberg et al. sum
  //   sum_r (-1)^(l-r-s) C(l-s, r) C(l+s, r+s-m) sin(th/2)^(2l-2r-s+m) cos(th/2)^(2r+s-m).
  T spin_profile(int l, const T& theta) const {
    const int s = p.s, m = p.m;
    const T sh = sin_(theta * T(0.5)), chh = cos_(theta * T(0.5));
    auto binom = [](int n, int k) -> double {
      if (k < 0 || k > n || n < 0) return 0.0;
      double r = 1.0;
      for (int t = 1; t <= k; ++t) r = r * (n - k + t) / t;
      return std::round(r);
    };
    T sum = T(0.0);
    for (int r = 0; r <= l - s; ++r) {
      const double c = binom(l - s, r) * binom(l + s, r + s - m);
      if (c == 0.0) continue;
      const int es = 2 * l - 2 * r - s + m, ec = 2 * r + s - m;
      T term = T(((l - r - s) % 2 == 0) ? c : -c);
      for (int e = 0; e < es; ++e) term = term * sh;
      for (int e = 0; e < ec; ++e) term = term * chh;
      sum = sum + term;
    }
    return sum;
  }

  // Initial data: Phi = A exp(-((r* - c)/w)^2) sY(theta), zero time derivative, so
  // Pi = Phi_t + b Phi' = b A G'(r*) sY(theta) with G' = -2 (r* - c)/w^2 G.
  void pulse(double center, double width, double amp_re, double amp_im, int ell) {
    const T cc = T(center), w = T(width), AR = T(amp_re), AI = T(amp_im);
    std::vector<T> prof(nth);
    for (int j = 0; j < nth; ++j) prof[j] = spin_profile(ell, th[j]);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < nrow; ++i) {
      const T z = (rs_node[i] - cc) / w;
      const T G = exp_(-(z * z));
      const T Gp = -(T(2.0) * z / w) * G;
      for (int j = 0; j < nth; ++j) {
        const size_t k = (size_t)i * nth + j;
        if (is_boundary_row(i)) {
          for (int c = 0; c < 4; ++c) u[c][k] = T(0.0);
          continue;
        }
        const T& b = cn[0][k];
        u[0][k] = AR * G * prof[j];
        u[1][k] = AI * G * prof[j];
        u[2][k] = b * (AR * Gp * prof[j]);
        u[3][k] = b * (AI * Gp * prof[j]);
      }
    }
    substeps_done = 0;
  }
};

struct Handle {
  long bits;
  Solver<double>* d = nullptr;
  Solver<mp>* m = nullptr;
};

template <class F>
auto dispatch(Handle* h, F&& f) {
  if (h->d) return f(*h->d);
  g_bits = h->bits;
  return f(*h->m);
}

}  // namespace

extern "C" {

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// bits == 53: IEEE double; bits > 53: MPFR with that many bits.
void* oracle_create(const oracle_params* p, int bits) {
  if (!p || bits < 53) return nullptr;
  Handle* h = new (std::nothrow) Handle;
  if (!h) return nullptr;
  h->bits = bits;
  int rc;
  if (bits == 53) {
    h->d = new Solver<double>;
    rc = h->d->setup(*p);
  } else {
    g_bits = bits;
    h->m = new Solver<mp>;
    rc = h->m->setup(*p);
  }
  if (rc != 0) {
    delete h->d;
    if (h->m) { g_bits = bits; delete h->m; }
    delete h;
    return nullptr;
  }
  return h;
}

void oracle_destroy(void* hv) {
  Handle* h = (Handle*)hv;
  if (!h) return;
  delete h->d;
  if (h->m) { g_bits = h->bits; delete h->m; }
  delete h;
}

int oracle_rows(void* hv) { return dispatch((Handle*)hv, [](auto& S) { return S.nrow; }); }

int oracle_set_pulse(void* hv, double center, double width, double amp_re, double amp_im, int ell) {
  Handle* h = (Handle*)hv;
  return dispatch(h, [&](auto& S) {
    if (ell < std::abs(S.p.m) || ell < std::abs(S.p.s) || !(width > 0)) return -1;
    S.pulse(center, width, amp_re, amp_im, ell);
    return 0;
  });
}

// planes: [4][words][nrow][nth] (nrow = window rows); value = sum over words.
int oracle_set_state(void* hv, const double* planes, int words) {
  Handle* h = (Handle*)hv;
  return dispatch(h, [&](auto& S) {
    using T = typename std::decay<decltype(S.dts)>::type;
    const int64_t plane = (int64_t)S.nrow * S.nth;
    for (int c = 0; c < 4; ++c)
      for (int64_t k = 0; k < plane; ++k)
        S.u[c][k] = from_words<T>(planes + ((int64_t)c * words) * plane + k, words, plane);
    S.substeps_done = 0;
    return 0;
  });
}

int oracle_get_state(void* hv, double* planes, int words) {
  Handle* h = (Handle*)hv;
  return dispatch(h, [&](auto& S) {
    const int64_t plane = (int64_t)S.nrow * S.nth;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < plane; ++k)
      for (int c = 0; c < 4; ++c) to_words(S.u[c][k], planes + ((int64_t)c * words) * plane + k, words, plane);
    return 0;
  });
}

// One theta row of the state (window-relative row index): out [4][words][nth].
int oracle_get_row(void* hv, int row, double* out, int words) {
  Handle* h = (Handle*)hv;
  return dispatch(h, [&](auto& S) {
    if (row < 0 || row >= S.nrow) return -1;
    for (int c = 0; c < 4; ++c)
      for (int j = 0; j < S.nth; ++j)
        to_words(S.u[c][(size_t)row * S.nth + j], out + ((int64_t)c * words) * S.nth + j, words, S.nth);
    return 0;
  });
}

// Coefficients: which = 0 nodes [8][words][nrow][nth], which = 1 half nodes [8][words][nrow-1][nth].
int oracle_get_coeffs(void* hv, int which, double* out, int words) {
  Handle* h = (Handle*)hv;
  return dispatch(h, [&](auto& S) {
    const int rows = which ? S.nrow - 1 : S.nrow;
    const int64_t plane = (int64_t)rows * S.nth;
    for (int c = 0; c < 8; ++c)
      for (int64_t k = 0; k < plane; ++k)
        to_words(which ? S.ch[c][k] : S.cn[c][k], out + ((int64_t)c * words) * plane + k, words, plane);
    return 0;
  });
}

// Grid tables: rstar and x = r - r+ at nodes ([words][nrow]) and half nodes ([words][nrow-1]),
// theta_j and cot theta_j ([words][nth]).
int oracle_get_grid(void* hv, double* rs_node, double* x_node, double* rs_half, double* x_half,
                    double* theta, double* cot_theta, int words) {
  Handle* h = (Handle*)hv;
  return dispatch(h, [&](auto& S) {
    for (int i = 0; i < S.nrow; ++i) {
      if (rs_node) to_words(S.rs_node[i], rs_node + i, words, S.nrow);
      if (x_node) to_words(S.x_node[i], x_node + i, words, S.nrow);
    }
    for (int i = 0; i < S.nrow - 1; ++i) {
      if (rs_half) to_words(S.rs_half[i], rs_half + i, words, S.nrow - 1);
      if (x_half) to_words(S.x_half[i], x_half + i, words, S.nrow - 1);
    }
    for (int j = 0; j < S.nth; ++j) {
      if (theta) to_words(S.th[j], theta + j, words, S.nth);
      if (cot_theta) to_words(S.cot_th[j], cot_theta + j, words, S.nth);
    }
    return 0;
  });
}

int oracle_step(void* hv, int64_t n_substeps) {
  Handle* h = (Handle*)hv;
  return dispatch(h, [&](auto& S) {
    for (int64_t n = 0; n < n_substeps; ++n) S.substep();
    return 0;
  });
}

int64_t oracle_substeps_done(void* hv) {
  return dispatch((Handle*)hv, [](auto& S) { return S.substeps_done; });
}

// r*(x) and x(r*) for a black hole (M, a), as word expansions; for tests of the tortoise map.
int oracle_tortoise(int bits, double M, double a, const double* x_words, int words, double* rstar_out,
                    int out_words) {
  oracle_params p{};
  p.M = M; p.a = a; p.s = 0; p.m = 0; p.rstar_min = -1; p.rstar_max = 1; p.n_r = 3; p.n_theta = 6;
  p.dt = 0.1; p.substeps = 1; p.theta_order = 10; p.parity = 1; p.row_lo = 0; p.row_hi = 2;
  Handle* h = (Handle*)oracle_create(&p, bits);
  if (!h) return -1;
  int rc = dispatch(h, [&](auto& S) {
    using T = typename std::decay<decltype(S.dts)>::type;
    to_words(S.rstar_of_x(from_words<T>(x_words, words, 1)), rstar_out, out_words, 1);
    return 0;
  });
  oracle_destroy(h);
  return rc;
}

int oracle_inverse_tortoise(int bits, double M, double a, const double* rstar_words, int words,
                            double* x_out, int out_words) {
  oracle_params p{};
  p.M = M; p.a = a; p.s = 0; p.m = 0; p.rstar_min = -1; p.rstar_max = 1; p.n_r = 3; p.n_theta = 6;
  p.dt = 0.1; p.substeps = 1; p.theta_order = 10; p.parity = 1; p.row_lo = 0; p.row_hi = 2;
  Handle* h = (Handle*)oracle_create(&p, bits);
  if (!h) return -1;
  int rc = dispatch(h, [&](auto& S) {
    using T = typename std::decay<decltype(S.dts)>::type;
    to_words(S.x_of_rstar(from_words<T>(rstar_words, words, 1)), x_out, out_words, 1);
    return 0;
  });
  oracle_destroy(h);
  return rc;
}

// Coefficients at arbitrary (x, theta) points: out [n][8] (one word each, i.e. rounded to double),
// for the symbolic pin. s, m, M, a as in the params.
int oracle_coeffs_at(int bits, const oracle_params* pp, int n, const double* x, const double* theta,
                     double* out) {
  oracle_params p = *pp;
  p.n_theta = 6; p.n_r = 3; p.row_lo = 0; p.row_hi = 2; p.substeps = 1; p.theta_order = 10;
  p.parity = 1; p.rstar_min = -1; p.rstar_max = 1; p.dt = 0.1;
  Handle* h = (Handle*)oracle_create(&p, bits);
  if (!h) return -1;
  int rc = dispatch(h, [&](auto& S) {
    using T = typename std::decay<decltype(S.dts)>::type;
    for (int k = 0; k < n; ++k) {
      S.th[0] = T(theta[k]);
      S.sin_th[0] = sin_(S.th[0]);
      S.cos_th[0] = cos_(S.th[0]);
      T o[8];
      S.coeffs(T(x[k]), 0, o);
      for (int c = 0; c < 8; ++c) out[k * 8 + c] = to_d(o[c]);
    }
    return 0;
  });
  oracle_destroy(h);
  return rc;
}

// max |sum(planes) - u| / max |u| over window rows [row_a, row_b] of all four components.
// planes: [4][words][nrow][nth] like oracle_get_state.
int oracle_max_rel_err(void* hv, const double* planes, int words, int row_a, int row_b, double* err,
                       double* umax) {
  Handle* h = (Handle*)hv;
  return dispatch(h, [&](auto& S) {
    using T = typename std::decay<decltype(S.dts)>::type;
    if (row_a < 0 || row_b >= S.nrow || row_a > row_b) return -1;
    const int64_t plane = (int64_t)S.nrow * S.nth;
    T emax = T(0.0), vmax = T(0.0);
    for (int c = 0; c < 4; ++c)
      for (int i = row_a; i <= row_b; ++i)
        for (int j = 0; j < S.nth; ++j) {
          const int64_t k = (int64_t)i * S.nth + j;
          const T g = from_words<T>(planes + ((int64_t)c * words) * plane + k, words, plane);
          const T e = abs_(g - S.u[c][k]);
          const T v = abs_(S.u[c][k]);
          if (emax < e) emax = e;
          if (vmax < v) vmax = v;
        }
    *umax = to_d(vmax);
    *err = (to_d(vmax) > 0) ? to_d(emax / vmax) : to_d(emax);
    return 0;
  });
}

}  // extern "C"

extern "C" {

// L_th f = f_thth + cot(th) f_th applied to one theta row f (word expansions, [words][nth]) on
// the cell-centred grid of nth cells, with parity ghosts and the given order: out [out_words][nth].
int oracle_theta_op(int bits, int nth, int order, int parity, const double* f, int words, double* out,
                    int out_words) {
  oracle_params p{};
  p.M = 1; p.a = 0; p.s = 0; p.m = 0; p.rstar_min = -1; p.rstar_max = 1; p.n_r = 3; p.n_theta = nth;
  p.dt = 0.1; p.substeps = 1; p.theta_order = order; p.parity = parity; p.row_lo = 0; p.row_hi = 2;
  Handle* h = (Handle*)oracle_create(&p, bits);
  if (!h) return -1;
  int rc = dispatch(h, [&](auto& S) {
    using T = typename std::decay<decltype(S.dts)>::type;
    std::vector<T> row(nth);
    for (int j = 0; j < nth; ++j) row[j] = from_words<T>(f + j, words, nth);
    for (int j = 0; j < nth; ++j) to_words(S.theta_op(row.data(), j), out + j, out_words, nth);
    return 0;
  });
  oracle_destroy(h);
  return rc;
}

// The unnormalised spin-weighted profile used for the initial data, at the grid's theta_j:
// out [out_words][nth].
int oracle_spin_profile(int bits, int s, int m, int ell, int nth, double* out, int out_words) {
  oracle_params p{};
  p.M = 1; p.a = 0; p.s = s; p.m = m; p.rstar_min = -1; p.rstar_max = 1; p.n_r = 3; p.n_theta = nth;
  p.dt = 0.1; p.substeps = 1; p.theta_order = 10; p.parity = 1; p.row_lo = 0; p.row_hi = 2;
  Handle* h = (Handle*)oracle_create(&p, bits);
  if (!h) return -1;
  int rc = dispatch(h, [&](auto& S) {
    for (int j = 0; j < nth; ++j) to_words(S.spin_profile(ell, S.th[j]), out + j, out_words, nth);
    return 0;
  });
  oracle_destroy(h);
  return rc;
}

}  // extern "C"

namespace {

// ------------------------------------------------------------------------------------
// Multipoles of the observed field (Sec. 3.C, Fig. 1): the tail of each multipole l is
// read from c_l(t) = 2 pi int_0^pi Phi(t, theta) sY_lm(theta) sin(theta) dtheta.
// ------------------------------------------------------------------------------------

// Fejer's first quadrature rule on [-1, 1] with the N nodes x_j = cos(theta_j),
// theta_j = (j + 1/2) pi / N (the solver's cell centres):
//   w_j = (2/N) [1 - 2 sum_{k=1}^{floor(N/2)} cos(2 k theta_j) / (4 k^2 - 1)].
template <class T>
T fejer_weight(int N, int j) {
  const T th = (T(double(j)) + T(0.5)) * pi_<T>() / T(double(N));
  T sum = T(0.0);
  for (int k = 1; k <= N / 2; ++k) sum = sum + cos_(T(2.0 * k) * th) / T(4.0 * k * k - 1.0);
  return T(2.0) / T(double(N)) * (T(1.0) - T(2.0) * sum);
}

// n! as an exact product in T (exact in double up to 18!, in 256-bit MPFR far beyond).
template <class T>
T factorial(int n) {
  T r = T(1.0);
  for (int t = 2; t <= n; ++t) r = r * T(double(t));
  return r;
}

// Binomial coefficient C(n, k) as a ratio of factorials in T (0 outside 0 <= k <= n).
template <class T>
T binomial(int n, int k) {
  if (n < 0 || k < 0 || k > n) return T(0.0);
  return factorial<T>(n) / (factorial<T>(k) * factorial<T>(n - k));
}

// Normalised spin-weighted spherical harmonic at phi = 0 (Goldberg et al. 1967):
//   sY_lm = (-1)^m sqrt((2l+1)/(4 pi) (l+m)!(l-m)!/((l+s)!(l-s)!))
//           sum_r C(l-s, r) C(l+s, r+s-m) (-1)^(l-r-s) sin(th/2)^(2l-2r-s+m) cos(th/2)^(2r+s-m).
template <class T>
T swsh(int s, int m, int l, const T& theta) {
  const T sh = sin_(theta * T(0.5)), ch = cos_(theta * T(0.5));
  T sum = T(0.0);
  for (int r = 0; r <= l - s; ++r) {
    const T c = binomial<T>(l - s, r) * binomial<T>(l + s, r + s - m);
    T term = ((l - r - s) % 2 == 0) ? c : -c;
    for (int e = 0; e < 2 * l - 2 * r - s + m; ++e) term = term * sh;
    for (int e = 0; e < 2 * r + s - m; ++e) term = term * ch;
    sum = sum + term;
  }
  const T norm = sqrt_(T(double(2 * l + 1)) / (T(4.0) * pi_<T>()) * factorial<T>(l + m) * factorial<T>(l - m) /
                       (factorial<T>(l + s) * factorial<T>(l - s)));
  return (m % 2 == 0 ? norm : -norm) * sum;
}

// c[t][l][part] = 2 pi sum_j w_j sY_lm(theta_j) Phi[t][part][j] for samples given as word
// expansions [n][2][words][nth]; out [n][n_ell][2][out_words].
template <class T>
void project(int s, int m, int nth, int ell_min, int ell_max, const double* samples, int words, int64_t n,
             double* out, int out_words) {
  const int n_ell = ell_max - ell_min + 1;
  const T pi = pi_<T>();
  std::vector<T> tab((size_t)n_ell * nth);
  for (int l = ell_min; l <= ell_max; ++l)
    for (int j = 0; j < nth; ++j) {
      const T th = (T(double(j)) + T(0.5)) * pi / T(double(nth));
      tab[(size_t)(l - ell_min) * nth + j] = T(2.0) * pi * fejer_weight<T>(nth, j) * swsh<T>(s, m, l, th);
    }
#pragma omp parallel for schedule(dynamic)
  for (int64_t t = 0; t < n; ++t)
    for (int l = 0; l < n_ell; ++l)
      for (int part = 0; part < 2; ++part) {
        const double* f = samples + ((size_t)t * 2 + part) * words * nth;
        T acc = T(0.0);
        for (int j = 0; j < nth; ++j) acc = acc + tab[(size_t)l * nth + j] * from_words<T>(f + j, words, nth);
        to_words(acc, out + (((size_t)t * n_ell + l) * 2 + part) * out_words, out_words, 1);
      }
}

}  // namespace

extern "C" {

// Fejer weights of the nth-cell grid: out [out_words][nth].
int oracle_fejer_weights(int bits, int nth, double* out, int out_words) {
  if (nth < 1) return -1;
  if (bits <= 53) {
    for (int j = 0; j < nth; ++j) to_words(fejer_weight<double>(nth, j), out + j, out_words, nth);
    return 0;
  }
  g_bits = bits;
  for (int j = 0; j < nth; ++j) to_words(fejer_weight<mp>(nth, j), out + j, out_words, nth);
  return 0;
}

// Normalised sY_lm at the given angles: out [out_words][n].
int oracle_swsh(int bits, int s, int m, int ell, int n, const double* theta, double* out, int out_words) {
  if (ell < std::abs(s) || ell < std::abs(m)) return -1;
  if (bits <= 53) {
    for (int j = 0; j < n; ++j) to_words(swsh<double>(s, m, ell, theta[j]), out + j, out_words, n);
    return 0;
  }
  g_bits = bits;
  for (int j = 0; j < n; ++j) to_words(swsh<mp>(s, m, ell, mp(theta[j])), out + j, out_words, n);
  return 0;
}

// Multipoles of recorded samples (see project above).
int oracle_project(int bits, int s, int m, int nth, int ell_min, int ell_max, const double* samples, int words,
                   int64_t n, double* out, int out_words) {
  if (ell_min < std::abs(s) || ell_min < std::abs(m) || ell_max < ell_min || nth < 1) return -1;
  if (bits <= 53) {
    project<double>(s, m, nth, ell_min, ell_max, samples, words, n, out, out_words);
    return 0;
  }
  g_bits = bits;
  project<mp>(s, m, nth, ell_min, ell_max, samples, words, n, out, out_words);
  return 0;
}

}  // extern "C"

extern "C" {

// Test-only forcing of the Pi equation for manufactured solutions (not part of the method):
// Pi_t - b Pi' = S_Pi + e^{-i omega t} F^, with F^ given as doubles at the window's nodes,
// fn [2 (re, im)][nrow][nth], and half nodes, fh [2][nrow-1][nth]. Eqs. lw1 / lw2 take it at
// t_n at half nodes and at t_n + dt/2 at nodes, like the rest of S. NULL tables switch it off.
int oracle_set_forcing(void* hv, double omega, const double* fn, const double* fh) {
  Handle* h = (Handle*)hv;
  return dispatch(h, [&](auto& S) {
    using T = typename std::decay<decltype(S.dts)>::type;
    if (!fn || !fh) {
      S.forced = false;
      return 0;
    }
    const size_t pn = (size_t)S.nrow * S.nth, ph = (size_t)(S.nrow - 1) * S.nth;
    for (int part = 0; part < 2; ++part) {
      S.fn[part].resize(pn);
      S.fh[part].resize(ph);
      for (size_t k = 0; k < pn; ++k) S.fn[part][k] = T(fn[part * pn + k]);
      for (size_t k = 0; k < ph; ++k) S.fh[part][k] = T(fh[part * ph + k]);
    }
    S.f_omega = T(omega);
    S.forced = true;
    return 0;
  });
}

// Overwrites one theta row of the state (window-relative row index) from in [4][words][nth]:
// used to place halo rows received from a neighbouring slab.
// Applies the theta filter to the current state (as at the start of an outer step); -1 if the
// problem has no filter.
int oracle_filter_rows(void* hv) {
  return dispatch((Handle*)hv, [&](auto& S) {
    if (S.p.theta_filter <= 0) return -1;
    S.filter_rows();
    return 0;
  });
}

int oracle_set_row(void* hv, int row, const double* in, int words) {
  Handle* h = (Handle*)hv;
  return dispatch(h, [&](auto& S) {
    using T = typename std::decay<decltype(S.dts)>::type;
    if (row < 0 || row >= S.nrow) return -1;
    for (int c = 0; c < 4; ++c)
      for (int j = 0; j < S.nth; ++j)
        S.u[c][(size_t)row * S.nth + j] = from_words<T>(in + ((int64_t)c * words) * S.nth + j, words, S.nth);
    return 0;
  });
}

}  // extern "C"
