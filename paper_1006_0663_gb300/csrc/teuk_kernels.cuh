// Device kernels of the Lax-Wendroff Teukolsky step (arXiv:1006.0663, Sec. 3.B-3.D), one
// template per arithmetic: W = 1 (FP64), 2 (double-double), 4 (quad-double).
//
// Data layout in HBM ("SoA word planes"): a field with C components on R rows is stored as
// [C][W][R][pitch] doubles, theta fastest, pitch = n_theta rounded up to 16 doubles (128 B),
// so every warp access along theta is one coalesced 128-byte line per word plane.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "mw_func.cuh"

namespace teuk {

template <int W> struct RT;
template <> struct RT<1> { using T = double; };
template <> struct RT<2> { using T = mw::dd; };
template <> struct RT<4> { using T = mw::qd; };

// ---- word-plane access -------------------------------------------------------------------
template <class R> __device__ __forceinline__ R ld_r(const double* __restrict__ p, size_t ws);
template <> __device__ __forceinline__ double ld_r<double>(const double* __restrict__ p, size_t) {
  return __ldg(p);
}
template <> __device__ __forceinline__ mw::dd ld_r<mw::dd>(const double* __restrict__ p, size_t ws) {
  return mw::dd{__ldg(p), __ldg(p + ws)};
}
template <> __device__ __forceinline__ mw::qd ld_r<mw::qd>(const double* __restrict__ p, size_t ws) {
  return mw::qd{__ldg(p), __ldg(p + ws), __ldg(p + 2 * ws), __ldg(p + 3 * ws)};
}
// plain (non-__ldg) loads for buffers written earlier in the same kernel
template <class R> __device__ __forceinline__ R ld_s(const double* p, size_t ws);
template <> __device__ __forceinline__ double ld_s<double>(const double* p, size_t) { return p[0]; }
template <> __device__ __forceinline__ mw::dd ld_s<mw::dd>(const double* p, size_t ws) {
  return mw::dd{p[0], p[ws]};
}
template <> __device__ __forceinline__ mw::qd ld_s<mw::qd>(const double* p, size_t ws) {
  return mw::qd{p[0], p[ws], p[2 * ws], p[3 * ws]};
}
__device__ __forceinline__ void st_r(double* p, size_t, double v) { p[0] = v; }
__device__ __forceinline__ void st_r(double* p, size_t ws, mw::dd v) { p[0] = v.h; p[ws] = v.l; }
__device__ __forceinline__ void st_r(double* p, size_t ws, mw::qd v) {
  p[0] = v.x0; p[ws] = v.x1; p[2 * ws] = v.x2; p[3 * ws] = v.x3;
}
template <class R> __host__ __device__ __forceinline__ R from_words(const double* w);
template <> __host__ __device__ __forceinline__ double from_words<double>(const double* w) { return w[0]; }
template <> __host__ __device__ __forceinline__ mw::dd from_words<mw::dd>(const double* w) { return mw::dd{w[0], w[1]}; }
template <> __host__ __device__ __forceinline__ mw::qd from_words<mw::qd>(const double* w) {
  return mw::qd{w[0], w[1], w[2], w[3]};
}
__host__ __device__ __forceinline__ void to_words(double v, double* w) { w[0] = v; w[1] = w[2] = w[3] = 0.0; }
__host__ __device__ __forceinline__ void to_words(mw::dd v, double* w) { w[0] = v.h; w[1] = v.l; w[2] = w[3] = 0.0; }
__host__ __device__ __forceinline__ void to_words(mw::qd v, double* w) { w[0] = v.x0; w[1] = v.x1; w[2] = v.x2; w[3] = v.x3; }

// ---- hot-path arithmetic ---------------------------------------------------------------------
__host__ __device__ __forceinline__ double v_add(double a, double b) { return a + b; }
__host__ __device__ __forceinline__ double v_sub(double a, double b) { return a - b; }
__host__ __device__ __forceinline__ double v_half(double a) { return 0.5 * a; }
__host__ __device__ __forceinline__ double v_neg(double a) { return -a; }
__host__ __device__ __forceinline__ mw::dd v_add(mw::dd a, mw::dd b) { return mw::dd_add_accurate(a, b); }
__host__ __device__ __forceinline__ mw::dd v_sub(mw::dd a, mw::dd b) { return mw::dd_sub_accurate(a, b); }
__host__ __device__ __forceinline__ mw::dd v_half(mw::dd a) { return mw::dd_scale2(a, 0.5); }
__host__ __device__ __forceinline__ mw::dd v_neg(mw::dd a) { return mw::dd_neg(a); }
__host__ __device__ __forceinline__ mw::qd v_add(mw::qd a, mw::qd b) { return mw::qd_add(a, b); }
__host__ __device__ __forceinline__ mw::qd v_sub(mw::qd a, mw::qd b) { return mw::qd_sub(a, b); }
__host__ __device__ __forceinline__ mw::qd v_half(mw::qd a) { return mw::qd_scale2(a, 0.5); }
__host__ __device__ __forceinline__ mw::qd v_neg(mw::qd a) { return mw::qd_neg(a); }

// Dot-product accumulators: acc = x0 + sum_k c_k v_k.
//   FP64: one FMA per term.
//   dd: Ogita-Rump-Oishi "Dot2" (SIAM J. Sci. Comput. 26, 2005) extended to double-word
//       operands: each product's leading part is formed exactly by TwoProd, the cross terms
//       c.h v.l + c.l v.h go into its error, the leading parts are summed by TwoSum and all
//       errors are gathered in one low-order word; one final TwoSum renormalises.
//   qd: quad-double multiply-add per term.
template <class R> struct Acc;
template <> struct Acc<double> {
  double s;
  __host__ __device__ __forceinline__ explicit Acc(double x0) : s(x0) {}
  __host__ __device__ __forceinline__ void mac(double c, double v) { s = mw::fma_(c, v, s); }
  __host__ __device__ __forceinline__ double get() const { return s; }
};
template <> struct Acc<mw::dd> {
  double s, e;
  __host__ __device__ __forceinline__ explicit Acc(mw::dd x0) : s(x0.h), e(x0.l) {}
  __host__ __device__ __forceinline__ void mac(mw::dd c, mw::dd v) {
    double p, pe, t;
    mw::two_prod(c.h, v.h, p, pe);
    pe = mw::fma_(c.h, v.l, pe);
    pe = mw::fma_(c.l, v.h, pe);
    mw::two_sum_ord(s, p, s, t);
    e = mw::add_(e, mw::add_(t, pe));
  }
  __host__ __device__ __forceinline__ mw::dd get() const {
    mw::dd r;
    mw::two_sum_ord(s, e, r.h, r.l);
    return r;
  }
};
// qd: the product c v of two quad-doubles is split by order of magnitude (c_i v_j is of
// order i + j): order-0..2 products are formed exactly by TwoProd, order-3 products rounded,
// higher orders dropped (as in HLB01's multiplication). Each order has its own running sum;
// every TwoSum into level k sends its exact error to level k + 1, level 3 is summed plainly,
// and one renormalisation at the end turns the four levels into a quad-double. The result
// equals the quad-double dot product to about 2^-200 of sum |c_k v_k|, at ~70 FP64
// operations per term instead of a quad-double multiply plus add (~168).
template <> struct Acc<mw::qd> {
  double l0, l1, l2, l3;
  __host__ __device__ __forceinline__ explicit Acc(mw::qd x0) : l0(x0.x0), l1(x0.x1), l2(x0.x2), l3(x0.x3) {}
  __host__ __device__ __forceinline__ void mac(mw::qd c, mw::qd v) {
    using namespace mw;
    double p00, e00, p01, e01, p10, e10, p02, e02, p11, e11, p20, e20, t;
    two_prod(c.x0, v.x0, p00, e00);
    two_prod(c.x0, v.x1, p01, e01);
    two_prod(c.x1, v.x0, p10, e10);
    two_prod(c.x0, v.x2, p02, e02);
    two_prod(c.x1, v.x1, p11, e11);
    two_prod(c.x2, v.x0, p20, e20);
    // level 0
    two_sum_ord(l0, p00, l0, t);
    // level 1: t, e00, p01, p10
    double q0, q1, q2, q3;
    two_sum_ord(l1, t, l1, q0);
    two_sum_ord(l1, e00, l1, q1);
    two_sum_ord(l1, p01, l1, q2);
    two_sum_ord(l1, p10, l1, q3);
    // level 2: q0..q3, e01, e10, p02, p11, p20
    double r0, r1, r2, r3, r4, r5, r6, r7, r8;
    two_sum_ord(l2, q0, l2, r0);
    two_sum_ord(l2, q1, l2, r1);
    two_sum_ord(l2, q2, l2, r2);
    two_sum_ord(l2, q3, l2, r3);
    two_sum_ord(l2, e01, l2, r4);
    two_sum_ord(l2, e10, l2, r5);
    two_sum_ord(l2, p02, l2, r6);
    two_sum_ord(l2, p11, l2, r7);
    two_sum_ord(l2, p20, l2, r8);
    // level 3: rounded
    double s3 = add_(add_(add_(r0, r1), add_(r2, r3)), add_(add_(r4, r5), add_(r6, r7)));
    s3 = add_(s3, add_(r8, add_(add_(e02, e11), e20)));
    s3 = fma_(c.x0, v.x3, s3);
    s3 = fma_(c.x1, v.x2, s3);
    s3 = fma_(c.x2, v.x1, s3);
    s3 = fma_(c.x3, v.x0, s3);
    l3 = add_(l3, s3);
  }
  __host__ __device__ __forceinline__ mw::qd get() const { return mw::qd_renorm(l0, l1, l2, l3, 0.0); }
};

// ---- kernel argument blocks ---------------------------------------------------------------
struct Geom {
  int n_r, n_th, pitch, parity;
};

struct SetupArgs {
  Geom g;
  int row0;      // global index of local row 0 (0 unless the handle holds an r* slab)
  int W;
  double M, a;
  int s, m;
  double rp[4], rm[4], tort_A[4], tort_B[4], ln2[4], ln2M[4], rsmin[4], dr[4];
  double dts[4], lambda[4];  // substep dt and dt/dr
  const double* sin_th;      // [W][n_th]
  const double* cos_th;      // [W][n_th]
  double* x_node;            // [W][n_r]
  double* x_half;            // [W][n_r-1]
  double* rs_node;           // [W][n_r]
  double* cn_raw;            // [8][W][n_r][pitch]
  double* ch_raw;            // [8][W][n_r-1][pitch]
  double* cn;                // folded node coefficients
  double* ch;                // folded half coefficients
};

// ---- set-up kernels ---------------------------------------------------------------------------
// Tortoise inversion (Sec. 3.B): r*(x) = r+ + x + A ln(x/2M) + B ln((x + r+ - r-)/2M) with
// x = r - r+; solved for x at every node and half node by Newton's method in xi = ln x,
// started from a bisection in double precision.
template <int W>
__global__ void tortoise_kernel(SetupArgs a) {
  using R = typename RT<W>::T;
  const int n_nodes = a.g.n_r, n_half = a.g.n_r - 1;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_nodes + n_half) return;
  const bool half = t >= n_nodes;
  const int i = half ? t - n_nodes : t;
  const R rp = from_words<R>(a.rp), rm = from_words<R>(a.rm);
  const R A = from_words<R>(a.tort_A), B = from_words<R>(a.tort_B);
  const R ln2 = from_words<R>(a.ln2), ln2M = from_words<R>(a.ln2M);
  const R dr = from_words<R>(a.dr);
  const double fi = half ? double(i + a.row0) + 0.5 : double(i + a.row0);  // exact
  const R target = mw::r_add(from_words<R>(a.rsmin), mw::r_mul_d(dr, fi));
  const R twoM = mw::r_from<R>(2.0 * a.M);
  // double-precision bracket
  const double td = mw::lead(target), rpd = mw::lead(rp), rmd = mw::lead(rm);
  const double Ad = mw::lead(A), Bd = mw::lead(B), l2M = std::log(2.0 * a.M);
  double lo = -745.0, hi = 45.0;
  for (int it = 0; it < 120; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double x = exp(mid);
    const double F = rpd + x + Ad * (mid - l2M) + Bd * log((x + rpd - rmd) / (2.0 * a.M)) - td;
    if (F < 0) lo = mid; else hi = mid;
  }
  R xi = mw::r_from<R>(0.5 * (lo + hi));
  const int nit = W == 1 ? 3 : (W == 2 ? 3 : 4);
  R x = mw::r_exp(xi, ln2);
  for (int it = 0; it < nit; ++it) {
    const R q = mw::r_add(x, mw::r_sub(rp, rm));
    const R F = mw::r_sub(mw::r_add(mw::r_add(rp, x),
                                    mw::r_add(mw::r_mul(A, mw::r_sub(xi, ln2M)),
                                              mw::r_mul(B, mw::r_log(mw::r_div(q, twoM), ln2)))),
                          target);
    const R dF = mw::r_add(mw::r_add(x, A), mw::r_div(mw::r_mul(B, x), q));
    xi = mw::r_sub(xi, mw::r_div(F, dF));
    x = mw::r_exp(xi, ln2);
  }
  double w[4];
  to_words(x, w);
  double* out = half ? a.x_half : a.x_node;
  const int rows = half ? n_half : n_nodes;
  for (int k = 0; k < W; ++k) out[(size_t)k * rows + i] = w[k];
  if (!half) {
    to_words(target, w);
    for (int k = 0; k < W; ++k) a.rs_node[(size_t)k * n_nodes + i] = w[k];
  }
}

// Coefficients of the first-order system at (x = r - r+, theta_j), from the Teukolsky
// equation (Eq. 1) with Psi = e^{i m phi~} r^3 Phi and Pi = Phi_t + b Phi' (Sec. 3.B):
//   R = r^2 + a^2, Delta = x (x + r+ - r-), Sigma^2 = R^2 - a^2 Delta sin^2 th, b = R/Sigma,
//   B = 4 i M a m r + 2 s [Delta (r + i a cos th) - M (r^2 - a^2)],
//   C = 2 r Delta + 2 s (r - M) R + 2 i m a R,
//   V = R^2 f''/f + C f'/f + 4 i s m a (r - M) + Delta [s - (m + s cos th)^2 / sin^2 th],
//   f'/f = 3 Delta/(r R), f''/f = 6 Delta [(r - M) r R + a^2 Delta]/(r^2 R^3),
//   c = a^2 Delta sin^2 th [R (r - M) - 2 r Delta]/Sigma^4 - (b B + 6 R Delta/r + C)/Sigma^2.
// Stored: b, c_R, c_I, Re B/S^2, Im B/S^2, Delta/S^2, Re V/S^2, Im V/S^2.
template <class R>
__device__ void system_coeffs(const SetupArgs& a, R x, R sn, R cs, R out[8]) {
  using namespace mw;
  const R M = r_from<R>(a.M), av = r_from<R>(a.a);
  const double s = a.s, m = a.m;
  const R rp = from_words<R>(a.rp), rm = from_words<R>(a.rm);
  const R r = r_add(rp, x);
  const R Delta = r_mul(x, r_add(x, r_sub(rp, rm)));
  const R a2 = r_mul(av, av);
  const R r2 = r_mul(r, r);
  const R Rr = r_add(r2, a2);
  const R sn2 = r_mul(sn, sn);
  const R Sig2 = r_sub(r_mul(Rr, Rr), r_mul(r_mul(a2, Delta), sn2));
  const R b = r_div(Rr, r_sqrt(Sig2));
  const R rR = r_mul(r, Rr);
  const R fp = r_div(r_mul_d(Delta, 3.0), rR);
  const R rmM = r_sub(r, M);
  const R fpp = r_div(r_mul_d(r_mul(Delta, r_add(r_mul(rmM, rR), r_mul(a2, Delta))), 6.0),
                      r_mul(r_mul(rR, rR), Rr));
  const R B_R = r_mul_d(r_sub(r_mul(Delta, r), r_mul(M, r_sub(r2, a2))), 2.0 * s);
  const R B_I = r_add(r_mul_d(r_mul(r_mul(M, av), r), 4.0 * m), r_mul_d(r_mul(r_mul(av, Delta), cs), 2.0 * s));
  const R C_R = r_add(r_mul_d(r_mul(r, Delta), 2.0), r_mul_d(r_mul(rmM, Rr), 2.0 * s));
  const R C_I = r_mul_d(r_mul(av, Rr), 2.0 * m);
  const R msc = r_add(r_from<R>(m), r_mul_d(cs, s));
  const R pot = r_mul(Delta, r_sub(r_from<R>(s), r_div(r_mul(msc, msc), sn2)));
  const R V_R = r_add(r_add(r_mul(r_mul(Rr, Rr), fpp), r_mul(C_R, fp)), pot);
  const R V_I = r_add(r_mul(C_I, fp), r_mul_d(r_mul(av, rmM), 4.0 * s * m));
  const R bbp = r_div(r_mul(r_mul(r_mul(a2, Delta), sn2), r_sub(r_mul(Rr, rmM), r_mul_d(r_mul(r, Delta), 2.0))),
                      r_mul(Sig2, Sig2));
  const R c_R = r_sub(bbp, r_div(r_add(r_add(r_mul(b, B_R), r_mul_d(r_div(r_mul(Rr, Delta), r), 6.0)), C_R), Sig2));
  const R c_I = r_neg(r_div(r_add(r_mul(b, B_I), C_I), Sig2));
  out[0] = b;
  out[1] = c_R;
  out[2] = c_I;
  out[3] = r_div(B_R, Sig2);
  out[4] = r_div(B_I, Sig2);
  out[5] = r_div(Delta, Sig2);
  out[6] = r_div(V_R, Sig2);
  out[7] = r_div(V_I, Sig2);
}

// Raw coefficients at every node / half node, and the per-substep folded tables:
//   half node:  H0 = l b/2, H1 = -h c_R/(2dr), H2 = h c_I/(2dr), H3 = 1/2 - h bR/4,
//               H4 = h bI/4, H5 = h g/4, H6 = h nR/4, H7 = h nI/4
//   node:       N0 = l b,   N1 = -h c_R/dr,    N2 = h c_I/dr,    N3 = -h bR/2,
//               N4 = h bI/2, N5 = h g/2, N6 = h nR/2, N7 = h nI/2
// with h = dt/k, l = h/dr, bR + i bI = B/Sigma^2, g = Delta/Sigma^2, nR + i nI = V/Sigma^2.
template <int W>
__global__ void coeff_kernel(SetupArgs a, int half) {
  using R = typename RT<W>::T;
  using namespace mw;
  const int rows = half ? a.g.n_r - 1 : a.g.n_r;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= a.g.n_th || i >= rows) return;
  const double* xs = half ? a.x_half : a.x_node;
  double w[4] = {0, 0, 0, 0};
  for (int k = 0; k < W; ++k) w[k] = xs[(size_t)k * rows + i];
  const R x = from_words<R>(w);
  for (int k = 0; k < W; ++k) w[k] = a.sin_th[(size_t)k * a.g.n_th + j];
  const R sn = from_words<R>(w);
  for (int k = 0; k < W; ++k) w[k] = a.cos_th[(size_t)k * a.g.n_th + j];
  const R cs = from_words<R>(w);
  R c[8];
  system_coeffs<R>(a, x, sn, cs, c);
  const size_t ws = (size_t)rows * a.g.pitch;
  const size_t base = (size_t)i * a.g.pitch + j;
  double* raw = half ? a.ch_raw : a.cn_raw;
  for (int q = 0; q < 8; ++q) st_r(raw + (size_t)q * W * ws + base, ws, c[q]);
  const R h = from_words<R>(a.dts), lam = from_words<R>(a.lambda);
  const R hdr = r_div(h, from_words<R>(a.dr));
  R f[8];
  if (half) {
    f[0] = r_scale2(r_mul(lam, c[0]), 0.5);
    f[1] = r_neg(r_scale2(r_mul(hdr, c[1]), 0.5));
    f[2] = r_scale2(r_mul(hdr, c[2]), 0.5);
    f[3] = r_sub(r_from<R>(0.5), r_scale2(r_mul(h, c[3]), 0.25));
    f[4] = r_scale2(r_mul(h, c[4]), 0.25);
    f[5] = r_scale2(r_mul(h, c[5]), 0.25);
    f[6] = r_scale2(r_mul(h, c[6]), 0.25);
    f[7] = r_scale2(r_mul(h, c[7]), 0.25);
  } else {
    f[0] = r_mul(lam, c[0]);
    f[1] = r_neg(r_mul(hdr, c[1]));
    f[2] = r_mul(hdr, c[2]);
    f[3] = r_neg(r_scale2(r_mul(h, c[3]), 0.5));
    f[4] = r_scale2(r_mul(h, c[4]), 0.5);
    f[5] = r_scale2(r_mul(h, c[5]), 0.5);
    f[6] = r_scale2(r_mul(h, c[6]), 0.5);
    f[7] = r_scale2(r_mul(h, c[7]), 0.5);
  }
  double* fold = half ? a.ch : a.cn;
  for (int q = 0; q < 8; ++q) st_r(fold + (size_t)q * W * ws + base, ws, f[q]);
}

struct PulseArgs {
  Geom g;
  int row0, n_r_global;   // global index of local row 0; rows of the whole grid
  double center, width, amp_re, amp_im;
  double ln2[4];
  const double* rs_node;  // [W][n_r]
  const double* prof;     // [W][n_th] angular profile sY(theta_j)
  const double* cn_raw;   // b at nodes = plane 0
  double* u;              // [4][W][n_r][pitch]
};

// Initial data: Phi = A exp(-((r* - c)/w)^2) sY(theta), zero time derivative so that
// Pi = b Phi_{r*} = b A G'(r*) sY(theta), G' = -2 (r* - c)/w^2 G. Boundary rows stay zero.
template <int W>
__global__ void pulse_kernel(PulseArgs a) {
  using R = typename RT<W>::T;
  using namespace mw;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (j >= a.g.n_th || i >= a.g.n_r) return;
  const size_t ws = (size_t)a.g.n_r * a.g.pitch;
  const size_t idx = (size_t)i * a.g.pitch + j;
  if (i + a.row0 == 0 || i + a.row0 == a.n_r_global - 1) {  // r* boundary rows (Sec. 3.B)
    for (int c = 0; c < 4; ++c) st_r(a.u + (size_t)c * W * ws + idx, ws, r_from<R>(0.0));
    return;
  }
  double w[4] = {0, 0, 0, 0};
  for (int k = 0; k < W; ++k) w[k] = a.rs_node[(size_t)k * a.g.n_r + i];
  const R rs = from_words<R>(w);
  for (int k = 0; k < W; ++k) w[k] = a.prof[(size_t)k * a.g.n_th + j];
  const R Y = from_words<R>(w);
  const R z = r_div_d(r_sub(rs, r_from<R>(a.center)), a.width);
  const R G = r_exp(r_neg(r_mul(z, z)), from_words<R>(a.ln2));
  const R Gp = r_mul(r_neg(r_div_d(r_scale2(z, 2.0), a.width)), G);
  const R b = ld_r<R>(a.cn_raw + idx, ws);
  const R GY = r_mul(G, Y), GpY = r_mul(Gp, Y);
  st_r(a.u + 0 * W * ws + idx, ws, r_mul_d(GY, a.amp_re));
  st_r(a.u + 1 * W * ws + idx, ws, r_mul_d(GY, a.amp_im));
  st_r(a.u + 2 * W * ws + idx, ws, r_mul(b, r_mul_d(GpY, a.amp_re)));
  st_r(a.u + 3 * W * ws + idx, ws, r_mul(b, r_mul_d(GpY, a.amp_im)));
}

// ---- programmatic dependent launch ---------------------------------------------------------
// The FP64 and FP64-error-free-transform step kernels (and the dissipation kernel) are
// launched so that their blocks may be scheduled while the previous kernel of the stream still
// runs (small grids spend more time in launches than in arithmetic: c1 +3 %; the integer
// engine's kernels measured slower that way and are launched normally). Before reading anything that kernel wrote, a kernel waits for it to complete
// and its writes to be visible (a no-op when it was launched without the attribute); only then
// does it let the next kernel be scheduled, so at most two kernels' blocks are resident and
// the earlier one's blocks have all started.
__device__ __forceinline__ void step_dependency() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---- dissipation (not part of the paper's method; off unless enabled) ---------------------
// Once per outer step, before its first Lax-Wendroff iteration, every component becomes
//   u - eps_r d_r^4 u - eps_th(i) d_th^12 u,
// eps_r = sigma_r dt / (16 dr*) (rows 2 .. n_r - 3 only), eps_th(i) = sigma_th c_th(i) dt /
// (4096 dtheta) with c_th(i) = max_j sqrt(Delta/Sigma^2) at node i (rows 1 .. n_r - 2), d_r^4 the
// undivided fourth difference along r* and d_th^12 = (d_th^2)^6 the undivided twelfth
// difference along theta with the parity ghosts: Kreiss-Oliger operators of order 4 and 12
// integrated over one outer step. Both differences read the same input u. Several iterations
// per dt = 0.25 dr* leave the scheme's own damping of short r* wavelengths too weak where the
// lower-order terms of the system make a frozen wave grow; the theta term damps the grid-scale
// theta modes whose frequencies set how many iterations the explicit midpoint-like iteration
// of the theta terms needs.
struct DissArgs {
  Geom g;
  const double* u;       // [4][W][n_r][pitch]
  double* out;           // same layout
  double eps[4];         // eps_r as W words
  int eps_single;        // eps_r is one double (sigma / 64 when dt = 0.25 dr*): a cheaper product
  int do_r;              // apply the r* term
  const double* eps_th;  // [W][n_r] or null: no theta term
};

// (d^2)^6 f_j = sum_q (-1)^q C(12, 6 + q) f_{j+q}: exact small-integer weights.
__device__ __forceinline__ double ko12_weight(int q) {
  constexpr double w[7] = {924, -792, 495, -220, 66, -12, 1};
  return w[q < 0 ? -q : q];
}

template <int W>
__global__ void dissipate_kernel(DissArgs a) {
  using R = typename RT<W>::T;
  step_dependency();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y, c = blockIdx.z;
  if (j >= a.g.n_th) return;
  const int n_th = a.g.n_th;
  const size_t ws = (size_t)a.g.n_r * a.g.pitch, p = (size_t)a.g.pitch;
  const double* base = a.u + (size_t)c * W * ws + (size_t)i * p + j;
  R v = ld_s<R>(base, ws);
  using namespace mw;
  if (a.do_r && i >= 2 && i <= a.g.n_r - 3) {
    R d4 = v_sub(ld_s<R>(base - 2 * p, ws), r_scale2(ld_s<R>(base - p, ws), 4.0));
    d4 = v_add(d4, r_mul_d(v, 6.0));
    d4 = v_sub(d4, r_scale2(ld_s<R>(base + p, ws), 4.0));
    d4 = v_add(d4, ld_s<R>(base + 2 * p, ws));
    v = v_sub(v, a.eps_single ? r_mul_d(d4, a.eps[0]) : r_mul(from_words<R>(a.eps), d4));
  }
  if (a.eps_th && i >= 1 && i <= a.g.n_r - 2) {
    const double* row = base - j;
    Acc<R> acc(r_from<R>(0.0));
#pragma unroll
    for (int q = -6; q <= 6; ++q) {
      int jj = j + q;
      bool ghost = false;
      if (jj < 0) { jj = -1 - jj; ghost = true; }
      else if (jj >= n_th) { jj = 2 * n_th - 1 - jj; ghost = true; }
      R f = ld_s<R>(row + jj, ws);
      if (ghost && a.g.parity < 0) f = v_neg(f);
      acc.mac(r_from<R>(ko12_weight(q)), f);
    }
    double e[4] = {0, 0, 0, 0};
    for (int k = 0; k < W; ++k) e[k] = a.eps_th[(size_t)k * a.g.n_r + i];
    v = v_sub(v, r_mul(from_words<R>(e), acc.get()));
  }
  st_r(a.out + (size_t)c * W * ws + (size_t)i * p + j, ws, v);
}

// ---- theta filter (not part of the paper's method; off unless enabled) ----------------------
// A multipole l oscillates near the photon sphere at about (l + 1/2) / (3 sqrt(3) M). Where
// that exceeds what the central r* differences carry (their frequencies stop at 1/dr*), the
// grid traps the multipole there and the first-order term c Phi' of the r^3-scaled system
// makes it grow. Once per outer step, after the dissipation kernel, every interior row of
// every component is replaced by its projection onto the normalised harmonics sY_lm,
// max(|s|, |m|) <= l < l_cut:
//   f_j <- sum_l sY_l(theta_j) c_l,   c_l = sum_j' 2 pi w_j' sY_l(theta_j') f_j',
// w_j Fejer's first-rule weights on the cell centres. The rule integrates polynomials in
// cos(theta) of degree < n_theta exactly, and sY_l sY_l' of one s and m is such a polynomial
// of degree l + l', so with 2 (l_cut - 1) < n_theta the harmonics are exactly orthonormal in
// this sum and the map is an orthogonal projection.
struct FilterArgs {
  Geom g;
  const double* u;    // [4][W][n_r][pitch]
  double* out;        // same layout; may be u (each block reads its row before writing)
  const double* tab;  // [2][n_ell][W][n_th]: 2 pi w_j sY_l(theta_j), then sY_l(theta_j)
  int n_ell;
  int split;          // partial dot products per coefficient (a power of two)
  long long* ctr;     // [2]: outer steps begun, blocks finished in this launch
  int period;         // project at outer steps whose index is a multiple of period
};

// Shared memory of filter_kernel, in doubles: the row's 4 components, the partial sums, the
// coefficients.
__host__ __device__ inline size_t filter_smem_doubles(int W, int n_th, int n_ell, int split) {
  return (size_t)W * (4 * (size_t)n_th + 4 * (size_t)n_ell * split + 4 * (size_t)n_ell);
}

// One block per interior row, all four components: the row to shared memory; each
// coefficient as `split` interleaved partial dot products in the target precision, added in
// the target precision; then the synthesis, one output per thread. At outer steps that do not
// project, the row is copied to `out` when it is another buffer. The last block to finish
// counts the outer step (every block has read the count before it finishes).
template <int W>
__device__ void filter_row(const FilterArgs& a, double* fsm);

template <int W>
__global__ void filter_kernel(FilterArgs a) {
  extern __shared__ double fsm[];
  __shared__ int project;
  if (threadIdx.x == 0) project = (*(volatile long long*)a.ctr) % a.period == 0;
  __syncthreads();
  if (project) filter_row<W>(a, fsm);
  else if (a.out != a.u) {
    const size_t ws = (size_t)a.g.n_r * a.g.pitch, off = (size_t)(blockIdx.x + 1) * a.g.pitch;
    for (int t = threadIdx.x; t < 4 * W * a.g.n_th; t += blockDim.x) {
      const int pl = t / a.g.n_th, j = t - pl * a.g.n_th;
      a.out[(size_t)pl * ws + off + j] = a.u[(size_t)pl * ws + off + j];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long done = atomicAdd(reinterpret_cast<unsigned long long*>(a.ctr + 1), 1ULL);
    if (done == gridDim.x - 1) {
      a.ctr[1] = 0;
      a.ctr[0] = a.ctr[0] + 1;
    }
  }
}

template <int W>
__device__ void filter_row(const FilterArgs& a, double* fsm) {
  using R = typename RT<W>::T;
  const int i = blockIdx.x + 1;
  const int n_th = a.g.n_th, n_ell = a.n_ell, S = a.split;
  const size_t ws = (size_t)a.g.n_r * a.g.pitch, p = (size_t)a.g.pitch;
  const int n_part = 4 * n_ell * S;
  double* row = fsm;                                 // [4][W][n_th]
  double* part = row + (size_t)4 * W * n_th;         // word planes of stride n_part
  double* coef = part + (size_t)n_part * W;          // [4][W][n_ell]
  for (int t = threadIdx.x; t < 4 * W * n_th; t += blockDim.x) {
    const int c = t / (W * n_th), r = t - c * W * n_th, k = r / n_th, j = r - k * n_th;
    row[t] = a.u[(size_t)(c * W + k) * ws + (size_t)i * p + j];
  }
  __syncthreads();
  const double* ta = a.tab;
  const double* ts = a.tab + (size_t)n_ell * W * n_th;
  for (int t = threadIdx.x; t < n_part; t += blockDim.x) {
    const int q = t % S, cl = t / S, l = cl % n_ell, c = cl / n_ell;
    const double* tl = ta + (size_t)l * W * n_th;
    const double* rc = row + (size_t)c * W * n_th;
    Acc<R> acc(mw::r_from<R>(0.0));
    for (int j = q; j < n_th; j += S) acc.mac(ld_r<R>(tl + j, n_th), ld_s<R>(rc + j, n_th));
    st_r(part + t, n_part, acc.get());
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 4 * n_ell; t += blockDim.x) {
    R sum = ld_s<R>(part + (size_t)t * S, n_part);
    for (int q = 1; q < S; ++q) sum = mw::r_add(sum, ld_s<R>(part + (size_t)t * S + q, n_part));
    const int c = t / n_ell, l = t - c * n_ell;
    st_r(coef + (size_t)c * W * n_ell + l, n_ell, sum);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 4 * n_th; t += blockDim.x) {
    const int c = t / n_th, j = t - c * n_th;
    const double* cc = coef + (size_t)c * W * n_ell;
    Acc<R> acc(mw::r_from<R>(0.0));
    for (int l = 0; l < n_ell; ++l) acc.mac(ld_r<R>(ts + (size_t)l * W * n_th + j, n_th), ld_s<R>(cc + l, n_ell));
    st_r(a.out + (size_t)c * W * ws + (size_t)i * p + j, ws, acc.get());
  }
}

// eps_th(i) = factor * sqrt(max_j g(i, j)), g = Delta/Sigma^2 (plane 5 of the raw node
// coefficients), factor = sigma_th dt / (4096 dtheta); one block per row. The largest g of a
// row is found by comparing the word expansions (normalised, so the words order the values).
template <int W>
__global__ void theta_ko_eps_kernel(Geom g, const double* cn_raw, double* eps_th, double fac0, double fac1,
                                    double fac2, double fac3) {
  using R = typename RT<W>::T;
  __shared__ double best[4][256];
  const int i = blockIdx.x;
  const size_t ws = (size_t)g.n_r * g.pitch;
  const double* plane = cn_raw + (size_t)5 * W * ws + (size_t)i * g.pitch;
  double m[4] = {-1.0, 0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < g.n_th; j += blockDim.x) {
    double v[4] = {0, 0, 0, 0};
    for (int k = 0; k < W; ++k) v[k] = plane[(size_t)k * ws + j];
    bool gt = false;
    for (int k = 0; k < W; ++k) {
      if (v[k] != m[k]) { gt = v[k] > m[k]; break; }
    }
    if (gt) for (int k = 0; k < 4; ++k) m[k] = v[k];
  }
  for (int k = 0; k < 4; ++k) best[k][threadIdx.x] = m[k];
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int t = 1; t < blockDim.x; ++t) {
    bool gt = false;
    for (int k = 0; k < W; ++k) {
      if (best[k][t] != m[k]) { gt = best[k][t] > m[k]; break; }
    }
    if (gt) for (int k = 0; k < 4; ++k) m[k] = best[k][t];
  }
  const double fw[4] = {fac0, fac1, fac2, fac3};
  const R e = mw::r_mul(from_words<R>(fw), mw::r_sqrt(from_words<R>(m)));
  double w[4];
  to_words(e, w);
  for (int k = 0; k < W; ++k) eps_th[(size_t)k * g.n_r + i] = w[k];
}

// ---- multipole projection of the recorded waveform (Sec. 3.C, Fig. 1) ----------------------
struct ProjectArgs {
  int n_th, n_ell;
  long long n, first, cap;  // samples, absolute index of the oldest one, ring capacity
  const double* ring;       // [cap][2][W][n_th]: Phi(i_obs, theta_j) per outer step
  const double* table;      // [n_ell][W][n_th]: quadrature weight x 2 pi x sY_lm(theta_j)
  double* out;              // [n][n_ell][2][W]
};

// c_l(t) = sum_j T_l(theta_j) Phi(t, theta_j): one dot product in the target precision per
// (sample, l, real/imaginary part), so that multipoles tens of orders of magnitude below the
// leading one keep their digits.
template <int W>
__global__ void project_kernel(ProjectArgs a) {
  using R = typename RT<W>::T;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= a.n * a.n_ell * 2) return;
  const int part = (int)(idx % 2);
  const int l = (int)((idx / 2) % a.n_ell);
  const long long t = idx / (2 * a.n_ell);
  const size_t n_th = (size_t)a.n_th;
  const double* src = a.ring + (size_t)((a.first + t) % a.cap) * 2 * W * n_th + (size_t)part * W * n_th;
  const double* tab = a.table + (size_t)l * W * n_th;
  Acc<R> acc(mw::r_from<R>(0.0));
  for (int j = 0; j < a.n_th; ++j) acc.mac(ld_r<R>(tab + j, n_th), ld_s<R>(src + j, n_th));
  double w[4];
  to_words(acc.get(), w);
  for (int k = 0; k < W; ++k) a.out[(size_t)idx * W + k] = w[k];
}

// ---- the Lax-Wendroff substep ----------------------------------------------------------------
struct StepArgs {
  Geom g;
  const double* u_in;      // [4][W][n_r][pitch], level n
  double* u_out;           // same layout, level n+1 (may alias u_in)
  double* uh;              // [4][W][n_r-1][pitch] half-step scratch
  const double* cn;        // folded node tables [8][W][n_r][pitch]
  const double* ch;        // folded half tables [8][W][n_r-1][pitch]
  const double* wts;       // theta stencil weights [11][W][n_th]
  double h4[4], h2[4];     // dt/(4k), dt/(2k)
  int radius;              // 5 (10th order) or 1 (2nd order)
  int record;              // write Phi(i_obs, .) to the ring after this substep
  int i_obs;
  long long ring_slot;     // slot to write, or -1: take it from *ring_counter % ring_cap
  const long long* ring_counter;  // samples recorded so far (device), used when ring_slot < 0
  long long ring_cap;
  double* ring;            // [cap][2][W][n_th]
  unsigned int* status;    // bit 0: non-finite value produced
  size_t uh_ws;            // plane stride of uh in doubles (0: the scratch of n_r - 1 rows)
  int uh_row0;             // half row h is stored at row h - uh_row0 of uh
};

// Plane stride of the half-step rows uh.
__device__ __forceinline__ size_t uh_plane(const StepArgs& a) {
  return a.uh_ws ? a.uh_ws : (size_t)(a.g.n_r - 1) * a.g.pitch;
}

// Centred theta operator at column j on a ghosted shared-memory row (index j + radius is
// column j): sum_q w[q][j] f[j + q], combined second-derivative and cot(th) first-derivative
// weights (Sec. 3.D, 11-point 10th-order stencil; 3-point for 2nd order).
// srow points at the shared-memory entry of column j - RAD of a ghosted row (word stride gstride).
template <class R, int W, int RAD>
__device__ __forceinline__ R theta_op(const double* srow, int gstride, const double* __restrict__ wts,
                                      int n_th, int j) {
  // fully unrolled (compile-time radius): a loop here costs extra FP64 moves per term
  const size_t wws = (size_t)n_th;
  Acc<R> acc(mw::r_from<R>(0.0));
#pragma unroll
  for (int q = 0; q < 2 * RAD + 1; ++q) {
    const R cq = ld_r<R>(wts + (size_t)q * W * wws + j, wws);
    const R vq = ld_s<R>(srow + q, gstride);
    acc.mac(cq, vq);
  }
  return acc.get();
}
template <class R, int W>
__device__ __forceinline__ R theta_op(const double* srow, int gstride, const double* __restrict__ wts,
                                      int n_th, int radius, int j) {
  return radius == 5 ? theta_op<R, W, 5>(srow, gstride, wts, n_th, j)
                     : theta_op<R, W, 1>(srow, gstride, wts, n_th, j);
}

// Writes value v of ghosted row column j, and its parity images across the poles.
template <class R>
__device__ __forceinline__ void put_ghosted(double* srow, int gstride, int n_th, int radius, int parity,
                                            int j, R v) {
  st_r(srow + j + radius, gstride, v);
  const R pv = parity > 0 ? v : v_neg(v);
  if (j < radius) st_r(srow + (radius - 1 - j), gstride, pv);               // column -1-j
  if (j >= n_th - radius) st_r(srow + (2 * n_th - 1 - j) + radius, gstride, pv);  // column 2n-1-j
}

__device__ __forceinline__ bool nonfinite(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7ff) == 0x7ff;
}
__device__ __forceinline__ double lead_of(double x) { return x; }
__device__ __forceinline__ double lead_of(mw::dd x) { return x.h; }
__device__ __forceinline__ double lead_of(mw::qd x) { return x.x0; }

// ---- per-row bodies, shared by the single-problem kernels and the batched kernel ----------
// A row is handled by TX threads along theta (thread tx takes columns tx, tx + TX, ...); sR
// and sI are that row's ghosted shared-memory buffers for the real and imaginary parts.

// Eq. lw1, first phase at half node h: s_Phi = Phi_{h+1} + Phi_h into the ghosted row.
template <int W>
__device__ __forceinline__ void half_row_prep(const StepArgs& a, int h, int tx, int TX, double* sR, double* sI) {
  using R = typename RT<W>::T;
  const int n_r = a.g.n_r, n_th = a.g.n_th, pitch = a.g.pitch, rad = a.radius;
  const int gstride = n_th + 2 * rad;
  const size_t ws = (size_t)n_r * pitch;
  const double* u = a.u_in;
  for (int j = tx; j < n_th; j += TX) {
    const size_t i0 = (size_t)h * pitch + j, i1 = i0 + pitch;
    const R sPR = v_add(ld_s<R>(u + 0 * W * ws + i1, ws), ld_s<R>(u + 0 * W * ws + i0, ws));
    const R sPI = v_add(ld_s<R>(u + 1 * W * ws + i1, ws), ld_s<R>(u + 1 * W * ws + i0, ws));
    put_ghosted<R>(sR, gstride, n_th, rad, a.g.parity, j, sPR);
    put_ghosted<R>(sI, gstride, n_th, rad, a.g.parity, j, sPI);
  }
}

// Eq. lw1 at half nodes h = 0 .. n_r-2:
//   u^{n+1/2}_{h} = (u_{h+1} + u_h)/2 - dt/2 [D (u_{h+1} - u_h)/dr - S(ubar, du)],
// written with the folded tables and s = u_{h+1} + u_h, d = u_{h+1} - u_h:
//   Phi_h  = s_Phi/2 - H0 d_Phi + (h/4) s_Pi,
//   Pi_h,R = H3 s_PiR + H4 s_PiI + H0 d_PiR + H1 d_PhiR + H2 d_PhiI + H5 L(s_Phi)_R + H6 s_PhiR - H7 s_PhiI,
//   Pi_h,I = H3 s_PiI - H4 s_PiR + H0 d_PiI + H1 d_PhiI - H2 d_PhiR + H5 L(s_Phi)_I + H6 s_PhiI + H7 s_PhiR.
// d_Pi is used once, so H0 d_Pi enters the dot product as the two terms H0 Pi_{h+1} and
// -H0 Pi_h (in double-double one Dot2 term costs 9 FP64 operations, an accurate subtraction 14).
// One point (h, j); sRj / sIj point at the ghosted s_Phi entries of column j - radius.
template <int W>
__device__ __forceinline__ void half_point(const StepArgs& a, int h, int j, const double* sRj, const double* sIj,
                                           int gstride) {
  using R = typename RT<W>::T;
  const int n_r = a.g.n_r, n_th = a.g.n_th, pitch = a.g.pitch, rad = a.radius;
  const size_t ws = (size_t)n_r * pitch;
  const size_t hs = (size_t)(n_r - 1) * pitch;
  const double* u = a.u_in;
  const R h4 = from_words<R>(a.h4);
  const size_t i0 = (size_t)h * pitch + j, i1 = i0 + pitch;
  const R uPR0 = ld_s<R>(u + 0 * W * ws + i0, ws), uPR1 = ld_s<R>(u + 0 * W * ws + i1, ws);
  const R uPI0 = ld_s<R>(u + 1 * W * ws + i0, ws), uPI1 = ld_s<R>(u + 1 * W * ws + i1, ws);
  const R uQR0 = ld_s<R>(u + 2 * W * ws + i0, ws), uQR1 = ld_s<R>(u + 2 * W * ws + i1, ws);
  const R uQI0 = ld_s<R>(u + 3 * W * ws + i0, ws), uQI1 = ld_s<R>(u + 3 * W * ws + i1, ws);
  const R sPR = ld_s<R>(sRj + rad, gstride), sPI = ld_s<R>(sIj + rad, gstride);
  const R dPR = v_sub(uPR1, uPR0), dPI = v_sub(uPI1, uPI0);
  const R sQR = v_add(uQR1, uQR0), sQI = v_add(uQI1, uQI0);
  const R LR = theta_op<R, W>(sRj, gstride, a.wts, n_th, rad, j);
  const R LI = theta_op<R, W>(sIj, gstride, a.wts, n_th, rad, j);
  const size_t ci = (size_t)h * pitch + j;
  const size_t us = uh_plane(a), cu = (size_t)(h - a.uh_row0) * pitch + j;
  const R H0 = ld_r<R>(a.ch + 0 * W * hs + ci, hs), H1 = ld_r<R>(a.ch + 1 * W * hs + ci, hs);
  const R H2 = ld_r<R>(a.ch + 2 * W * hs + ci, hs), H3 = ld_r<R>(a.ch + 3 * W * hs + ci, hs);
  const R H4 = ld_r<R>(a.ch + 4 * W * hs + ci, hs), H5 = ld_r<R>(a.ch + 5 * W * hs + ci, hs);
  const R H6 = ld_r<R>(a.ch + 6 * W * hs + ci, hs), H7 = ld_r<R>(a.ch + 7 * W * hs + ci, hs);
  Acc<R> pr(v_half(sPR));
  pr.mac(v_neg(H0), dPR);
  pr.mac(h4, sQR);
  Acc<R> pi(v_half(sPI));
  pi.mac(v_neg(H0), dPI);
  pi.mac(h4, sQI);
  Acc<R> qr(mw::r_from<R>(0.0));
  qr.mac(H3, sQR); qr.mac(H4, sQI); qr.mac(H0, uQR1); qr.mac(v_neg(H0), uQR0); qr.mac(H1, dPR); qr.mac(H2, dPI);
  qr.mac(H5, LR); qr.mac(H6, sPR); qr.mac(v_neg(H7), sPI);
  Acc<R> qi(mw::r_from<R>(0.0));
  qi.mac(H3, sQI); qi.mac(v_neg(H4), sQR); qi.mac(H0, uQI1); qi.mac(v_neg(H0), uQI0); qi.mac(H1, dPI);
  qi.mac(v_neg(H2), dPR);
  qi.mac(H5, LI); qi.mac(H6, sPI); qi.mac(H7, sPR);
  st_r(a.uh + 0 * W * us + cu, us, pr.get());
  st_r(a.uh + 1 * W * us + cu, us, pi.get());
  st_r(a.uh + 2 * W * us + cu, us, qr.get());
  st_r(a.uh + 3 * W * us + cu, us, qi.get());
}

template <int W>
__device__ __forceinline__ void half_row_out(const StepArgs& a, int h, int tx, int TX, const double* sR,
                                             const double* sI, int c0 = 0, int c1 = -1) {
  const int gstride = a.g.n_th + 2 * a.radius;
  if (c1 < 0) c1 = a.g.n_th;
  // columns c0 .. c1-1; two per iteration when a thread owns several: independent dependency
  // chains that the scheduler interleaves (latency of chained FP64 operations)
  int j = c0 + tx;
  for (; j + TX < c1; j += 2 * TX) {
    half_point<W>(a, h, j, sR + j, sI + j, gstride);
    half_point<W>(a, h, j + TX, sR + j + TX, sI + j + TX, gstride);
  }
  if (j < c1) half_point<W>(a, h, j, sR + j, sI + j, gstride);
}

// Eq. lw2, first phase at node i: s_Phi = Phi_{i+1/2} + Phi_{i-1/2} into the ghosted row.
template <int W>
__device__ __forceinline__ void full_row_prep(const StepArgs& a, int i, int tx, int TX, double* sR, double* sI) {
  using R = typename RT<W>::T;
  const int n_r = a.g.n_r, n_th = a.g.n_th, pitch = a.g.pitch, rad = a.radius;
  const int gstride = n_th + 2 * rad;
  (void)n_r;
  const size_t hs = uh_plane(a);
  const double* uh = a.uh;
  for (int j = tx; j < n_th; j += TX) {
    const size_t p = (size_t)(i - a.uh_row0) * pitch + j, m = p - pitch;  // half rows i+1/2 and i-1/2
    const R sPR = v_add(ld_s<R>(uh + 0 * W * hs + p, hs), ld_s<R>(uh + 0 * W * hs + m, hs));
    const R sPI = v_add(ld_s<R>(uh + 1 * W * hs + p, hs), ld_s<R>(uh + 1 * W * hs + m, hs));
    put_ghosted<R>(sR, gstride, n_th, rad, a.g.parity, j, sPR);
    put_ghosted<R>(sI, gstride, n_th, rad, a.g.parity, j, sPI);
  }
}

// Eq. lw2 at nodes i = 1 .. n_r-2 (rows 0 and n_r-1 stay zero, Sec. 3.B):
//   u^{n+1}_i = u^n_i - dt [D (u_{i+1/2} - u_{i-1/2})/dr - S(ubar, du)],
// with s = u_{i+1/2} + u_{i-1/2}, d = u_{i+1/2} - u_{i-1/2} and the folded node tables:
//   Phi'  = Phi - N0 d_Phi + (h/2) s_Pi,
//   Pi'_R = Pi_R + N0 d_PiR + N1 d_PhiR + N2 d_PhiI + N3 s_PiR + N4 s_PiI + N5 L(s_Phi)_R + N6 s_PhiR - N7 s_PhiI,
//   Pi'_I = Pi_I + N0 d_PiI + N1 d_PhiI - N2 d_PhiR + N3 s_PiI - N4 s_PiR + N5 L(s_Phi)_I + N6 s_PhiI + N7 s_PhiR.
// As in the half step, N0 d_Pi enters as the two terms N0 Pi_{i+1/2} and -N0 Pi_{i-1/2}.
// One point (i, j); returns true if a non-finite value was produced. `slot` is the observer
// ring slot to fill (negative: none).
template <int W>
__device__ __forceinline__ bool full_point(const StepArgs& a, int i, int j, const double* sRj, const double* sIj,
                                           int gstride, long long slot) {
  using R = typename RT<W>::T;
  const int n_r = a.g.n_r, n_th = a.g.n_th, pitch = a.g.pitch, rad = a.radius;
  const size_t ws = (size_t)n_r * pitch;
  const size_t hs = uh_plane(a);
  const double* uh = a.uh;
  const R h2 = from_words<R>(a.h2);
  const size_t p = (size_t)(i - a.uh_row0) * pitch + j, m = p - pitch;
  const R hPR1 = ld_s<R>(uh + 0 * W * hs + p, hs), hPR0 = ld_s<R>(uh + 0 * W * hs + m, hs);
  const R hPI1 = ld_s<R>(uh + 1 * W * hs + p, hs), hPI0 = ld_s<R>(uh + 1 * W * hs + m, hs);
  const R hQR1 = ld_s<R>(uh + 2 * W * hs + p, hs), hQR0 = ld_s<R>(uh + 2 * W * hs + m, hs);
  const R hQI1 = ld_s<R>(uh + 3 * W * hs + p, hs), hQI0 = ld_s<R>(uh + 3 * W * hs + m, hs);
  const R sPR = ld_s<R>(sRj + rad, gstride), sPI = ld_s<R>(sIj + rad, gstride);
  const R dPR = v_sub(hPR1, hPR0), dPI = v_sub(hPI1, hPI0);
  const R sQR = v_add(hQR1, hQR0), sQI = v_add(hQI1, hQI0);
  const R LR = theta_op<R, W>(sRj, gstride, a.wts, n_th, rad, j);
  const R LI = theta_op<R, W>(sIj, gstride, a.wts, n_th, rad, j);
  const size_t ci = (size_t)i * pitch + j;
  const R N0 = ld_r<R>(a.cn + 0 * W * ws + ci, ws), N1 = ld_r<R>(a.cn + 1 * W * ws + ci, ws);
  const R N2 = ld_r<R>(a.cn + 2 * W * ws + ci, ws), N3 = ld_r<R>(a.cn + 3 * W * ws + ci, ws);
  const R N4 = ld_r<R>(a.cn + 4 * W * ws + ci, ws), N5 = ld_r<R>(a.cn + 5 * W * ws + ci, ws);
  const R N6 = ld_r<R>(a.cn + 6 * W * ws + ci, ws), N7 = ld_r<R>(a.cn + 7 * W * ws + ci, ws);
  const R PR = ld_s<R>(a.u_in + 0 * W * ws + ci, ws), PI = ld_s<R>(a.u_in + 1 * W * ws + ci, ws);
  const R QR = ld_s<R>(a.u_in + 2 * W * ws + ci, ws), QI = ld_s<R>(a.u_in + 3 * W * ws + ci, ws);
  Acc<R> pr(PR);
  pr.mac(v_neg(N0), dPR);
  pr.mac(h2, sQR);
  Acc<R> pi(PI);
  pi.mac(v_neg(N0), dPI);
  pi.mac(h2, sQI);
  Acc<R> qr(QR);
  qr.mac(N0, hQR1); qr.mac(v_neg(N0), hQR0); qr.mac(N1, dPR); qr.mac(N2, dPI); qr.mac(N3, sQR);
  qr.mac(N4, sQI); qr.mac(N5, LR); qr.mac(N6, sPR); qr.mac(v_neg(N7), sPI);
  Acc<R> qi(QI);
  qi.mac(N0, hQI1); qi.mac(v_neg(N0), hQI0); qi.mac(N1, dPI); qi.mac(v_neg(N2), dPR); qi.mac(N3, sQI);
  qi.mac(v_neg(N4), sQR);
  qi.mac(N5, LI); qi.mac(N6, sPI); qi.mac(N7, sPR);
  const R oPR = pr.get(), oPI = pi.get(), oQR = qr.get(), oQI = qi.get();
  st_r(a.u_out + 0 * W * ws + ci, ws, oPR);
  st_r(a.u_out + 1 * W * ws + ci, ws, oPI);
  st_r(a.u_out + 2 * W * ws + ci, ws, oQR);
  st_r(a.u_out + 3 * W * ws + ci, ws, oQI);
  if (slot >= 0 && i == a.i_obs) {
    double* dst = a.ring + (size_t)slot * 2 * W * n_th;
    st_r(dst + 0 * W * n_th + j, n_th, oPR);
    st_r(dst + 1 * W * n_th + j, n_th, oPI);
  }
  return nonfinite(lead_of(oPR)) | nonfinite(lead_of(oPI)) | nonfinite(lead_of(oQR)) | nonfinite(lead_of(oQI));
}

template <int W>
__device__ __forceinline__ bool full_row_out(const StepArgs& a, int i, int tx, int TX, const double* sR,
                                             const double* sI, long long slot, int c0 = 0, int c1 = -1) {
  const int gstride = a.g.n_th + 2 * a.radius;
  if (c1 < 0) c1 = a.g.n_th;
  bool bad = false;
  int j = c0 + tx;
  for (; j + TX < c1; j += 2 * TX) {
    bad |= full_point<W>(a, i, j, sR + j, sI + j, gstride, slot);
    bad |= full_point<W>(a, i, j + TX, sR + j + TX, sI + j + TX, gstride, slot);
  }
  if (j < c1) bad |= full_point<W>(a, i, j, sR + j, sI + j, gstride, slot);
  return bad;
}

// ---- warp-segment kernels: one warp per (row, 32 theta columns) --------------------------
// Each warp computes the averaged Phi of its 32 columns plus `radius` columns on each side
// (the halo is recomputed, with the parity reflection at the poles), synchronises only
// itself, then produces its 32 points. Thousands of independent warps keep every SM's FP64
// pipe busy to the end of the launch. V selects the register budget (<= 255, 128, 85).
template <int W>
__device__ __forceinline__ void seg_prep(const StepArgs& a, const double* src, size_t plane, int row0, int j0,
                                         int lane, double* sR, double* sI) {
  using R = typename RT<W>::T;
  const int n_th = a.g.n_th, pitch = a.g.pitch, rad = a.radius;
  const int gs = 32 + 2 * rad;
  const int cmax = min(j0 + 31, n_th - 1) + rad;  // last column any lane needs
  for (int idx = lane; idx < gs; idx += 32) {
    const int c = j0 - rad + idx;
    if (c > cmax) continue;
    int cc = c;
    bool ghost = false;
    if (c < 0) { cc = -1 - c; ghost = true; }
    else if (c >= n_th) { cc = 2 * n_th - 1 - c; ghost = true; }
    const size_t k0 = (size_t)row0 * pitch + cc, k1 = k0 + pitch;
    R sPR = v_add(ld_s<R>(src + 0 * W * plane + k1, plane), ld_s<R>(src + 0 * W * plane + k0, plane));
    R sPI = v_add(ld_s<R>(src + 1 * W * plane + k1, plane), ld_s<R>(src + 1 * W * plane + k0, plane));
    if (ghost && a.g.parity < 0) {
      sPR = v_neg(sPR);
      sPI = v_neg(sPI);
    }
    st_r(sR + idx, gs, sPR);
    st_r(sI + idx, gs, sPI);
  }
}

template <int W, int V = 0>
__global__ void __launch_bounds__(128, 2 * (V + 1)) half_seg_kernel(StepArgs a, int nseg) {
  step_dependency();
  extern __shared__ double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int unit = blockIdx.x * (blockDim.x >> 5) + warp;
  const int h = unit / nseg, j0 = (unit % nseg) * 32;
  if (h >= a.g.n_r - 1) return;  // whole warps only: no block-wide barrier below
  const int gs = 32 + 2 * a.radius;
  double* sR = sm + (size_t)warp * 2 * W * gs;
  double* sI = sR + (size_t)W * gs;
  seg_prep<W>(a, a.u_in, (size_t)a.g.n_r * a.g.pitch, h, j0, lane, sR, sI);
  __syncwarp();
  const int j = j0 + lane;
  if (j < a.g.n_th) half_point<W>(a, h, j, sR + lane, sI + lane, gs);
}

template <int W, int V = 0>
__global__ void __launch_bounds__(128, 2 * (V + 1)) full_seg_kernel(StepArgs a, int nseg) {
  step_dependency();
  extern __shared__ double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int unit = blockIdx.x * (blockDim.x >> 5) + warp;
  const int i = 1 + unit / nseg, j0 = (unit % nseg) * 32;
  if (i >= a.g.n_r - 1) return;
  const int gs = 32 + 2 * a.radius;
  double* sR = sm + (size_t)warp * 2 * W * gs;
  double* sI = sR + (size_t)W * gs;
  seg_prep<W>(a, a.uh, (size_t)(a.g.n_r - 1) * a.g.pitch, i - 1, j0, lane, sR, sI);
  __syncwarp();
  const int j = j0 + lane;
  long long slot = -1;
  if (a.record) slot = a.ring_slot >= 0 ? a.ring_slot : (*a.ring_counter) % a.ring_cap;
  const bool bad = j < a.g.n_th && full_point<W>(a, i, j, sR + lane, sI + lane, gs, slot);
  if (bad) atomicOr(a.status, 1u);
}

// ---- single-problem kernels: blockDim.y rows per block, blockDim.x threads along theta ------
// V selects the register budget: V = 0, 1: at least V + 1 blocks of up to 256 threads per SM
// (<= 255, 128 registers); V = 2: at least 5 blocks of up to 128 threads (<= 102 registers,
// 20 warps per SM). The autotuner picks the fastest variant per problem.
template <int V> struct RowBounds { static constexpr int threads = 256, blocks = V + 1; };
template <> struct RowBounds<2> { static constexpr int threads = 128, blocks = 5; };
template <int W, int V = 0>
__global__ void __launch_bounds__(RowBounds<V>::threads, RowBounds<V>::blocks) half_kernel(StepArgs a) {
  step_dependency();
  extern __shared__ double sm[];
  const int gstride = a.g.n_th + 2 * a.radius;
  const int h = blockIdx.x * blockDim.y + threadIdx.y;
  const bool ok = h < a.g.n_r - 1;
  double* sR = sm + (size_t)threadIdx.y * 2 * W * gstride;
  double* sI = sR + (size_t)W * gstride;
  if (ok) half_row_prep<W>(a, h, threadIdx.x, blockDim.x, sR, sI);
  __syncthreads();
  if (ok) half_row_out<W>(a, h, threadIdx.x, blockDim.x, sR, sI);
}

template <int W, int V = 0>
__global__ void __launch_bounds__(RowBounds<V>::threads, RowBounds<V>::blocks) full_kernel(StepArgs a) {
  step_dependency();
  extern __shared__ double sm[];
  const int gstride = a.g.n_th + 2 * a.radius;
  const int i = 1 + blockIdx.x * blockDim.y + threadIdx.y;
  const bool ok = i < a.g.n_r - 1;
  double* sR = sm + (size_t)threadIdx.y * 2 * W * gstride;
  double* sI = sR + (size_t)W * gstride;
  if (ok) full_row_prep<W>(a, i, threadIdx.x, blockDim.x, sR, sI);
  __syncthreads();
  if (!ok) return;
  long long slot = -1;
  if (a.record) slot = a.ring_slot >= 0 ? a.ring_slot : (*a.ring_counter) % a.ring_cap;
  if (full_row_out<W>(a, i, threadIdx.x, blockDim.x, sR, sI, slot)) atomicOr(a.status, 1u);
}

// ---- fused iteration for small problems: one launch per Lax-Wendroff iteration -------------
// Block b produces the full-step rows i0 .. i1 (i0 = 1 + b R, R = blockDim.y - 1) into u_out,
// which must be another buffer than u_in: the blocks next to it read the rows beside its own
// from u_in. It first forms the R + 1 half rows i0 - 1 .. i1 that these rows need (the first
// one is also formed by the block below; both get the same bits) in its own shared memory,
// then the full-step rows, with the row bodies of the two-kernel form: the results are the
// same bits as theirs. One launch per iteration halves the launches of small grids, whose
// iterations are shorter than the launch cost.
template <int W>
__global__ void __launch_bounds__(256, 1) fused_kernel(StepArgs a) {
  step_dependency();
  extern __shared__ double sm[];
  const int R = blockDim.y - 1, n_r = a.g.n_r, pitch = a.g.pitch;
  const int gstride = a.g.n_th + 2 * a.radius;
  const int i0 = 1 + blockIdx.x * R;
  const int i1 = min(i0 + R - 1, n_r - 2);
  StepArgs b = a;
  b.uh = sm;  // [4][W][R + 1][pitch]
  b.uh_ws = (size_t)(R + 1) * pitch;
  b.uh_row0 = i0 - 1;
  const int y = threadIdx.y;
  double* sR = sm + (size_t)4 * W * (R + 1) * pitch + (size_t)y * 2 * W * gstride;
  double* sI = sR + (size_t)W * gstride;
  const int h = i0 - 1 + y;
  const bool hok = h <= i1;
  if (hok) half_row_prep<W>(b, h, threadIdx.x, blockDim.x, sR, sI);
  __syncthreads();
  if (hok) half_row_out<W>(b, h, threadIdx.x, blockDim.x, sR, sI);
  __syncthreads();
  const int i = i0 + y;
  const bool fok = y < R && i <= i1;
  if (fok) full_row_prep<W>(b, i, threadIdx.x, blockDim.x, sR, sI);
  __syncthreads();
  if (!fok) return;
  long long slot = -1;
  if (a.record) slot = a.ring_slot >= 0 ? a.ring_slot : (*a.ring_counter) % a.ring_cap;
  if (full_row_out<W>(b, i, threadIdx.x, blockDim.x, sR, sI, slot)) atomicOr(a.status, 1u);
}

// ---- balanced kernels: the same number of points for every block ----------------------------
// The launch has exactly as many blocks as fit on the GPU at once (blockDim.x threads along
// theta, one ghosted row of shared memory each). Block b takes the points
// [b P / G, (b + 1) P / G) of the row-major (row, theta) range of P points, so every SM gets the
// same share of the FP64 work whatever the row count, without a partly filled last wave of
// blocks. A block walks the rows its range touches: all its threads build the whole ghosted
// row in shared memory, then take the range's columns of that row.
template <int W, int V = 0>
__global__ void __launch_bounds__(RowBounds<V>::threads, RowBounds<V>::blocks) half_bal_kernel(StepArgs a) {
  step_dependency();
  extern __shared__ double sm[];
  const int n_th = a.g.n_th, gstride = n_th + 2 * a.radius;
  const long long total = (long long)(a.g.n_r - 1) * n_th;
  const long long p0 = total * blockIdx.x / gridDim.x, p1 = total * (blockIdx.x + 1) / gridDim.x;
  double* sR = sm;
  double* sI = sm + (size_t)W * gstride;
  for (long long p = p0; p < p1;) {
    const int h = (int)(p / n_th), c0 = (int)(p % n_th);
    const int c1 = (int)(p1 - p < (long long)(n_th - c0) ? c0 + (p1 - p) : n_th);
    half_row_prep<W>(a, h, threadIdx.x, blockDim.x, sR, sI);
    __syncthreads();
    half_row_out<W>(a, h, threadIdx.x, blockDim.x, sR, sI, c0, c1);
    __syncthreads();
    p += c1 - c0;
  }
}

template <int W, int V = 0>
__global__ void __launch_bounds__(RowBounds<V>::threads, RowBounds<V>::blocks) full_bal_kernel(StepArgs a) {
  step_dependency();
  extern __shared__ double sm[];
  const int n_th = a.g.n_th, gstride = n_th + 2 * a.radius;
  const long long total = (long long)(a.g.n_r - 2) * n_th;
  const long long p0 = total * blockIdx.x / gridDim.x, p1 = total * (blockIdx.x + 1) / gridDim.x;
  double* sR = sm;
  double* sI = sm + (size_t)W * gstride;
  long long slot = -1;
  if (a.record) slot = a.ring_slot >= 0 ? a.ring_slot : (*a.ring_counter) % a.ring_cap;
  bool bad = false;
  for (long long p = p0; p < p1;) {
    const int i = 1 + (int)(p / n_th), c0 = (int)(p % n_th);
    const int c1 = (int)(p1 - p < (long long)(n_th - c0) ? c0 + (p1 - p) : n_th);
    full_row_prep<W>(a, i, threadIdx.x, blockDim.x, sR, sI);
    __syncthreads();
    bad |= full_row_out<W>(a, i, threadIdx.x, blockDim.x, sR, sI, slot, c0, c1);
    __syncthreads();
    p += c1 - c0;
  }
  if (bad) atomicOr(a.status, 1u);
}

// ---- persistent kernel for small problems: many iterations in one launch ---------------------
// A small grid cannot keep the GPU busy between launches: the launches of one iteration cost
// more than its arithmetic. Here one cooperative launch runs n_outer outer steps of k
// iterations. Block b owns the half rows and nodes [b R, (b + 1) R) (R = blockDim.y rows, one
// thread row each). Only neighbouring blocks depend on each other:
//   half step n of block b reads state row (b + 1) R, written by block b + 1's full step n - 1;
//   full step n of block b reads half row b R - 1, written by block b - 1's half step n, and
//   overwrites state row b R, which that half step reads.
// So each block publishes two counters, half_done[b] and full_done[b] (iterations finished in
// this launch), and before each phase waits for the neighbour's counter: thread 0 polls with
// an acquire load (a bounded number of times), the block's barrier passes the ordering on to
// its other threads; after each phase thread 0 publishes with a fence and a release store.
// A wait that reaches its limit sets status bit 2 and the abort word, on which every other
// wait gives up too, so the launch always ends. Arithmetic: the row kernels' point functions,
// so the results are bit-identical to the one-launch-per-phase kernels.
struct PersistArgs {
  StepArgs a;             // state updated in place (u_in == u_out), half rows, tables, ring
  int k;                  // iterations per outer step
  int n_outer;            // outer steps in this launch
  long long ring_base;    // samples recorded before this launch
  int* flags;             // [2 * gridDim.x + 1]: half_done, full_done, abort (zeroed before the launch)
  int spin_log2;          // a wait gives up after 2^spin_log2 polls
  int stall_block;        // test hook: this block never publishes its counters (-1: none)
};

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0 waits until *f >= target (or gives up); the result reaches the whole block. (Polling
// with relaxed loads and one acquire fence at the end measured slower than acquire loads.)
__device__ __forceinline__ bool persist_wait(const PersistArgs& p, const int* f, int target, int* ok_sm) {
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    int ok = 1;
    if (f) {
      const long long limit = 1ll << p.spin_log2;
      const int* abortw = p.flags + 2 * gridDim.x;
      ok = 0;
      for (long long it = 0; it < limit; ++it) {
        if (ld_acquire_gpu(f) >= target) { ok = 1; break; }
        if (ld_acquire_gpu(abortw)) break;
      }
      if (!ok) {
        atomicOr(p.a.status, 2u);
        atomicExch(p.flags + 2 * gridDim.x, 1);
      }
    }
    *ok_sm = ok;
  }
  __syncthreads();
  return *ok_sm != 0;
}

// After the block barrier, thread 0 fences the block's writes and publishes with a release store.
__device__ __forceinline__ void persist_publish(const PersistArgs& p, int* f, int value) {
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0 && (int)blockIdx.x != p.stall_block) {
    __threadfence();
    st_release_gpu(f, value);
  }
}

// blockDim = (threads along theta, R rows); grid = ceil((n_r - 1) / R) co-resident blocks.
// (Doing a block's rows that need nothing from a neighbour before the wait, and only the
// neighbour-dependent row after it, measured slower on the 256 x 64 FP64 grid: each stage
// leaves part of the block idle.)
template <int W>
__global__ void __launch_bounds__(256, 1) persist_kernel(PersistArgs p) {
  extern __shared__ double sm[];
  __shared__ int s_ok;
  const StepArgs& a = p.a;
  const int G = gridDim.x, b = blockIdx.x, ty = threadIdx.y, tx = threadIdx.x, TX = blockDim.x;
  const int gstride = a.g.n_th + 2 * a.radius;
  double* sR = sm + (size_t)ty * 2 * W * gstride;
  double* sI = sR + (size_t)W * gstride;
  const int h = b * (int)blockDim.y + ty;  // this thread row's half row and node
  const bool h_ok = h < a.g.n_r - 1;
  const bool i_ok = h >= 1 && h < a.g.n_r - 1;
  int* half_done = p.flags;
  int* full_done = p.flags + G;
  const int* next_full = b + 1 < G ? full_done + b + 1 : nullptr;
  const int* prev_half = b > 0 ? half_done + b - 1 : nullptr;
  bool bad = false;
  int n = 0;
  for (int s = 0; s < p.n_outer; ++s) {
    for (int q = 0; q < p.k; ++q) {
      ++n;
      // Eq. lw1: state row (b + 1) R must hold iteration n - 1
      if (!persist_wait(p, n > 1 ? next_full : nullptr, n - 1, &s_ok)) goto done;
      if (h_ok) half_row_prep<W>(a, h, tx, TX, sR, sI);
      __syncthreads();
      if (h_ok) half_row_out<W>(a, h, tx, TX, sR, sI);
      persist_publish(p, half_done + b, n);
      // Eq. lw2: half row b R - 1 must hold iteration n (and be read before row b R changes)
      if (!persist_wait(p, prev_half, n, &s_ok)) goto done;
      if (i_ok) full_row_prep<W>(a, h, tx, TX, sR, sI);
      __syncthreads();
      if (i_ok) {
        const long long slot = (q == p.k - 1 && a.ring_cap > 0) ? (p.ring_base + s) % a.ring_cap : -1;
        bad |= full_row_out<W>(a, h, tx, TX, sR, sI, slot);
      }
      persist_publish(p, full_done + b, n);
    }
  }
done:
  if (bad) atomicOr(a.status, 1u);
}

// Arguments of the integer-engine step kernels (teuk_ix.cuh). Planes of the engine's
// coefficient tables: the eight folded coefficients of the step, with plane 5 (H5 / N5, the
// factor of the theta operator) replaced by H5 A2 and plane 8 holding H5 A1 cot theta_j.
constexpr int kIxPlanes = 9;

struct IxArgs {
  StepArgs a;           // geometry, state, half-step rows, ring, status
  const uint4* cnm;     // node coefficients [kIxPlanes][kU4][n_r][pitch]: mantissas
  const int* cne;       //   exponent-sign words [kIxPlanes][n_r][pitch]
  const uint4* chm;     // half-node coefficients [kIxPlanes][kU4][n_r - 1][pitch]
  const int* che;
  int stage;            // 1: each block copies its rows of the tables into shared memory first
  int wait_log2;        // the wait for those copies gives up after 2^wait_log2 tries
  int stall_block;      // test hook: this block arms its copy barrier but issues no copy (-1: none)
};

// ---- batched execution: many problems of uneven size in one cooperative launch ------------
struct BatchMember {
  StepArgs a;            // the member's buffers (state updated in place, scratch, tables)
  int k;                 // Lax-Wendroff iterations per outer step
  int tx;                // threads along theta per row
  int rows;              // rows per work item (tx * rows <= blockDim.x)
  int item_begin;        // first work item of this member
  long long ring_base;   // samples already in the member's observer ring
  long long ring_cap;    // ring capacity, 0 = no observer
};

struct BatchArgs {
  const BatchMember* m;     // sorted by k, descending
  const int* item_member;   // member of each work item
  const int* active_items;  // [k_max]: number of items whose member has k > q (a prefix)
  int k_max;
  int n_outer;
};

// Outer steps of all members: in round q = 0 .. k_max-1 every member with k > q performs one
// Lax-Wendroff iteration, as a half-step phase over all their work items, a grid-wide
// barrier, a full-step phase, another barrier. Work items hold the same number of grid points
// (rows x theta = blockDim.x), so the grid-stride loops stay balanced across uneven members.
template <int W>
__global__ void __launch_bounds__(256, 2) batch_kernel(BatchArgs b) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  extern __shared__ double sm[];
  for (int s = 0; s < b.n_outer; ++s) {
    for (int q = 0; q < b.k_max; ++q) {
      const int n_act = b.active_items[q];
      for (int it = blockIdx.x; it < n_act; it += gridDim.x) {
        const BatchMember& M = b.m[b.item_member[it]];
        const int tx = threadIdx.x % M.tx, ty = threadIdx.x / M.tx;
        const int h = (it - M.item_begin) * M.rows + ty;
        const bool ok = ty < M.rows && h < M.a.g.n_r - 1;
        const int gstride = M.a.g.n_th + 2 * M.a.radius;
        double* sR = sm + (size_t)(ty < M.rows ? ty : 0) * 2 * W * gstride;
        double* sI = sR + (size_t)W * gstride;
        if (ok) half_row_prep<W>(M.a, h, tx, M.tx, sR, sI);
        __syncthreads();
        if (ok) half_row_out<W>(M.a, h, tx, M.tx, sR, sI);
        __syncthreads();
      }
      grid.sync();
      for (int it = blockIdx.x; it < n_act; it += gridDim.x) {
        const BatchMember& M = b.m[b.item_member[it]];
        const int tx = threadIdx.x % M.tx, ty = threadIdx.x / M.tx;
        const int i = 1 + (it - M.item_begin) * M.rows + ty;
        const bool ok = ty < M.rows && i < M.a.g.n_r - 1;
        const int gstride = M.a.g.n_th + 2 * M.a.radius;
        double* sR = sm + (size_t)(ty < M.rows ? ty : 0) * 2 * W * gstride;
        double* sI = sR + (size_t)W * gstride;
        if (ok) full_row_prep<W>(M.a, i, tx, M.tx, sR, sI);
        __syncthreads();
        if (ok) {
          const long long slot = (q == M.k - 1 && M.ring_cap > 0) ? (M.ring_base + s) % M.ring_cap : -1;
          if (full_row_out<W>(M.a, i, tx, M.tx, sR, sI, slot)) atomicOr(M.a.status, 1u);
        }
        __syncthreads();
      }
      grid.sync();
    }
  }
}

}  // namespace teuk
