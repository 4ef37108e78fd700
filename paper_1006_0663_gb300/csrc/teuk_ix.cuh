// Double-double and quad-double step kernels on the integer engine (ix.cuh, ixq.cuh): the
// same two kernels per Lax-Wendroff iteration as teuk_kernels.cuh (Eqs. lw1, lw2 with the
// folded coefficient tables and the 10th/2nd-order theta stencil, Sec. 3.B-3.D), with every
// dot product formed exactly on the integer pipe and rounded once to the handle's precision.
// The state and the half-step rows stay multi-word doubles in HBM; the coefficient tables and
// stencil weights are kept in the engine's format: the mantissa as 1 (dd) or 2 (qd) uint4 per
// value in planes of their own, the exponent and sign as one int (e * 2 + neg).
#pragma once

#include "ix.cuh"
#include "ixq.cuh"
#include "teuk_kernels.cuh"

namespace teuk {

#define IXD __device__ __forceinline__
#define IXHD __host__ __device__ __forceinline__

// Engine types and operations per arithmetic (W = words per real).
template <int W> struct IxT;
template <> struct IxT<2> {
  using Num = ix::Num;
  using Acc = ix::Acc;
  static constexpr int kLimbs = 4, kU4 = 1, kTop = 126;  // leading bit of a converted value
  static IXHD Num load(const double* p, size_t ws, uint32_t& bad) { return ix::from_dd(p[0], p[ws], bad); }
  static IXHD Num add(const Num& a, const Num& b, uint32_t nb) { return ix::add(a, b, nb); }
  static IXHD int pexp(int ec, int ev) { return ix::prod_exp(ec, ev); }
  static IXHD void zero(Acc& acc) { ix::acc_zero(acc); }
  static IXHD void prod(Acc& acc, const uint32_t* cm, const uint32_t* vm, uint32_t neg, int ep, int mx) {
    ix::acc_prod(acc, cm, vm, neg, ep, mx);
  }
  static IXHD int base(int mx) { return ix::acc_base(mx); }
  static IXHD Num to_num(const Acc& acc, int B) { return ix::to_num(acc, B); }
  static IXHD void to_words(const Acc& acc, int B, double* w) {
    const mw::dd r = ix::to_dd(acc, B);
    w[0] = r.h;
    w[1] = r.l;
  }
  static IXHD Num zero_num() { return ix::zero(); }
};
template <> struct IxT<4> {
  using Num = ix::Num8;
  using Acc = ix::Acc10;
  static constexpr int kLimbs = 8, kU4 = 2, kTop = 254;
  static IXHD Num load(const double* p, size_t ws, uint32_t& bad) {
    return ix::from_qd(p[0], p[ws], p[2 * ws], p[3 * ws], bad);
  }
  static IXHD Num add(const Num& a, const Num& b, uint32_t nb) { return ix::add8(a, b, nb); }
  static IXHD int pexp(int ec, int ev) { return ix::prod_exp8(ec, ev); }
  static IXHD void zero(Acc& acc) { ix::acc_zero10(acc); }
  static IXHD void prod(Acc& acc, const uint32_t* cm, const uint32_t* vm, uint32_t neg, int ep, int mx) {
    ix::acc_prod10(acc, cm, vm, neg, ep, mx);
  }
  static IXHD int base(int mx) { return ix::acc_base10(mx); }
  static IXHD Num to_num(const Acc& acc, int B) { return ix::to_num8(acc, B); }
  static IXHD void to_words(const Acc& acc, int B, double* w) {
    const mw::qd r = ix::to_qd(acc, B);
    w[0] = r.x0; w[1] = r.x1; w[2] = r.x2; w[3] = r.x3;
  }
  static IXHD Num zero_num() { return ix::zero8(); }
};

// The constant 2^k (k = 0: one, k = -1: one half) in engine format.
template <int W>
IXHD typename IxT<W>::Num ix_pow2(int k) {
  typename IxT<W>::Num r = IxT<W>::zero_num();
  r.m[IxT<W>::kLimbs - 1] = 0x40000000u;  // bit 32 L - 2
  r.e = k - IxT<W>::kTop;
  r.neg = 0;
  return r;
}

struct IxArgs {
  StepArgs a;           // geometry, state, half-step rows, ring, status
  const uint4* cnm;     // folded node coefficients [8][kU4][n_r][pitch]: mantissas
  const int* cne;       //   exponent-sign words [8][n_r][pitch]
  const uint4* chm;     // folded half-node coefficients [8][kU4][n_r - 1][pitch]
  const int* che;
  const uint4* wm;      // theta weights [2 radius + 1][kU4][n_th]
  const int* we;
};

template <class N>
__host__ __device__ __forceinline__ int ix_en(const N& x) { return x.e * 2 + (int)x.neg; }

// Mantissa of value r of plane c in a [C][kU4][per_plane] uint4 array.
template <int W>
IXD void ix_ldm(const uint4* base, size_t per_plane, size_t c, size_t r, uint32_t* m) {
#pragma unroll
  for (int u = 0; u < IxT<W>::kU4; ++u) {
    const uint4 v = __ldg(base + (c * IxT<W>::kU4 + u) * per_plane + r);
    m[4 * u] = v.x; m[4 * u + 1] = v.y; m[4 * u + 2] = v.z; m[4 * u + 3] = v.w;
  }
}

// Table conversion (set-up): count values of planes [C][W][rows][pitch] (word stride ws)
// into mantissa planes [C][kU4][per_plane] and exponent-sign words [C][per_plane].
template <int W>
__global__ void ix_table_kernel(const double* src, size_t ws, size_t per_plane, size_t count, uint4* dm, int* de) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const size_t c = k / per_plane, r = k % per_plane;
  uint32_t bad = 0;
  const typename IxT<W>::Num x = IxT<W>::load(src + (W * c) * ws + r, ws, bad);
#pragma unroll
  for (int u = 0; u < IxT<W>::kU4; ++u)
    dm[(c * IxT<W>::kU4 + u) * per_plane + r] = make_uint4(x.m[4 * u], x.m[4 * u + 1], x.m[4 * u + 2], x.m[4 * u + 3]);
  de[k] = ix_en(x);
}

// Ghosted shared row of one component: mantissas [kU4][gstride] (uint4), exponent-sign
// words [gstride] (int).
struct IxRow {
  uint4* m;
  int* e;
};
template <int W>
IXD typename IxT<W>::Num ix_row_get(const IxRow& row, int gstride, int idx) {
  typename IxT<W>::Num r;
#pragma unroll
  for (int u = 0; u < IxT<W>::kU4; ++u) {
    const uint4 v = row.m[u * gstride + idx];
    r.m[4 * u] = v.x; r.m[4 * u + 1] = v.y; r.m[4 * u + 2] = v.z; r.m[4 * u + 3] = v.w;
  }
  const int en = row.e[idx];
  r.e = en >> 1;  // arithmetic shift: floor(en / 2)
  r.neg = (uint32_t)en & 1u;
  return r;
}
template <int W>
IXD void ix_row_put(const IxRow& row, int gstride, int idx, const typename IxT<W>::Num& v, int en) {
#pragma unroll
  for (int u = 0; u < IxT<W>::kU4; ++u)
    row.m[u * gstride + idx] = make_uint4(v.m[4 * u], v.m[4 * u + 1], v.m[4 * u + 2], v.m[4 * u + 3]);
  row.e[idx] = en;
}
// Writes v as column j of a ghosted row (and its parity images across the poles).
template <int W>
IXD void ix_put_ghosted(const IxRow& row, int gstride, int n_th, int radius, int parity, int j,
                        const typename IxT<W>::Num& v) {
  const int en = ix_en(v), pen = parity > 0 ? en : (en ^ 1);
  ix_row_put<W>(row, gstride, j + radius, v, en);
  if (j < radius) ix_row_put<W>(row, gstride, radius - 1 - j, v, pen);
  if (j >= n_th - radius) ix_row_put<W>(row, gstride, 2 * n_th - 1 - j + radius, v, pen);
}

IXHD int imax(int a, int b) { return a > b ? a : b; }

// One term c * v with c from a coefficient table (plane q, index ci), sign flipped if flip.
template <int W>
IXD void ix_tterm(typename IxT<W>::Acc& acc, const uint4* tm, size_t per_plane, int q, size_t ci, int ce,
                  const typename IxT<W>::Num& v, uint32_t flip, int mx) {
  uint32_t c[IxT<W>::kLimbs];
  ix_ldm<W>(tm, per_plane, q, ci, c);
  IxT<W>::prod(acc, c, v.m, ((uint32_t)ce & 1u) ^ v.neg ^ flip, IxT<W>::pexp(ce >> 1, v.e), mx);
}
template <int W>
IXD void ix_nterm(typename IxT<W>::Acc& acc, const typename IxT<W>::Num& c, const typename IxT<W>::Num& v,
                  uint32_t flip, int mx) {
  IxT<W>::prod(acc, c.m, v.m, c.neg ^ v.neg ^ flip, IxT<W>::pexp(c.e, v.e), mx);
}
template <int W>
IXD int ix_texp(int ce, const typename IxT<W>::Num& v) { return IxT<W>::pexp(ce >> 1, v.e); }

template <int W>
IXD void ix_store(double* p, size_t ws, const typename IxT<W>::Acc& acc, int B, uint32_t bad, double* w) {
  IxT<W>::to_words(acc, B, w);
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
  for (int k = 0; k < W; ++k) p[k * ws] = bad ? nan : w[k];
}

// Theta operator at column j of a ghosted engine-format row.
template <int W, int RAD>
IXD typename IxT<W>::Num ix_theta(const IxArgs& x, const IxRow& row, int gstride, int j) {
  const size_t n_th = (size_t)x.a.g.n_th;
  int mx = 2 * ix::kZeroE;
#pragma unroll
  for (int q = 0; q < 2 * RAD + 1; ++q) mx = imax(mx, IxT<W>::pexp(__ldg(x.we + q * n_th + j) >> 1, row.e[j + q] >> 1));
  typename IxT<W>::Acc acc;
  IxT<W>::zero(acc);
#pragma unroll
  for (int q = 0; q < 2 * RAD + 1; ++q)
    ix_tterm<W>(acc, x.wm, n_th, q, j, __ldg(x.we + q * n_th + j), ix_row_get<W>(row, gstride, j + q), 0u, mx);
  return IxT<W>::to_num(acc, IxT<W>::base(mx));
}
template <int W>
IXD typename IxT<W>::Num ix_theta(const IxArgs& x, const IxRow& row, int gstride, int j) {
  return x.a.radius == 5 ? ix_theta<W, 5>(x, row, gstride, j) : ix_theta<W, 1>(x, row, gstride, j);
}

// Eq. lw1, first phase: s_Phi = Phi_{h+1} + Phi_h of row h into the ghosted rows.
template <int W>
IXD void ix_half_prep(const IxArgs& x, int h, int tx, int TX, const IxRow& sR, const IxRow& sI, int gstride) {
  const StepArgs& a = x.a;
  const size_t ws = (size_t)a.g.n_r * a.g.pitch;
  for (int j = tx; j < a.g.n_th; j += TX) {
    const size_t i0 = (size_t)h * a.g.pitch + j, i1 = i0 + a.g.pitch;
    uint32_t bad = 0;
    const auto vR = IxT<W>::add(IxT<W>::load(a.u_in + i1, ws, bad), IxT<W>::load(a.u_in + i0, ws, bad), 0u);
    const auto vI = IxT<W>::add(IxT<W>::load(a.u_in + W * ws + i1, ws, bad),
                                IxT<W>::load(a.u_in + W * ws + i0, ws, bad), 0u);
    ix_put_ghosted<W>(sR, gstride, a.g.n_th, a.radius, a.g.parity, j, vR);
    ix_put_ghosted<W>(sI, gstride, a.g.n_th, a.radius, a.g.parity, j, vI);
  }
}

// Eq. lw1 at half node h, column j (same terms as half_point in teuk_kernels.cuh).
template <int W>
IXD void ix_half_point(const IxArgs& x, int h, int j, const IxRow& sR, const IxRow& sI, int gstride,
                       const typename IxT<W>::Num& half, const typename IxT<W>::Num& h4) {
  using T = IxT<W>;
  using Num = typename T::Num;
  const StepArgs& a = x.a;
  const int pitch = a.g.pitch, rad = a.radius;
  const size_t ws = (size_t)a.g.n_r * pitch, hs = (size_t)(a.g.n_r - 1) * pitch;
  const size_t i0 = (size_t)h * pitch + j, i1 = i0 + pitch;
  uint32_t bad = 0;
  const double* u = a.u_in;
  const Num uPR0 = T::load(u + 0 * W * ws + i0, ws, bad), uPR1 = T::load(u + 0 * W * ws + i1, ws, bad);
  const Num uPI0 = T::load(u + 1 * W * ws + i0, ws, bad), uPI1 = T::load(u + 1 * W * ws + i1, ws, bad);
  const Num uQR0 = T::load(u + 2 * W * ws + i0, ws, bad), uQR1 = T::load(u + 2 * W * ws + i1, ws, bad);
  const Num uQI0 = T::load(u + 3 * W * ws + i0, ws, bad), uQI1 = T::load(u + 3 * W * ws + i1, ws, bad);
  const Num dPR = T::add(uPR1, uPR0, 1u), dPI = T::add(uPI1, uPI0, 1u);
  const Num sQR = T::add(uQR1, uQR0, 0u), sQI = T::add(uQI1, uQI0, 0u);
  // one exact difference and one product are cheaper here than two products, and free the
  // four Pi values early
  const Num dQR = T::add(uQR1, uQR0, 1u), dQI = T::add(uQI1, uQI0, 1u);
  const Num sPR = ix_row_get<W>(sR, gstride, j + rad), sPI = ix_row_get<W>(sI, gstride, j + rad);
  const Num LR = ix_theta<W>(x, sR, gstride, j), LI = ix_theta<W>(x, sI, gstride, j);
  const size_t ci = (size_t)h * pitch + j;
  int ce[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) ce[q] = __ldg(x.che + q * hs + ci);
#define TT(q, v, f) ix_tterm<W>(acc, x.chm, hs, q, ci, ce[q], v, f, mx)
#define TE(q, v) ix_texp<W>(ce[q], v)
  typename T::Acc acc;
  int mx;
  double w[4];
  // Phi_R = s_PhiR/2 - H0 d_PhiR + (h/4) s_PiR
  mx = imax(imax(T::pexp(half.e, sPR.e), TE(0, dPR)), T::pexp(h4.e, sQR.e));
  T::zero(acc);
  ix_nterm<W>(acc, half, sPR, 0u, mx);
  TT(0, dPR, 1u);
  ix_nterm<W>(acc, h4, sQR, 0u, mx);
  ix_store<W>(a.uh + 0 * W * hs + ci, hs, acc, T::base(mx), bad, w);
  // Phi_I
  mx = imax(imax(T::pexp(half.e, sPI.e), TE(0, dPI)), T::pexp(h4.e, sQI.e));
  T::zero(acc);
  ix_nterm<W>(acc, half, sPI, 0u, mx);
  TT(0, dPI, 1u);
  ix_nterm<W>(acc, h4, sQI, 0u, mx);
  ix_store<W>(a.uh + 1 * W * hs + ci, hs, acc, T::base(mx), bad, w);
  // Pi_R = H3 s_PiR + H4 s_PiI + H0 (Pi_R,h+1 - Pi_R,h) + H1 d_PhiR + H2 d_PhiI + H5 L_R + H6 s_PhiR - H7 s_PhiI
  mx = imax(imax(imax(TE(3, sQR), TE(4, sQI)), TE(0, dQR)),
            imax(imax(TE(1, dPR), TE(2, dPI)), imax(TE(5, LR), imax(TE(6, sPR), TE(7, sPI)))));
  T::zero(acc);
  TT(3, sQR, 0u); TT(4, sQI, 0u); TT(0, dQR, 0u); TT(1, dPR, 0u);
  TT(2, dPI, 0u); TT(5, LR, 0u); TT(6, sPR, 0u); TT(7, sPI, 1u);
  ix_store<W>(a.uh + 2 * W * hs + ci, hs, acc, T::base(mx), bad, w);
  // Pi_I = H3 s_PiI - H4 s_PiR + H0 (Pi_I,h+1 - Pi_I,h) + H1 d_PhiI - H2 d_PhiR + H5 L_I + H6 s_PhiI + H7 s_PhiR
  mx = imax(imax(imax(TE(3, sQI), TE(4, sQR)), TE(0, dQI)),
            imax(imax(TE(1, dPI), TE(2, dPR)), imax(TE(5, LI), imax(TE(6, sPI), TE(7, sPR)))));
  T::zero(acc);
  TT(3, sQI, 0u); TT(4, sQR, 1u); TT(0, dQI, 0u); TT(1, dPI, 0u);
  TT(2, dPR, 1u); TT(5, LI, 0u); TT(6, sPI, 0u); TT(7, sPR, 0u);
  ix_store<W>(a.uh + 3 * W * hs + ci, hs, acc, T::base(mx), bad, w);
#undef TT
#undef TE
}

// Eq. lw2, first phase: s_Phi = Phi_{i+1/2} + Phi_{i-1/2} into the ghosted rows.
template <int W>
IXD void ix_full_prep(const IxArgs& x, int i, int tx, int TX, const IxRow& sR, const IxRow& sI, int gstride) {
  const StepArgs& a = x.a;
  const size_t hs = (size_t)(a.g.n_r - 1) * a.g.pitch;
  for (int j = tx; j < a.g.n_th; j += TX) {
    const size_t p = (size_t)i * a.g.pitch + j, m = p - a.g.pitch;
    uint32_t bad = 0;
    const auto vR = IxT<W>::add(IxT<W>::load(a.uh + p, hs, bad), IxT<W>::load(a.uh + m, hs, bad), 0u);
    const auto vI = IxT<W>::add(IxT<W>::load(a.uh + W * hs + p, hs, bad), IxT<W>::load(a.uh + W * hs + m, hs, bad), 0u);
    ix_put_ghosted<W>(sR, gstride, a.g.n_th, a.radius, a.g.parity, j, vR);
    ix_put_ghosted<W>(sI, gstride, a.g.n_th, a.radius, a.g.parity, j, vI);
  }
}

// Eq. lw2 at node i, column j (same terms as full_point); returns true for a non-finite value.
template <int W>
IXD bool ix_full_point(const IxArgs& x, int i, int j, const IxRow& sR, const IxRow& sI, int gstride,
                       const typename IxT<W>::Num& one, const typename IxT<W>::Num& h2, long long slot) {
  using T = IxT<W>;
  using Num = typename T::Num;
  const StepArgs& a = x.a;
  const int pitch = a.g.pitch, rad = a.radius, n_th = a.g.n_th;
  const size_t ws = (size_t)a.g.n_r * pitch, hs = (size_t)(a.g.n_r - 1) * pitch;
  const size_t p = (size_t)i * pitch + j, m = p - pitch;
  uint32_t bad = 0;
  const double* uh = a.uh;
  const Num hPR1 = T::load(uh + 0 * W * hs + p, hs, bad), hPR0 = T::load(uh + 0 * W * hs + m, hs, bad);
  const Num hPI1 = T::load(uh + 1 * W * hs + p, hs, bad), hPI0 = T::load(uh + 1 * W * hs + m, hs, bad);
  const Num hQR1 = T::load(uh + 2 * W * hs + p, hs, bad), hQR0 = T::load(uh + 2 * W * hs + m, hs, bad);
  const Num hQI1 = T::load(uh + 3 * W * hs + p, hs, bad), hQI0 = T::load(uh + 3 * W * hs + m, hs, bad);
  const Num dPR = T::add(hPR1, hPR0, 1u), dPI = T::add(hPI1, hPI0, 1u);
  const Num sQR = T::add(hQR1, hQR0, 0u), sQI = T::add(hQI1, hQI0, 0u);
  const Num dQR = T::add(hQR1, hQR0, 1u), dQI = T::add(hQI1, hQI0, 1u);
  const Num sPR = ix_row_get<W>(sR, gstride, j + rad), sPI = ix_row_get<W>(sI, gstride, j + rad);
  const Num LR = ix_theta<W>(x, sR, gstride, j), LI = ix_theta<W>(x, sI, gstride, j);
  const size_t ci = (size_t)i * pitch + j;
  const Num PR = T::load(a.u_in + 0 * W * ws + ci, ws, bad), PI = T::load(a.u_in + 1 * W * ws + ci, ws, bad);
  const Num QR = T::load(a.u_in + 2 * W * ws + ci, ws, bad), QI = T::load(a.u_in + 3 * W * ws + ci, ws, bad);
  int ce[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) ce[q] = __ldg(x.cne + q * ws + ci);
#define TT(q, v, f) ix_tterm<W>(acc, x.cnm, ws, q, ci, ce[q], v, f, mx)
#define TE(q, v) ix_texp<W>(ce[q], v)
  typename T::Acc acc;
  int mx;
  double o0[4], o1[4], w[4];
  // Phi_R' = Phi_R - N0 d_PhiR + (h/2) s_PiR
  mx = imax(imax(T::pexp(one.e, PR.e), TE(0, dPR)), T::pexp(h2.e, sQR.e));
  T::zero(acc);
  ix_nterm<W>(acc, one, PR, 0u, mx);
  TT(0, dPR, 1u);
  ix_nterm<W>(acc, h2, sQR, 0u, mx);
  ix_store<W>(a.u_out + 0 * W * ws + ci, ws, acc, T::base(mx), bad, o0);
  // Phi_I'
  mx = imax(imax(T::pexp(one.e, PI.e), TE(0, dPI)), T::pexp(h2.e, sQI.e));
  T::zero(acc);
  ix_nterm<W>(acc, one, PI, 0u, mx);
  TT(0, dPI, 1u);
  ix_nterm<W>(acc, h2, sQI, 0u, mx);
  ix_store<W>(a.u_out + 1 * W * ws + ci, ws, acc, T::base(mx), bad, o1);
  // Pi_R' = Pi_R + N0 (h_PiR,i+1/2 - h_PiR,i-1/2) + N1 d_PhiR + N2 d_PhiI + N3 s_PiR + N4 s_PiI + N5 L_R
  //         + N6 s_PhiR - N7 s_PhiI
  mx = imax(imax(T::pexp(one.e, QR.e), imax(TE(0, dQR), TE(1, dPR))),
            imax(imax(TE(2, dPI), TE(3, sQR)), imax(imax(TE(4, sQI), TE(5, LR)), imax(TE(6, sPR), TE(7, sPI)))));
  T::zero(acc);
  ix_nterm<W>(acc, one, QR, 0u, mx);
  TT(0, dQR, 0u); TT(1, dPR, 0u); TT(2, dPI, 0u); TT(3, sQR, 0u);
  TT(4, sQI, 0u); TT(5, LR, 0u); TT(6, sPR, 0u); TT(7, sPI, 1u);
  ix_store<W>(a.u_out + 2 * W * ws + ci, ws, acc, T::base(mx), bad, w);
  const bool bad2 = nonfinite(w[0]);
  // Pi_I' = Pi_I + N0 (h_PiI,i+1/2 - h_PiI,i-1/2) + N1 d_PhiI - N2 d_PhiR + N3 s_PiI - N4 s_PiR + N5 L_I
  //         + N6 s_PhiI + N7 s_PhiR
  mx = imax(imax(T::pexp(one.e, QI.e), imax(TE(0, dQI), TE(1, dPI))),
            imax(imax(TE(2, dPR), TE(3, sQI)), imax(imax(TE(4, sQR), TE(5, LI)), imax(TE(6, sPI), TE(7, sPR)))));
  T::zero(acc);
  ix_nterm<W>(acc, one, QI, 0u, mx);
  TT(0, dQI, 0u); TT(1, dPI, 0u); TT(2, dPR, 1u); TT(3, sQI, 0u);
  TT(4, sQR, 1u); TT(5, LI, 0u); TT(6, sPI, 0u); TT(7, sPR, 0u);
  ix_store<W>(a.u_out + 3 * W * ws + ci, ws, acc, T::base(mx), bad, w);
#undef TT
#undef TE
  if (slot >= 0 && i == a.i_obs && !bad) {
    double* dst = a.ring + (size_t)slot * 2 * W * n_th;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      dst[k * n_th + j] = o0[k];
      dst[(W + k) * n_th + j] = o1[k];
    }
  }
  return bad || bad2 || nonfinite(o0[0]) || nonfinite(o1[0]) || nonfinite(w[0]);
}

// Shared memory of the engine kernels, for blockDim.y rows: mantissas [rows][2][kU4][gstride]
// (uint4) first, then the exponent-sign words [rows][2][gstride] (int).
template <int W>
IXD void ix_rows(int gstride, IxRow& sR, IxRow& sI) {
  extern __shared__ uint4 ixsm[];
  const int rows = blockDim.y, y = threadIdx.y;
  constexpr int U = IxT<W>::kU4;
  int* ebase = reinterpret_cast<int*>(ixsm + (size_t)rows * 2 * U * gstride);
  sR.m = ixsm + (size_t)y * 2 * U * gstride;
  sI.m = sR.m + (size_t)U * gstride;
  sR.e = ebase + (size_t)y * 2 * gstride;
  sI.e = sR.e + gstride;
}

template <int W, int V>
__global__ void __launch_bounds__(RowBounds<V>::threads, RowBounds<V>::blocks) half_ix_kernel(IxArgs x) {
  const int gstride = x.a.g.n_th + 2 * x.a.radius;
  IxRow sR, sI;
  ix_rows<W>(gstride, sR, sI);
  const int h = blockIdx.x * blockDim.y + threadIdx.y;
  const bool ok = h < x.a.g.n_r - 1;
  if (ok) ix_half_prep<W>(x, h, threadIdx.x, blockDim.x, sR, sI, gstride);
  __syncthreads();
  if (!ok) return;
  uint32_t bad = 0;
  const auto half = ix_pow2<W>(-1);
  const auto h4 = IxT<W>::load(x.a.h4, 1, bad);
  for (int j = threadIdx.x; j < x.a.g.n_th; j += blockDim.x) ix_half_point<W>(x, h, j, sR, sI, gstride, half, h4);
}

template <int W, int V>
__global__ void __launch_bounds__(RowBounds<V>::threads, RowBounds<V>::blocks) full_ix_kernel(IxArgs x) {
  const int gstride = x.a.g.n_th + 2 * x.a.radius;
  IxRow sR, sI;
  ix_rows<W>(gstride, sR, sI);
  const int i = 1 + blockIdx.x * blockDim.y + threadIdx.y;
  const bool ok = i < x.a.g.n_r - 1;
  if (ok) ix_full_prep<W>(x, i, threadIdx.x, blockDim.x, sR, sI, gstride);
  __syncthreads();
  if (!ok) return;
  uint32_t bad = 0;
  const auto one = ix_pow2<W>(0);
  const auto h2 = IxT<W>::load(x.a.h2, 1, bad);
  long long slot = -1;
  if (x.a.record) slot = x.a.ring_slot >= 0 ? x.a.ring_slot : (*x.a.ring_counter) % x.a.ring_cap;
  bool anybad = false;
  for (int j = threadIdx.x; j < x.a.g.n_th; j += blockDim.x)
    anybad |= ix_full_point<W>(x, i, j, sR, sI, gstride, one, h2, slot);
  if (anybad) atomicOr(x.a.status, 1u);
}

#undef IXD
#undef IXHD

}  // namespace teuk
