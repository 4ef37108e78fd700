// Double-double step kernels on the integer engine (ix.cuh): the same two kernels per
// Lax-Wendroff iteration as teuk_kernels.cuh (Eqs. lw1, lw2 with the folded coefficient
// tables and the 10th/2nd-order theta stencil, Sec. 3.B-3.D), with every dot product formed
// exactly on the integer pipe and rounded once to double-double. The state and the half-step
// rows stay double-double in HBM; the coefficient tables and stencil weights are kept in the
// engine's format (128-bit mantissa as uint4, exponent and sign as one int: e * 2 + neg).
#pragma once

#include "ix.cuh"
#include "teuk_kernels.cuh"

namespace teuk {

struct IxArgs {
  StepArgs a;           // geometry, state, half-step rows, ring, status (double-double)
  const uint4* cnm;     // folded node coefficients [8][n_r][pitch]: mantissas
  const int* cne;       //   exponent-sign words
  const uint4* chm;     // folded half-node coefficients [8][n_r - 1][pitch]
  const int* che;
  const uint4* wm;      // theta weights [2 radius + 1][n_th]
  const int* we;
};

__host__ __device__ __forceinline__ int ix_en(const ix::Num& x) { return x.e * 2 + (int)x.neg; }
__host__ __device__ __forceinline__ ix::Num ix_num(uint4 m, int en) {
  ix::Num r;
  r.m[0] = m.x; r.m[1] = m.y; r.m[2] = m.z; r.m[3] = m.w;
  r.e = en >> 1;  // arithmetic shift: floor(en / 2)
  r.neg = (uint32_t)en & 1u;
  return r;
}
__host__ __device__ __forceinline__ uint4 ix_m(const ix::Num& x) { return make_uint4(x.m[0], x.m[1], x.m[2], x.m[3]); }

// Table conversion (set-up): count double-double values of planes [C][2][rows][pitch] (word
// stride ws) into mantissa / exponent-sign arrays [C][rows][pitch].
__global__ void ix_table_kernel(const double* src, size_t ws, size_t per_plane, size_t count, uint4* dm, int* de) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const size_t c = k / per_plane, r = k % per_plane;
  uint32_t bad = 0;
  const ix::Num x = ix::from_dd(src[(2 * c) * ws + r], src[(2 * c + 1) * ws + r], bad);
  dm[k] = ix_m(x);
  de[k] = ix_en(x);
}

// One term c * v of a dot product (c from a table, v in registers), sign flipped if `flip`.
__device__ __forceinline__ int ix_texp(int ce, const ix::Num& v) { return ix::prod_exp(ce >> 1, v.e); }
__device__ __forceinline__ void ix_term(ix::Acc& acc, uint4 cm, int ce, const ix::Num& v, uint32_t flip, int maxE) {
  const uint32_t c[4] = {cm.x, cm.y, cm.z, cm.w};
  ix::acc_prod(acc, c, v.m, ((uint32_t)ce & 1u) ^ v.neg ^ flip, ix_texp(ce, v), maxE);
}
__device__ __forceinline__ void ix_term(ix::Acc& acc, const ix::Num& c, const ix::Num& v, uint32_t flip, int maxE) {
  ix::acc_prod(acc, c.m, v.m, c.neg ^ v.neg ^ flip, ix::prod_exp(c.e, v.e), maxE);
}
__device__ __forceinline__ int imax(int a, int b) { return a > b ? a : b; }

__device__ __forceinline__ ix::Num ix_load(const double* p, size_t ws, uint32_t& bad) {
  return ix::from_dd(p[0], p[ws], bad);
}
__device__ __forceinline__ void ix_store_dd(double* p, size_t ws, mw::dd v, uint32_t bad) {
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  p[0] = bad ? nan : v.h;
  p[ws] = bad ? nan : v.l;
}

// Writes v as ghosted-row entry of column j (and its parity images across the poles).
__device__ __forceinline__ void ix_put_ghosted(uint4* sm, int* se, int n_th, int radius, int parity, int j,
                                               const ix::Num& v) {
  const uint4 m = ix_m(v);
  const int en = ix_en(v), pen = parity > 0 ? en : (en ^ 1);
  sm[j + radius] = m;
  se[j + radius] = en;
  if (j < radius) { sm[radius - 1 - j] = m; se[radius - 1 - j] = pen; }
  if (j >= n_th - radius) { sm[2 * n_th - 1 - j + radius] = m; se[2 * n_th - 1 - j + radius] = pen; }
}

// Theta operator at column j on a ghosted engine-format row (srm/sre point at column j - RAD).
template <int RAD>
__device__ __forceinline__ ix::Num ix_theta(const IxArgs& x, const uint4* srm, const int* sre, int j) {
  const size_t n_th = (size_t)x.a.g.n_th;
  int maxE = 2 * ix::kZeroE;
#pragma unroll
  for (int q = 0; q < 2 * RAD + 1; ++q)
    maxE = imax(maxE, ix::prod_exp(__ldg(x.we + q * n_th + j) >> 1, sre[q] >> 1));
  ix::Acc acc;
  ix::acc_zero(acc);
#pragma unroll
  for (int q = 0; q < 2 * RAD + 1; ++q) {
    const int ce = __ldg(x.we + q * n_th + j);
    ix_term(acc, __ldg(x.wm + q * n_th + j), ce, ix_num(srm[q], sre[q]), 0u, maxE);
  }
  return ix::to_num(acc, ix::acc_base(maxE));
}
__device__ __forceinline__ ix::Num ix_theta(const IxArgs& x, const uint4* srm, const int* sre, int j) {
  return x.a.radius == 5 ? ix_theta<5>(x, srm, sre, j) : ix_theta<1>(x, srm, sre, j);
}

// Eq. lw1, first phase: s_Phi = Phi_{h+1} + Phi_h of row h into the ghosted engine-format row.
__device__ __forceinline__ void ix_half_prep(const IxArgs& x, int h, int tx, int TX, uint4* sRm, int* sRe, uint4* sIm,
                                             int* sIe) {
  const StepArgs& a = x.a;
  const size_t ws = (size_t)a.g.n_r * a.g.pitch;
  for (int j = tx; j < a.g.n_th; j += TX) {
    const size_t i0 = (size_t)h * a.g.pitch + j, i1 = i0 + a.g.pitch;
    uint32_t bad = 0;
    const ix::Num sR = ix::add(ix_load(a.u_in + i1, ws, bad), ix_load(a.u_in + i0, ws, bad), 0u);
    const ix::Num sI = ix::add(ix_load(a.u_in + 2 * ws + i1, ws, bad), ix_load(a.u_in + 2 * ws + i0, ws, bad), 0u);
    ix_put_ghosted(sRm, sRe, a.g.n_th, a.radius, a.g.parity, j, sR);
    ix_put_ghosted(sIm, sIe, a.g.n_th, a.radius, a.g.parity, j, sI);
  }
}

// Eq. lw1 at half node h, column j (same terms as half_point in teuk_kernels.cuh).
__device__ __forceinline__ void ix_half_point(const IxArgs& x, int h, int j, const uint4* sRm, const int* sRe,
                                              const uint4* sIm, const int* sIe, const ix::Num& half,
                                              const ix::Num& h4) {
  const StepArgs& a = x.a;
  const int pitch = a.g.pitch, rad = a.radius;
  const size_t ws = (size_t)a.g.n_r * pitch, hs = (size_t)(a.g.n_r - 1) * pitch;
  const size_t i0 = (size_t)h * pitch + j, i1 = i0 + pitch;
  uint32_t bad = 0;
  const double* u = a.u_in;
  const ix::Num uPR0 = ix_load(u + 0 * ws + i0, ws, bad), uPR1 = ix_load(u + 0 * ws + i1, ws, bad);
  const ix::Num uPI0 = ix_load(u + 2 * ws + i0, ws, bad), uPI1 = ix_load(u + 2 * ws + i1, ws, bad);
  const ix::Num uQR0 = ix_load(u + 4 * ws + i0, ws, bad), uQR1 = ix_load(u + 4 * ws + i1, ws, bad);
  const ix::Num uQI0 = ix_load(u + 6 * ws + i0, ws, bad), uQI1 = ix_load(u + 6 * ws + i1, ws, bad);
  const ix::Num dPR = ix::add(uPR1, uPR0, 1u), dPI = ix::add(uPI1, uPI0, 1u);
  const ix::Num sQR = ix::add(uQR1, uQR0, 0u), sQI = ix::add(uQI1, uQI0, 0u);
  const ix::Num sPR = ix_num(sRm[j + rad], sRe[j + rad]), sPI = ix_num(sIm[j + rad], sIe[j + rad]);
  const ix::Num LR = ix_theta(x, sRm + j, sRe + j, j), LI = ix_theta(x, sIm + j, sIe + j, j);
  const size_t ci = (size_t)h * pitch + j;
  int ce[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) ce[q] = __ldg(x.che + q * hs + ci);
  // coefficient mantissas are read at each use (L1 hits) to keep fewer registers live
  const uint4* cmp = x.chm + ci;
#define CM(q) __ldg(cmp + (q) * hs)
  ix::Acc acc;
  int mx;
  // Phi_R = s_PhiR/2 - H0 d_PhiR + (h/4) s_PiR
  mx = imax(imax(ix::prod_exp(half.e, sPR.e), ix_texp(ce[0], dPR)), ix::prod_exp(h4.e, sQR.e));
  ix::acc_zero(acc);
  ix_term(acc, half, sPR, 0u, mx);
  ix_term(acc, CM(0), ce[0], dPR, 1u, mx);
  ix_term(acc, h4, sQR, 0u, mx);
  ix_store_dd(a.uh + 0 * hs + ci, hs, ix::to_dd(acc, ix::acc_base(mx)), bad);
  // Phi_I
  mx = imax(imax(ix::prod_exp(half.e, sPI.e), ix_texp(ce[0], dPI)), ix::prod_exp(h4.e, sQI.e));
  ix::acc_zero(acc);
  ix_term(acc, half, sPI, 0u, mx);
  ix_term(acc, CM(0), ce[0], dPI, 1u, mx);
  ix_term(acc, h4, sQI, 0u, mx);
  ix_store_dd(a.uh + 2 * hs + ci, hs, ix::to_dd(acc, ix::acc_base(mx)), bad);
  // Pi_R = H3 s_PiR + H4 s_PiI + H0 (Pi_R,h+1 - Pi_R,h) + H1 d_PhiR + H2 d_PhiI + H5 L_R + H6 s_PhiR - H7 s_PhiI
  mx = imax(imax(imax(ix_texp(ce[3], sQR), ix_texp(ce[4], sQI)), imax(ix_texp(ce[0], uQR1), ix_texp(ce[0], uQR0))),
            imax(imax(ix_texp(ce[1], dPR), ix_texp(ce[2], dPI)),
                 imax(ix_texp(ce[5], LR), imax(ix_texp(ce[6], sPR), ix_texp(ce[7], sPI)))));
  ix::acc_zero(acc);
  ix_term(acc, CM(3), ce[3], sQR, 0u, mx);
  ix_term(acc, CM(4), ce[4], sQI, 0u, mx);
  ix_term(acc, CM(0), ce[0], uQR1, 0u, mx);
  ix_term(acc, CM(0), ce[0], uQR0, 1u, mx);
  ix_term(acc, CM(1), ce[1], dPR, 0u, mx);
  ix_term(acc, CM(2), ce[2], dPI, 0u, mx);
  ix_term(acc, CM(5), ce[5], LR, 0u, mx);
  ix_term(acc, CM(6), ce[6], sPR, 0u, mx);
  ix_term(acc, CM(7), ce[7], sPI, 1u, mx);
  ix_store_dd(a.uh + 4 * hs + ci, hs, ix::to_dd(acc, ix::acc_base(mx)), bad);
  // Pi_I = H3 s_PiI - H4 s_PiR + H0 (Pi_I,h+1 - Pi_I,h) + H1 d_PhiI - H2 d_PhiR + H5 L_I + H6 s_PhiI + H7 s_PhiR
  mx = imax(imax(imax(ix_texp(ce[3], sQI), ix_texp(ce[4], sQR)), imax(ix_texp(ce[0], uQI1), ix_texp(ce[0], uQI0))),
            imax(imax(ix_texp(ce[1], dPI), ix_texp(ce[2], dPR)),
                 imax(ix_texp(ce[5], LI), imax(ix_texp(ce[6], sPI), ix_texp(ce[7], sPR)))));
  ix::acc_zero(acc);
  ix_term(acc, CM(3), ce[3], sQI, 0u, mx);
  ix_term(acc, CM(4), ce[4], sQR, 1u, mx);
  ix_term(acc, CM(0), ce[0], uQI1, 0u, mx);
  ix_term(acc, CM(0), ce[0], uQI0, 1u, mx);
  ix_term(acc, CM(1), ce[1], dPI, 0u, mx);
  ix_term(acc, CM(2), ce[2], dPR, 1u, mx);
  ix_term(acc, CM(5), ce[5], LI, 0u, mx);
  ix_term(acc, CM(6), ce[6], sPI, 0u, mx);
  ix_term(acc, CM(7), ce[7], sPR, 0u, mx);
  ix_store_dd(a.uh + 6 * hs + ci, hs, ix::to_dd(acc, ix::acc_base(mx)), bad);
#undef CM
}

// Eq. lw2, first phase: s_Phi = Phi_{i+1/2} + Phi_{i-1/2} into the ghosted engine-format row.
__device__ __forceinline__ void ix_full_prep(const IxArgs& x, int i, int tx, int TX, uint4* sRm, int* sRe, uint4* sIm,
                                             int* sIe) {
  const StepArgs& a = x.a;
  const size_t hs = (size_t)(a.g.n_r - 1) * a.g.pitch;
  for (int j = tx; j < a.g.n_th; j += TX) {
    const size_t p = (size_t)i * a.g.pitch + j, m = p - a.g.pitch;
    uint32_t bad = 0;
    const ix::Num sR = ix::add(ix_load(a.uh + p, hs, bad), ix_load(a.uh + m, hs, bad), 0u);
    const ix::Num sI = ix::add(ix_load(a.uh + 2 * hs + p, hs, bad), ix_load(a.uh + 2 * hs + m, hs, bad), 0u);
    ix_put_ghosted(sRm, sRe, a.g.n_th, a.radius, a.g.parity, j, sR);
    ix_put_ghosted(sIm, sIe, a.g.n_th, a.radius, a.g.parity, j, sI);
  }
}

// Eq. lw2 at node i, column j (same terms as full_point); returns true for a non-finite value.
__device__ __forceinline__ bool ix_full_point(const IxArgs& x, int i, int j, const uint4* sRm, const int* sRe,
                                              const uint4* sIm, const int* sIe, const ix::Num& one,
                                              const ix::Num& h2, long long slot) {
  const StepArgs& a = x.a;
  const int pitch = a.g.pitch, rad = a.radius, n_th = a.g.n_th;
  const size_t ws = (size_t)a.g.n_r * pitch, hs = (size_t)(a.g.n_r - 1) * pitch;
  const size_t p = (size_t)i * pitch + j, m = p - pitch;
  uint32_t bad = 0;
  const double* uh = a.uh;
  const ix::Num hPR1 = ix_load(uh + 0 * hs + p, hs, bad), hPR0 = ix_load(uh + 0 * hs + m, hs, bad);
  const ix::Num hPI1 = ix_load(uh + 2 * hs + p, hs, bad), hPI0 = ix_load(uh + 2 * hs + m, hs, bad);
  const ix::Num hQR1 = ix_load(uh + 4 * hs + p, hs, bad), hQR0 = ix_load(uh + 4 * hs + m, hs, bad);
  const ix::Num hQI1 = ix_load(uh + 6 * hs + p, hs, bad), hQI0 = ix_load(uh + 6 * hs + m, hs, bad);
  const ix::Num dPR = ix::add(hPR1, hPR0, 1u), dPI = ix::add(hPI1, hPI0, 1u);
  const ix::Num sQR = ix::add(hQR1, hQR0, 0u), sQI = ix::add(hQI1, hQI0, 0u);
  const ix::Num sPR = ix_num(sRm[j + rad], sRe[j + rad]), sPI = ix_num(sIm[j + rad], sIe[j + rad]);
  const ix::Num LR = ix_theta(x, sRm + j, sRe + j, j), LI = ix_theta(x, sIm + j, sIe + j, j);
  const size_t ci = (size_t)i * pitch + j;
  const ix::Num PR = ix_load(a.u_in + 0 * ws + ci, ws, bad), PI = ix_load(a.u_in + 2 * ws + ci, ws, bad);
  const ix::Num QR = ix_load(a.u_in + 4 * ws + ci, ws, bad), QI = ix_load(a.u_in + 6 * ws + ci, ws, bad);
  int ce[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) ce[q] = __ldg(x.cne + q * ws + ci);
  const uint4* cmp = x.cnm + ci;
#define CM(q) __ldg(cmp + (q) * ws)
  ix::Acc acc;
  int mx;
  mw::dd out[4];
  // Phi_R' = Phi_R - N0 d_PhiR + (h/2) s_PiR
  mx = imax(imax(ix::prod_exp(one.e, PR.e), ix_texp(ce[0], dPR)), ix::prod_exp(h2.e, sQR.e));
  ix::acc_zero(acc);
  ix_term(acc, one, PR, 0u, mx);
  ix_term(acc, CM(0), ce[0], dPR, 1u, mx);
  ix_term(acc, h2, sQR, 0u, mx);
  out[0] = ix::to_dd(acc, ix::acc_base(mx));
  // Phi_I'
  mx = imax(imax(ix::prod_exp(one.e, PI.e), ix_texp(ce[0], dPI)), ix::prod_exp(h2.e, sQI.e));
  ix::acc_zero(acc);
  ix_term(acc, one, PI, 0u, mx);
  ix_term(acc, CM(0), ce[0], dPI, 1u, mx);
  ix_term(acc, h2, sQI, 0u, mx);
  out[1] = ix::to_dd(acc, ix::acc_base(mx));
  // Pi_R' = Pi_R + N0 (h_PiR,i+1/2 - h_PiR,i-1/2) + N1 d_PhiR + N2 d_PhiI + N3 s_PiR + N4 s_PiI + N5 L_R
  //         + N6 s_PhiR - N7 s_PhiI
  mx = imax(imax(imax(ix::prod_exp(one.e, QR.e), ix_texp(ce[0], hQR1)), imax(ix_texp(ce[0], hQR0), ix_texp(ce[1], dPR))),
            imax(imax(ix_texp(ce[2], dPI), ix_texp(ce[3], sQR)),
                 imax(imax(ix_texp(ce[4], sQI), ix_texp(ce[5], LR)), imax(ix_texp(ce[6], sPR), ix_texp(ce[7], sPI)))));
  ix::acc_zero(acc);
  ix_term(acc, one, QR, 0u, mx);
  ix_term(acc, CM(0), ce[0], hQR1, 0u, mx);
  ix_term(acc, CM(0), ce[0], hQR0, 1u, mx);
  ix_term(acc, CM(1), ce[1], dPR, 0u, mx);
  ix_term(acc, CM(2), ce[2], dPI, 0u, mx);
  ix_term(acc, CM(3), ce[3], sQR, 0u, mx);
  ix_term(acc, CM(4), ce[4], sQI, 0u, mx);
  ix_term(acc, CM(5), ce[5], LR, 0u, mx);
  ix_term(acc, CM(6), ce[6], sPR, 0u, mx);
  ix_term(acc, CM(7), ce[7], sPI, 1u, mx);
  out[2] = ix::to_dd(acc, ix::acc_base(mx));
  // Pi_I' = Pi_I + N0 (h_PiI,i+1/2 - h_PiI,i-1/2) + N1 d_PhiI - N2 d_PhiR + N3 s_PiI - N4 s_PiR + N5 L_I
  //         + N6 s_PhiI + N7 s_PhiR
  mx = imax(imax(imax(ix::prod_exp(one.e, QI.e), ix_texp(ce[0], hQI1)), imax(ix_texp(ce[0], hQI0), ix_texp(ce[1], dPI))),
            imax(imax(ix_texp(ce[2], dPR), ix_texp(ce[3], sQI)),
                 imax(imax(ix_texp(ce[4], sQR), ix_texp(ce[5], LI)), imax(ix_texp(ce[6], sPI), ix_texp(ce[7], sPR)))));
  ix::acc_zero(acc);
  ix_term(acc, one, QI, 0u, mx);
  ix_term(acc, CM(0), ce[0], hQI1, 0u, mx);
  ix_term(acc, CM(0), ce[0], hQI0, 1u, mx);
  ix_term(acc, CM(1), ce[1], dPI, 0u, mx);
  ix_term(acc, CM(2), ce[2], dPR, 1u, mx);
  ix_term(acc, CM(3), ce[3], sQI, 0u, mx);
  ix_term(acc, CM(4), ce[4], sQR, 1u, mx);
  ix_term(acc, CM(5), ce[5], LI, 0u, mx);
  ix_term(acc, CM(6), ce[6], sPI, 0u, mx);
  ix_term(acc, CM(7), ce[7], sPR, 0u, mx);
  out[3] = ix::to_dd(acc, ix::acc_base(mx));
#undef CM
  for (int c = 0; c < 4; ++c) ix_store_dd(a.u_out + 2 * c * ws + ci, ws, out[c], bad);
  if (slot >= 0 && i == a.i_obs && !bad) {
    double* dst = a.ring + (size_t)slot * 2 * 2 * n_th;
    dst[0 * n_th + j] = out[0].h;
    dst[1 * n_th + j] = out[0].l;
    dst[2 * n_th + j] = out[1].h;
    dst[3 * n_th + j] = out[1].l;
  }
  return bad || nonfinite(out[0].h) || nonfinite(out[1].h) || nonfinite(out[2].h) || nonfinite(out[3].h);
}

// Shared memory of the engine kernels: per row, mantissas [2][gstride] (uint4) first, then the
// exponent-sign words [2][gstride] (int), for blockDim.y rows.
__device__ __forceinline__ void ix_rows(int gstride, uint4*& sRm, int*& sRe, uint4*& sIm, int*& sIe) {
  extern __shared__ uint4 ixsm[];
  const int rows = blockDim.y, y = threadIdx.y;
  uint4* mbase = ixsm;
  int* ebase = reinterpret_cast<int*>(ixsm + (size_t)rows * 2 * gstride);
  sRm = mbase + (size_t)y * 2 * gstride;
  sIm = sRm + gstride;
  sRe = ebase + (size_t)y * 2 * gstride;
  sIe = sRe + gstride;
}

template <int V>
__global__ void __launch_bounds__(RowBounds<V>::threads, RowBounds<V>::blocks) half_ix_kernel(IxArgs x) {
  const int gstride = x.a.g.n_th + 2 * x.a.radius;
  uint4 *sRm, *sIm;
  int *sRe, *sIe;
  ix_rows(gstride, sRm, sRe, sIm, sIe);
  const int h = blockIdx.x * blockDim.y + threadIdx.y;
  const bool ok = h < x.a.g.n_r - 1;
  if (ok) ix_half_prep(x, h, threadIdx.x, blockDim.x, sRm, sRe, sIm, sIe);
  __syncthreads();
  if (!ok) return;
  uint32_t bad = 0;
  const ix::Num half{{0u, 0u, 0u, 0x40000000u}, -127, 0u};
  const ix::Num h4 = ix::from_dd(x.a.h4[0], x.a.h4[1], bad);
  for (int j = threadIdx.x; j < x.a.g.n_th; j += blockDim.x) ix_half_point(x, h, j, sRm, sRe, sIm, sIe, half, h4);
}

template <int V>
__global__ void __launch_bounds__(RowBounds<V>::threads, RowBounds<V>::blocks) full_ix_kernel(IxArgs x) {
  const int gstride = x.a.g.n_th + 2 * x.a.radius;
  uint4 *sRm, *sIm;
  int *sRe, *sIe;
  ix_rows(gstride, sRm, sRe, sIm, sIe);
  const int i = 1 + blockIdx.x * blockDim.y + threadIdx.y;
  const bool ok = i < x.a.g.n_r - 1;
  if (ok) ix_full_prep(x, i, threadIdx.x, blockDim.x, sRm, sRe, sIm, sIe);
  __syncthreads();
  if (!ok) return;
  uint32_t bad = 0;
  const ix::Num one{{0u, 0u, 0u, 0x40000000u}, -126, 0u};
  const ix::Num h2 = ix::from_dd(x.a.h2[0], x.a.h2[1], bad);
  long long slot = -1;
  if (x.a.record) slot = x.a.ring_slot >= 0 ? x.a.ring_slot : (*x.a.ring_counter) % x.a.ring_cap;
  bool anybad = false;
  for (int j = threadIdx.x; j < x.a.g.n_th; j += blockDim.x)
    anybad |= ix_full_point(x, i, j, sRm, sRe, sIm, sIe, one, h2, slot);
  if (anybad) atomicOr(x.a.status, 1u);
}

}  // namespace teuk
