// Per-precision set-up and launchers of the teuk library. Compiled once per arithmetic with
// -DTEUK_WORDS=1 (FP64), 2 (double-double) or 4 (quad-double).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ix.cuh"
#include "teuk_internal.h"
#include "teuk_kernels.cuh"
#if TEUK_WORDS != 1
#include "teuk_ix.cuh"
#endif

#ifndef TEUK_WORDS
#error "TEUK_WORDS must be 1, 2 or 4"
#endif

#define TEUK_CAT2(a, b) a##b
#define TEUK_CAT(a, b) TEUK_CAT2(a, b)
#define TEUK_SUFFIX(name) TEUK_CAT(name, TEUK_WORDS)

namespace teuk {
// one named namespace per arithmetic: the three units are built from the same file
namespace TEUK_SUFFIX(prec_w) {

constexpr int W = TEUK_WORDS;
using R = typename RT<W>::T;
using namespace mw;

void put(double* dst, R v) { to_words(v, dst); }

// Host-side word planes of a 1D table in the target precision: out[k * n + j].
void store_plane(std::vector<double>& out, int n, int j, R v) {
  double w[4];
  to_words(v, w);
  for (int k = 0; k < W; ++k) out[(size_t)k * n + j] = w[k];
}

// 10th-order (Sec. 3.D) and 2nd-order (Sec. 3.B) centred weights on a uniform grid,
// scaled to integers: d2 / 25200 and d1 / 2520 for the 11-point stencil.
const double kD2_10[11] = {8, -125, 1000, -6000, 42000, -73766, 42000, -6000, 1000, -125, 8};
const double kD1_10[11] = {-2, 25, -150, 600, -2100, 0, 2100, -600, 150, -25, 2};
const double kD2_2[3] = {1, -2, 1};
const double kD1_2[3] = {-1, 0, 1};

int setup_impl(teuk_s* h) {
  const teuk_grid& g = h->grid;
  const int n_r = h->n_r, n_th = h->n_th, pitch = h->pitch;
  const R M = r_from<R>(h->M), a = r_from<R>(h->a);
  const R root = r_sqrt(r_sub(r_mul(M, M), r_mul(a, a)));
  const R rp = r_add(M, root);
  const R rm = r_div(r_mul(a, a), rp);  // r+ r- = a^2
  const R twoM = r_from<R>(2.0 * h->M);
  const R A = r_div(r_mul(twoM, rp), r_sub(rp, rm));
  const R B = r_neg(r_div(r_mul(twoM, rm), r_sub(rp, rm)));
  const R pi = r_pi<R>();
  const R ln2 = r_ln2<R>();
  const R ln2M = r_log(twoM, ln2);
  const R rsmin = r_from<R>(g.rstar_min);
  const R dr = r_div(r_sub(r_from<R>(g.rstar_max), rsmin), r_from<R>(double(g.n_r - 1)));  // global rows
  const R dt = g.dt > 0 ? r_from<R>(g.dt) : r_scale2(dr, 0.25);
  const R dts = r_div(dt, r_from<R>(double(h->k)));
  const R lambda = r_div(dts, dr);
  h->dt_outer = lead(dt);
  h->dr_d = lead(dr);
  h->rsmin_d = g.rstar_min;
  put(h->dt_w, dt);
  put(h->dr_w, dr);
  put(h->h4_w, r_scale2(dts, 0.25));
  put(h->h2_w, r_scale2(dts, 0.5));
  put(h->ln2_w, ln2);

  // theta grid (cell centred), sin, cos and the combined stencil weights
  const R dth = r_div(pi, r_from<R>(double(n_th)));
  const int rad = h->radius, nq = 2 * rad + 1;
  const double* d2 = rad == 5 ? kD2_10 : kD2_2;
  const double* d1 = rad == 5 ? kD1_10 : kD1_2;
  const R A2 = rad == 5 ? r_div(r_from<R>(1.0), r_mul_d(r_mul(dth, dth), 25200.0))
                        : r_div(r_from<R>(1.0), r_mul(dth, dth));
  const R A1 = rad == 5 ? r_div(r_from<R>(1.0), r_mul_d(dth, 2520.0))
                        : r_div(r_from<R>(1.0), r_mul_d(dth, 2.0));
  std::vector<double> sn((size_t)W * n_th), cs((size_t)W * n_th), wt((size_t)nq * W * n_th);
  std::vector<double> lf((size_t)2 * W * n_th);  // weight_q = A2 d2_q + (A1 cot) d1_q
  for (int j = 0; j < n_th; ++j) {
    const R th = r_mul_d(dth, double(j) + 0.5);
    R s, c;
    r_sincos(th, pi, s, c);
    store_plane(sn, n_th, j, s);
    store_plane(cs, n_th, j, c);
    const R cot = r_div(c, s);
    {
      double w[4];
      to_words(A2, w);
      for (int k = 0; k < W; ++k) lf[(size_t)k * n_th + j] = w[k];
      to_words(r_mul(A1, cot), w);
      for (int k = 0; k < W; ++k) lf[((size_t)W + k) * n_th + j] = w[k];
    }
    for (int q = 0; q < nq; ++q) {
      const R wq = r_add(r_mul_d(A2, d2[q]), r_mul(r_mul_d(A1, d1[q]), cot));
      double w[4];
      to_words(wq, w);
      for (int k = 0; k < W; ++k) wt[((size_t)q * W + k) * n_th + j] = w[k];
    }
  }
  TEUK_CUDA(h, cudaMemcpyAsync(h->sin_th, sn.data(), sn.size() * 8, cudaMemcpyHostToDevice, h->stream));
  TEUK_CUDA(h, cudaMemcpyAsync(h->cos_th, cs.data(), cs.size() * 8, cudaMemcpyHostToDevice, h->stream));
  TEUK_CUDA(h, cudaMemcpyAsync(h->wts, wt.data(), wt.size() * 8, cudaMemcpyHostToDevice, h->stream));
  TEUK_CUDA(h, cudaMemcpyAsync(h->lfac, lf.data(), lf.size() * 8, cudaMemcpyHostToDevice, h->stream));

  SetupArgs sa{};
  sa.g = Geom{n_r, n_th, pitch, h->parity};
  sa.row0 = h->row0;
  sa.W = W;
  sa.M = h->M;
  sa.a = h->a;
  sa.s = h->s;
  sa.m = h->m;
  put(sa.rp, rp); put(sa.rm, rm); put(sa.tort_A, A); put(sa.tort_B, B);
  put(sa.ln2, ln2); put(sa.ln2M, ln2M); put(sa.rsmin, rsmin); put(sa.dr, dr);
  put(sa.dts, dts); put(sa.lambda, lambda);
  sa.sin_th = h->sin_th;
  sa.cos_th = h->cos_th;
  sa.x_node = h->x_node;
  sa.x_half = h->x_half;
  sa.rs_node = h->rs_node;
  sa.cn_raw = h->cn_raw;
  sa.ch_raw = h->ch_raw;
  sa.cn = h->cn;
  sa.ch = h->ch;
  const int rows_total = 2 * n_r - 1;
  tortoise_kernel<W><<<(rows_total + 63) / 64, 64, 0, h->stream>>>(sa);
  TEUK_CUDA(h, cudaGetLastError());
  dim3 blk(64);
  coeff_kernel<W><<<dim3((n_th + 63) / 64, n_r), blk, 0, h->stream>>>(sa, 0);
  TEUK_CUDA(h, cudaGetLastError());
  coeff_kernel<W><<<dim3((n_th + 63) / 64, n_r - 1), blk, 0, h->stream>>>(sa, 1);
  TEUK_CUDA(h, cudaGetLastError());
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  return TEUK_OK;
}

double binom(int n, int k) {
  if (k < 0 || n < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int t = 1; t <= k; ++t) r = r * (n - k + t) / t;
  return std::round(r);
}

// Goldberg et al. (1967) sum of sY_lm(theta), without its normalisation and e^{i m phi}:
//   sum_r (-1)^(l-r-s) C(l-s, r) C(l+s, r+s-m) sin(th/2)^(2l-2r-s+m) cos(th/2)^(2r+s-m).
// The binomial coefficients are exact doubles for l <= 40; their product is formed in R.
R goldberg_sum(int ell, int s, int m, R sh, R ch) {
  R sum = r_from<R>(0.0);
  for (int r = 0; r <= ell - s; ++r) {
    const double b1 = binom(ell - s, r), b2 = binom(ell + s, r + s - m);
    if (b1 == 0.0 || b2 == 0.0) continue;
    R term = r_mul(r_from<R>(b1), r_from<R>(b2));
    if ((ell - r - s) % 2 != 0) term = r_neg(term);
    for (int e = 0; e < 2 * ell - 2 * r - s + m; ++e) term = r_mul(term, sh);
    for (int e = 0; e < 2 * r + s - m; ++e) term = r_mul(term, ch);
    sum = r_add(sum, term);
  }
  return sum;
}

// sin(theta_j / 2), cos(theta_j / 2) at the cell centre theta_j = (j + 1/2) pi / n_theta.
void half_angle(const R& pi, int n_th, int j, R& sh, R& ch) {
  const R dth = r_div(pi, r_from<R>(double(n_th)));
  const R half_th = r_scale2(r_mul_d(dth, double(j) + 0.5), 0.5);
  r_sincos(half_th, pi, sh, ch);
}

int pulse_impl(teuk_s* h, double center, double width, double ar, double ai, int ell) {
  const int n_th = h->n_th, s = h->s, m = h->m;
  const R pi = r_pi<R>();
  std::vector<double> prof((size_t)W * n_th);
  for (int j = 0; j < n_th; ++j) {
    R sh, ch;
    half_angle(pi, n_th, j, sh, ch);
    store_plane(prof, n_th, j, goldberg_sum(ell, s, m, sh, ch));
  }
  TEUK_CUDA(h, cudaMemcpyAsync(h->prof, prof.data(), prof.size() * 8, cudaMemcpyHostToDevice, h->stream));
  PulseArgs pa{};
  pa.g = Geom{h->n_r, n_th, h->pitch, h->parity};
  pa.row0 = h->row0;
  pa.n_r_global = h->grid.n_r;
  pa.center = center;
  pa.width = width;
  pa.amp_re = ar;
  pa.amp_im = ai;
  std::memcpy(pa.ln2, h->ln2_w, sizeof(pa.ln2));
  pa.rs_node = h->rs_node;
  pa.prof = h->prof;
  pa.cn_raw = h->cn_raw;
  pa.u = h->u;
  pulse_kernel<W><<<dim3((n_th + 63) / 64, h->n_r), 64, 0, h->stream>>>(pa);
  TEUK_CUDA(h, cudaGetLastError());
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  return TEUK_OK;
}

// Multipole projection of the recorded waveform (Sec. 3.C: the tail of each multipole l of
// the field seen by an observer, Fig. 1). For l = ell_min .. ell_max:
//   c_l(t) = 2 pi int_0^pi Phi(t, theta) sY_lm(theta) sin(theta) dtheta
// with the normalised harmonic sY_lm = (-1)^m sqrt((2l+1)/(4 pi) (l+m)!(l-m)!/((l+s)!(l-s)!))
// x goldberg_sum. With x = cos(theta) the integral is int_{-1}^{1} Phi sY dx, and the cell
// centres x_j = cos((j + 1/2) pi / N) are the nodes of Fejer's first rule, weights
//   w_j = (2/N) [1 - 2 sum_{k=1}^{floor(N/2)} cos(2 k theta_j) / (4 k^2 - 1)],
// exact for polynomials of degree < N (the integrand of a regular field is a polynomial in x
// times its smooth amplitude). The cosines are cos(pi q / (2N)) with the integer
// q = 2k(2j+1) reduced exactly to the first quadrant. harmonic_table gives sY_lm(theta_j) as
// words [n_ell][W][n_th], times 2 pi w_j when `weighted` (the projection's table).
std::vector<double> harmonic_table(int s, int m, int n_th, int ell_min, int ell_max, bool weighted) {
  const int n_ell = ell_max - ell_min + 1;
  const R pi = r_pi<R>();
  // quarter-wave table cos(pi q / (2N)), q = 0 .. N
  std::vector<R> qc(n_th + 1);
  const R step = r_scale2(r_div(pi, r_from<R>(double(n_th))), 0.5);
  for (int q = 0; q <= n_th; ++q) {
    R sq, cq;
    r_sincos(r_mul_d(step, double(q)), pi, sq, cq);
    qc[q] = cq;
  }
  qc[0] = r_from<R>(1.0);
  qc[n_th] = r_from<R>(0.0);
  auto cos_q = [&](long long q) -> R {
    q %= 4LL * n_th;
    if (q > 2LL * n_th) q = 4LL * n_th - q;        // cos(2 pi - x) = cos(x)
    if (q > n_th) return r_neg(qc[2 * n_th - q]);  // cos(pi - x) = -cos(x)
    return qc[q];
  };
  std::vector<R> inv_k(n_th / 2 + 1);
  for (int k = 1; k <= n_th / 2; ++k) inv_k[k] = r_div(r_from<R>(1.0), r_from<R>(4.0 * k * k - 1.0));
  std::vector<R> wq(n_th);
  for (int j = 0; j < n_th; ++j) {
    R sum = r_from<R>(0.0);
    for (int k = 1; k <= n_th / 2; ++k) sum = r_add(sum, r_mul(cos_q(2LL * k * (2 * j + 1)), inv_k[k]));
    // 2 pi w_j = (4 pi / N) (1 - 2 sum)
    wq[j] = r_mul(r_div(r_scale2(pi, 4.0), r_from<R>(double(n_th))), r_sub(r_from<R>(1.0), r_scale2(sum, 2.0)));
  }
  std::vector<double> table((size_t)n_ell * W * n_th);
  for (int l = ell_min; l <= ell_max; ++l) {
    // (l+m)!(l-m)! / ((l+s)!(l-s)!) as a product of exact integer ratios
    R ratio = r_from<R>(1.0);
    for (int t = 2; t <= l + m; ++t) ratio = r_mul_d(ratio, double(t));
    for (int t = 2; t <= l - m; ++t) ratio = r_mul_d(ratio, double(t));
    for (int t = 2; t <= l + s; ++t) ratio = r_div_d(ratio, double(t));
    for (int t = 2; t <= l - s; ++t) ratio = r_div_d(ratio, double(t));
    R norm = r_sqrt(r_div(r_mul_d(ratio, double(2 * l + 1)), r_scale2(pi, 4.0)));
    if (m % 2 != 0) norm = r_neg(norm);
    std::vector<double> row((size_t)W * n_th);
    for (int j = 0; j < n_th; ++j) {
      R sh, ch;
      half_angle(pi, n_th, j, sh, ch);
      const R y = r_mul(norm, goldberg_sum(l, s, m, sh, ch));
      store_plane(row, n_th, j, weighted ? r_mul(wq[j], y) : y);
    }
    std::memcpy(table.data() + (size_t)(l - ell_min) * W * n_th, row.data(), row.size() * sizeof(double));
  }
  return table;
}

int project_impl(teuk_s* h, int ell_min, int ell_max, double* out, int64_t n, int64_t first) {
  const int n_th = h->n_th, n_ell = ell_max - ell_min + 1;
  const std::vector<double> table = harmonic_table(h->s, h->m, n_th, ell_min, ell_max, true);
  double* d_table = nullptr;
  double* d_out = nullptr;
  const size_t n_out = (size_t)n * n_ell * 2 * W;
  auto release = [&]() {
    if (d_table) cudaFree(d_table);
    if (d_out) cudaFree(d_out);
  };
  cudaError_t e;
  if ((e = cudaMalloc(&d_table, table.size() * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&d_out, n_out * sizeof(double))) != cudaSuccess) {
    release();
    return cuda_fail(h, e, "cudaMalloc (projection)");
  }
  ProjectArgs pa{};
  pa.n_th = n_th;
  pa.n_ell = n_ell;
  pa.n = n;
  pa.first = first;
  pa.cap = h->ring_cap;
  pa.ring = h->ring;
  pa.table = d_table;
  pa.out = d_out;
  const long long threads = (long long)n * n_ell * 2;
  if ((e = cudaMemcpyAsync(d_table, table.data(), table.size() * sizeof(double), cudaMemcpyHostToDevice,
                           h->stream)) == cudaSuccess) {
    project_kernel<W><<<(unsigned)((threads + 127) / 128), 128, 0, h->stream>>>(pa);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, d_out, n_out * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  release();
  if (e != cudaSuccess) return cuda_fail(h, e, "projection");
  return TEUK_OK;
}

// r* dissipation strength eps = sigma dt / (16 dr*) in the target precision.
int dissipation_impl(teuk_s* h, double sigma) {
  const R dt = from_words<R>(h->dt_w), dr = from_words<R>(h->dr_w);
  put(h->ko_eps_w, r_div(r_mul(r_from<R>(sigma), dt), r_mul(r_from<R>(16.0), dr)));
  return TEUK_OK;
}

// theta dissipation: eps_th(i) = sigma c_th(i) dt / (4096 dtheta) per row, in the target
// precision (h->eps_th allocated by the caller); *max_rate = max_i 4096 eps_th(i), the largest
// damping factor of one step (the grid-scale theta mode is multiplied by 1 - max_rate).
int theta_dissipation_impl(teuk_s* h, double sigma, double* max_rate) {
  const R dt = from_words<R>(h->dt_w);
  const R dth = r_div(r_pi<R>(), r_from<R>(double(h->n_th)));
  const R fac = r_div(r_mul(r_from<R>(sigma), dt), r_mul(r_from<R>(4096.0), dth));
  double f[4];
  put(f, fac);
  theta_ko_eps_kernel<W><<<h->n_r, 256, 0, h->stream>>>(Geom{h->n_r, h->n_th, h->pitch, h->parity}, h->cn_raw,
                                                         h->eps_th, f[0], f[1], f[2], f[3]);
  TEUK_CUDA(h, cudaGetLastError());
  std::vector<double> lead_eps(h->n_r);
  TEUK_CUDA(h, cudaMemcpyAsync(lead_eps.data(), h->eps_th, h->n_r * sizeof(double), cudaMemcpyDeviceToHost,
                               h->stream));
  TEUK_CUDA(h, cudaStreamSynchronize(h->stream));
  double mx = 0;
  for (double e : lead_eps) mx = e > mx ? e : mx;
  *max_rate = 4096.0 * mx;
  return TEUK_OK;
}

// Launch of filter_kernel: 256 threads per row; each coefficient split into the largest power
// of two (at most 8) of partial dot products that keeps the 4 n_ell coefficients within them.
constexpr int kFilterThreads = 256;
int filter_split(int n_ell) {
  int sp = 1;
  while (sp < 8 && 4 * n_ell * sp * 2 <= kFilterThreads) sp *= 2;
  return sp;
}
size_t filter_smem(int n_th, int n_ell) {
  return filter_smem_doubles(W, n_th, n_ell, filter_split(n_ell)) * sizeof(double);
}

// Tables of the theta filter: [2][n_ell][W][n_th], first 2 pi w_j sY_lm(theta_j) (analysis),
// then sY_lm(theta_j) (synthesis), l = max(|s|, |m|) .. l_cut - 1. The harmonics come from
// the quad-double evaluation and keep their leading W words: the Goldberg sum alternates,
// and at l ~ 20 its terms are ~1e5 times its value, which a W-word evaluation would leave in
// the result.
int filter_tables_impl(teuk_s* h, int l_cut) {
  const int l_low = std::max(std::abs(h->s), std::abs(h->m)), n_ell = l_cut - l_low, n_th = h->n_th;
  std::vector<double> tab((size_t)2 * n_ell * W * n_th);
  for (int part = 0; part < 2; ++part) {
    const std::vector<double> q = harmonics_w4(h->s, h->m, n_th, l_low, l_cut - 1, part == 0);
    double* dst = tab.data() + (size_t)part * n_ell * W * n_th;
    for (int l = 0; l < n_ell; ++l)
      for (int k = 0; k < W; ++k)
        std::memcpy(dst + ((size_t)l * W + k) * n_th, q.data() + ((size_t)l * 4 + k) * n_th, n_th * sizeof(double));
  }
  if (h->filt) cudaFree(h->filt);
  h->filt = nullptr;
  TEUK_CUDA(h, cudaMalloc(&h->filt, tab.size() * sizeof(double)));
  TEUK_CUDA(h, cudaMemcpy(h->filt, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice));
  const size_t smem = filter_smem(n_th, n_ell);
  if (smem > 48 * 1024)
    TEUK_CUDA(h, cudaFuncSetAttribute(filter_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  return TEUK_OK;
}

// The operators of an outer step's start: the dissipation kernel into u_ko, then either the
// theta filter kernel from u_ko back into the state (it projects every filter_period-th outer
// step and copies otherwise) or a copy back; the filter alone works in place. The filter
// kernel is launched without programmatic dependence: its blocks would otherwise become
// resident early behind the dissipation kernel, and the step kernels behind it.
int dissipate_impl(teuk_s* h) {
  const bool ko = h->ko_sigma > 0 || h->ko_theta > 0;
  if (ko) {
    DissArgs da{};
    da.g = Geom{h->n_r, h->n_th, h->pitch, h->parity};
    da.u = h->u;
    da.out = h->u_ko;
    std::memcpy(da.eps, h->ko_eps_w, sizeof(da.eps));
    da.eps_single = h->ko_eps_w[1] == 0 && h->ko_eps_w[2] == 0 && h->ko_eps_w[3] == 0;
    da.do_r = h->ko_sigma > 0;
    da.eps_th = h->ko_theta > 0 ? h->eps_th : nullptr;
    TEUK_CUDA(h, launch_dep(dissipate_kernel<W>, dim3((h->n_th + 63) / 64, h->n_r, 4), dim3(64), 0, h->stream,
                            da));
    TEUK_CUDA(h, cudaGetLastError());
    h->launches += 1;
  }
  if (h->filter_lcut > 0) {
    FilterArgs fa{};
    fa.g = Geom{h->n_r, h->n_th, h->pitch, h->parity};
    fa.u = ko ? h->u_ko : h->u;
    fa.out = h->u;
    fa.tab = h->filt;
    fa.n_ell = h->filter_n_ell();
    fa.split = filter_split(fa.n_ell);
    fa.ctr = h->d_filter_ctr;
    fa.period = h->filter_period;
    filter_kernel<W><<<dim3(h->n_r - 2), dim3(kFilterThreads), filter_smem(h->n_th, fa.n_ell), h->stream>>>(fa);
    TEUK_CUDA(h, cudaGetLastError());
    h->launches += 1;
  } else if (ko) {
    TEUK_CUDA(h, cudaMemcpyAsync(h->u, h->u_ko, (size_t)4 * W * h->n_r * h->pitch * sizeof(double),
                                 cudaMemcpyDeviceToDevice, h->stream));
  }
  return TEUK_OK;
}

// Arithmetic engine of the double-double step (0: FP64 error-free transforms, 1: integer
// engine). The integer engine keeps the coefficient tables in its own format, converted here
// once from the multi-word tables, with the theta operator's factors folded into plane 5 and
// a ninth plane (ix_fold_kernel).
int engine_impl(teuk_s* h, int engine) {
  if (engine == 0) {
    h->engine = 0;
    return TEUK_OK;
  }
#if TEUK_WORDS != 1
  if (!h->ix_m) {
    const int rc = W == 2 ? ix_tables_w2(h) : ix_tables_w4(h);
    if (rc != TEUK_OK) return rc;
  }
  h->engine = 1;
  return TEUK_OK;
#else
  h->last_error = "the integer engine is for double-double and quad-double handles";
  return TEUK_ERR_INVALID_ARG;
#endif
}

// Launch shape of the step kernels: threads along theta (x, one warp multiple up to 256) and
// rows per block (y). Default: about 128 threads per block, so that the last wave of blocks
// still spreads over every SM; teuk_tune picks the fastest rows-per-block instead.
void step_shape(const teuk_s* h, dim3& blk) {
  int tx, ty;
  row_block_shape(h, tx, ty);
  blk = dim3(tx, ty);
}

// Grid of the balanced kernels: every block that fits on the GPU at once (occupancy x SMs),
// computed once per (variant, threads) and kept in the handle.
template <int V>
int bal_grid(teuk_s* h, dim3 blk, size_t smem) {
  const int key = V * 4096 + (int)blk.x;
  if (h->bal_key == key) return TEUK_OK;
  if (smem > 48 * 1024) {
    TEUK_CUDA(h, cudaFuncSetAttribute(half_bal_kernel<W, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TEUK_CUDA(h, cudaFuncSetAttribute(full_bal_kernel<W, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  int sms = 0, per_h = 0, per_f = 0;
  TEUK_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  TEUK_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_h, half_bal_kernel<W, V>, (int)blk.x, smem));
  TEUK_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_f, full_bal_kernel<W, V>, (int)blk.x, smem));
  if (per_h < 1 || per_f < 1) return cuda_fail(h, cudaErrorInvalidConfiguration, "balanced kernels do not fit");
  h->bal_grid[0] = per_h * sms;
  h->bal_grid[1] = per_f * sms;
  h->bal_key = key;
  return TEUK_OK;
}

// Host-side preparation of the current launch shape (before a graph capture).
int prepare_impl(teuk_s* h) {
  if (h->kernel_family != 2) return TEUK_OK;
  dim3 blk;
  step_shape(h, blk);
  const size_t smem = (size_t)2 * W * (h->n_th + 2 * h->radius) * sizeof(double);
  switch (h->kernel_variant) {
    case 1: return bal_grid<1>(h, blk, smem);
    case 2: return bal_grid<2>(h, blk, smem);
    default: return bal_grid<0>(h, blk, smem);
  }
}

// Launches the half and full kernels of the handle's register-budget variant.
template <int V>
int launch_pair_v(teuk_s* h, const StepArgs& sa, dim3 blk, size_t smem) {
  const int nh = h->n_r - 1, nf = h->n_r - 2;
#if TEUK_WORDS != 1
  if (h->engine == 1)  // integer engine (teuk_ixk.cu)
    return W == 2 ? ix_launch_pair_w2(h, sa, blk, V) : ix_launch_pair_w4(h, sa, blk, V);
#endif
  if (h->kernel_family == 1) {
    const int nseg = (h->n_th + 31) / 32;
    const size_t seg_smem = (size_t)4 * 2 * W * (32 + 2 * h->radius) * sizeof(double);
    const int64_t units_h = (int64_t)nh * nseg, units_f = (int64_t)nf * nseg;
    cudaEvent_t ev = nullptr;
    time_begin(h, &ev);
    TEUK_CUDA(h, launch_dep(half_seg_kernel<W, V>, dim3((unsigned)((units_h + 3) / 4)), dim3(128), seg_smem,
                            h->stream, sa, nseg));
    time_end(h, 0, ev);
    time_begin(h, &ev);
    TEUK_CUDA(h, launch_dep(full_seg_kernel<W, V>, dim3((unsigned)((units_f + 3) / 4)), dim3(128), seg_smem,
                            h->stream, sa, nseg));
    time_end(h, 1, ev);
    h->launches += 2;
    TEUK_CUDA(h, cudaGetLastError());
    return TEUK_OK;
  }
  if (h->kernel_family == 2) {
    const int rc = bal_grid<V>(h, blk, smem);
    if (rc != TEUK_OK) return rc;
    cudaEvent_t ev = nullptr;
    time_begin(h, &ev);
    TEUK_CUDA(h, launch_dep(half_bal_kernel<W, V>, dim3(h->bal_grid[0]), dim3(blk.x), smem, h->stream, sa));
    time_end(h, 0, ev);
    time_begin(h, &ev);
    TEUK_CUDA(h, launch_dep(full_bal_kernel<W, V>, dim3(h->bal_grid[1]), dim3(blk.x), smem, h->stream, sa));
    time_end(h, 1, ev);
    h->launches += 2;
    TEUK_CUDA(h, cudaGetLastError());
    return TEUK_OK;
  }
  if (smem > 48 * 1024) {  // above the default dynamic limit (quad-double, n_theta > 700)
    TEUK_CUDA(h, cudaFuncSetAttribute(half_kernel<W, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TEUK_CUDA(h, cudaFuncSetAttribute(full_kernel<W, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  cudaEvent_t ev = nullptr;
  time_begin(h, &ev);
  TEUK_CUDA(h, launch_dep(half_kernel<W, V>, dim3((nh + blk.y - 1) / blk.y), blk, smem, h->stream, sa));
  time_end(h, 0, ev);
  time_begin(h, &ev);
  TEUK_CUDA(h, launch_dep(full_kernel<W, V>, dim3((nf + blk.y - 1) / blk.y), blk, smem, h->stream, sa));
  time_end(h, 1, ev);
  h->launches += 2;
  TEUK_CUDA(h, cudaGetLastError());
  return TEUK_OK;
}

int launch_pair(teuk_s* h, const StepArgs& sa, dim3 blk, size_t smem) {
  switch (h->kernel_variant) {
    case 1: return launch_pair_v<1>(h, sa, blk, smem);
    case 2: return launch_pair_v<2>(h, sa, blk, smem);
    default: return launch_pair_v<0>(h, sa, blk, smem);
  }
}

// One iteration in one launch (kernel family 4): from the buffer that holds the state into the
// other one (h->u2 is allocated with zero boundary rows, which no launch writes); the caller
// copies the state back into h->u when a sequence of iterations ends in h->u2.
int fused_impl(teuk_s* h, StepArgs sa) {
  if (!h->u2) {
    h->last_error = "fused iterations need the second state buffer (teuk_set_launch_shape variant 10)";
    return TEUK_ERR_INVALID_ARG;
  }
  sa.u_in = h->in_u2 ? h->u2 : h->u;
  sa.u_out = h->in_u2 ? h->u : h->u2;
  int tx, R;
  fused_shape(h, tx, R);
  const size_t smem = fused_smem(h, R);
  if (smem > 48 * 1024)
    TEUK_CUDA(h, cudaFuncSetAttribute(fused_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int G = (h->n_r - 2 + R - 1) / R;
  cudaEvent_t ev = nullptr;
  time_begin(h, &ev);
  TEUK_CUDA(h, launch_dep(fused_kernel<W>, dim3(G), dim3(tx, R + 1), smem, h->stream, sa));
  time_end(h, 1, ev);
  TEUK_CUDA(h, cudaGetLastError());
  h->in_u2 = !h->in_u2;
  h->launches += 1;
  return TEUK_OK;
}

int substep_impl(teuk_s* h, bool record, int64_t slot) {
  StepArgs sa{};
  sa.g = Geom{h->n_r, h->n_th, h->pitch, h->parity};
  sa.u_in = h->u;
  sa.u_out = h->u;
  sa.uh = h->uh;
  sa.cn = h->cn;
  sa.ch = h->ch;
  sa.wts = h->wts;
  std::memcpy(sa.h4, h->h4_w, sizeof(sa.h4));
  std::memcpy(sa.h2, h->h2_w, sizeof(sa.h2));
  sa.radius = h->radius;
  sa.record = record ? 1 : 0;
  sa.i_obs = h->i_obs;
  sa.ring_slot = slot;
  sa.ring_counter = h->d_ring_counter;
  sa.ring_cap = h->ring_cap;
  sa.ring = h->ring;
  sa.status = h->status;
  if (h->kernel_family == 4 && h->engine == 0) return fused_impl(h, sa);
  dim3 blk;
  step_shape(h, blk);
  const size_t smem = (size_t)blk.y * 2 * W * (h->n_th + 2 * h->radius) * sizeof(double);
  return launch_pair(h, sa, blk, smem);
}

// Persistent launch (kernel family 3, FP64 error-free transforms or FP64): n_outer outer steps
// of k iterations in one cooperative launch of ceil((n_r - 1) / R) blocks of
// (threads_theta, R) threads, R = h->rows_per_block; the observer ring gets one sample per
// outer step from slot ring_base on. TEUK_ERR_INVALID_ARG if the blocks cannot all be resident.
int persist_impl(teuk_s* h, int64_t n_outer, long long ring_base) {
  if (h->engine == 1) {
    h->last_error = "persistent launches run the FP64 and FP64-error-free-transform kernels only";
    return TEUK_ERR_INVALID_ARG;
  }
  const int R = h->rows_per_block > 0 ? h->rows_per_block : 1;
  int tx = ((h->n_th + 31) / 32) * 32;
  if (tx > 256 / R) tx = 256 / R;
  if (h->threads_theta > 0 && h->threads_theta < tx) tx = h->threads_theta;
  if (tx < 32 || tx * R > 256) {
    h->last_error = "persistent launch: threads_theta x rows must be 32..256";
    return TEUK_ERR_INVALID_ARG;
  }
  const int G = (h->n_r - 1 + R - 1) / R;
  const size_t smem = (size_t)R * 2 * W * (h->n_th + 2 * h->radius) * sizeof(double);
  if (smem > 48 * 1024)
    TEUK_CUDA(h, cudaFuncSetAttribute(persist_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0, sms = 0;
  TEUK_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persist_kernel<W>, tx * R, smem));
  TEUK_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  if (per_sm * sms < G) {
    h->last_error = "persistent launch: " + std::to_string(G) + " blocks cannot all be resident (" +
                    std::to_string(per_sm * sms) + " fit)";
    return TEUK_ERR_INVALID_ARG;
  }
  if ((int64_t)n_outer * h->k >= ((int64_t)1 << 31)) return TEUK_ERR_INVALID_ARG;
  if (h->pflags_cap < 2 * G + 1) {
    if (h->pflags) cudaFree(h->pflags);
    h->pflags = nullptr;
    h->pflags_cap = 0;
    TEUK_CUDA(h, cudaMalloc(&h->pflags, (size_t)(2 * G + 1) * sizeof(int)));
    h->pflags_cap = 2 * G + 1;
  }
  TEUK_CUDA(h, cudaMemsetAsync(h->pflags, 0, (size_t)(2 * G + 1) * sizeof(int), h->stream));
  PersistArgs pa{};
  StepArgs& sa = pa.a;
  sa.g = Geom{h->n_r, h->n_th, h->pitch, h->parity};
  sa.u_in = h->u;
  sa.u_out = h->u;
  sa.uh = h->uh;
  sa.cn = h->cn;
  sa.ch = h->ch;
  sa.wts = h->wts;
  std::memcpy(sa.h4, h->h4_w, sizeof(sa.h4));
  std::memcpy(sa.h2, h->h2_w, sizeof(sa.h2));
  sa.radius = h->radius;
  sa.record = 0;
  sa.i_obs = h->i_obs;
  sa.ring_slot = -1;
  sa.ring_counter = nullptr;
  sa.ring_cap = h->ring ? h->ring_cap : 0;
  sa.ring = h->ring;
  sa.status = h->status;
  pa.k = h->k;
  pa.n_outer = (int)n_outer;
  pa.ring_base = ring_base;
  pa.flags = h->pflags;
  pa.stall_block = h->test_stall_block;
  pa.spin_log2 = h->test_stall_block >= 0 ? h->wait_log2 : 22;
  void* params[] = {&pa};
  TEUK_CUDA(h, cudaLaunchCooperativeKernel((const void*)persist_kernel<W>, dim3(G), dim3(tx, R), params, smem,
                                           h->stream));
  h->launches += 1;
  return TEUK_OK;
}

// One Lax-Wendroff iteration from u_in to u_out (may alias) with the half-step rows in a
// caller-supplied scratch area; used by the no-allocation entry point (teuk_noalloc.cu).
int substep_buffers_impl(teuk_s* h, const double* u_in, double* u_out, double* scratch) {
  StepArgs sa{};
  sa.g = Geom{h->n_r, h->n_th, h->pitch, h->parity};
  sa.u_in = u_in;
  sa.u_out = u_out;
  sa.uh = scratch;
  sa.cn = h->cn;
  sa.ch = h->ch;
  sa.wts = h->wts;
  std::memcpy(sa.h4, h->h4_w, sizeof(sa.h4));
  std::memcpy(sa.h2, h->h2_w, sizeof(sa.h2));
  sa.radius = h->radius;
  sa.record = 0;
  sa.i_obs = -1;
  sa.ring_slot = 0;
  sa.ring_counter = nullptr;
  sa.ring_cap = 0;
  sa.ring = nullptr;
  sa.status = h->status;
  dim3 blk;
  step_shape(h, blk);
  const size_t smem = (size_t)blk.y * 2 * W * (h->n_th + 2 * h->radius) * sizeof(double);
  const bool timing = h->timing;
  h->timing = false;  // no events on this path
  const int rc = launch_pair(h, sa, blk, smem);
  h->timing = timing;
  return rc;
}

// ---- multi-word self test ---------------------------------------------------------------------
template <class RR>
__host__ __device__ RR apply_op(int op, RR x, RR y, RR acc, RR ln2) {
  switch (op) {
    case 0: return v_add(x, y);
    case 1: return v_sub(x, y);
    case 2: return r_mul(x, y);
    case 3: return r_div(x, y);
    case 4: return r_sqrt(x);
    case 5: return r_exp(x, ln2);
    case 6: return r_log(x, ln2);
    default: {
      Acc<RR> ac(acc);
      ac.mac(x, y);
      return ac.get();
    }
  }
}

// op 8: out[t] + sum_{q < 11} a[(t+q) % n] b[(t+q) % n] through one accumulator (the length
// of the theta stencil), without intermediate renormalisation.
__host__ __device__ R dot11(const double* a, const double* b, const double* out, int64_t n, int64_t t) {
  double wo[4] = {0, 0, 0, 0};
  for (int k = 0; k < W; ++k) wo[k] = out[k * n + t];
  Acc<R> acc(from_words<R>(wo));
  for (int q = 0; q < 11; ++q) {
    const int64_t u = (t + q) % n;
    double wa[4] = {0, 0, 0, 0}, wb[4] = {0, 0, 0, 0};
    for (int k = 0; k < W; ++k) { wa[k] = a[k * n + u]; wb[k] = b[k * n + u]; }
    acc.mac(from_words<R>(wa), from_words<R>(wb));
  }
  return acc.get();
}

// op 9 (double-double and quad-double): the same sum through the integer engine (ix.cuh,
// ixq.cuh): the 11 products and the initial value as terms of one fixed-point dot product,
// rounded once. ops 10 / 11: a + b / a - b through the engine's sum of two numbers, then rounded;
// op 12: a / 2 + b as two products by powers of two.
#if TEUK_WORDS != 1
__host__ __device__ R ix_dot11(const double* a, const double* b, const double* out, int64_t n, int64_t t) {
  using T = IxT<W>;
  uint32_t bad = 0;
  typename T::Num c[12], v[12];
  c[0] = ix_pow2<W>(0);
  v[0] = T::load(out + t, n, bad);
  for (int q = 0; q < 11; ++q) {
    const int64_t u = (t + q) % n;
    c[q + 1] = T::load(a + u, n, bad);
    v[q + 1] = T::load(b + u, n, bad);
  }
  int mx = 2 * ix::kZeroE;
  for (int q = 0; q < 12; ++q) mx = imax(mx, T::pexp(c[q].e, v[q].e));
  typename T::Acc acc;
  T::zero(acc);
  for (int q = 0; q < 12; ++q) T::prod(acc, c[q].m, v[q].m, c[q].neg ^ v[q].neg, T::pexp(c[q].e, v[q].e), mx);
  double w[4] = {0, 0, 0, 0};
  T::to_words(acc, T::base(mx), w);
  return from_words<R>(w);
}
__host__ __device__ R ix_addsub(int op, const double* a, const double* b, int64_t n, int64_t t) {
  using T = IxT<W>;
  uint32_t bad = 0;
  const typename T::Num one = ix_pow2<W>(0);
  if (op == 12) {  // a / 2 + b: both terms through the power-of-two products
    const typename T::Num half = ix_pow2<W>(-1), x = T::load(a + t, n, bad), y = T::load(b + t, n, bad);
    const int ex = T::pexp(half.e, x.e), ey = T::pexp(one.e, y.e), mx = ex > ey ? ex : ey;
    typename T::Acc acc;
    T::zero(acc);
    T::prod_pow2(acc, x.m, x.neg, ex, mx);
    T::prod_pow2(acc, y.m, y.neg, ey, mx);
    double w[4] = {0, 0, 0, 0};
    T::to_words(acc, T::base(mx), w);
    return from_words<R>(w);
  }
  const typename T::Num v = T::add(T::load(a + t, n, bad), T::load(b + t, n, bad), op == 11 ? 1u : 0u);
  const int mx = T::pexp(one.e, v.e);
  typename T::Acc acc;
  T::zero(acc);
  T::prod(acc, one.m, v.m, v.neg, mx, mx);
  double w[4] = {0, 0, 0, 0};
  T::to_words(acc, T::base(mx), w);
  return from_words<R>(w);
}
#else
__host__ __device__ R ix_dot11(const double*, const double*, const double*, int64_t, int64_t) { return 0.0; }
__host__ __device__ R ix_addsub(int, const double*, const double*, int64_t, int64_t) { return 0.0; }
#endif

__global__ void mw_eval_kernel(int op, const double* a, const double* b, double* out, double* res, int64_t n,
                               R ln2) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double wa[4] = {0, 0, 0, 0}, wb[4] = {0, 0, 0, 0}, wo[4] = {0, 0, 0, 0};
  if (op >= 8) {
    to_words(op == 8 ? dot11(a, b, out, n, t) : op == 9 ? ix_dot11(a, b, out, n, t) : ix_addsub(op, a, b, n, t), wo);
    for (int k = 0; k < W; ++k) res[k * n + t] = wo[k];
    return;
  }
  for (int k = 0; k < W; ++k) { wa[k] = a[k * n + t]; wb[k] = b[k * n + t]; wo[k] = out[k * n + t]; }
  const R r = apply_op<R>(op, from_words<R>(wa), from_words<R>(wb), from_words<R>(wo), ln2);
  to_words(r, wo);
  for (int k = 0; k < W; ++k) res[k * n + t] = wo[k];
}

int mw_eval_impl(int op, int device, const double* a, const double* b, double* out, int64_t n) {
  const R ln2 = r_ln2<R>();
  if (op >= 9 && W == 1) return TEUK_ERR_INVALID_ARG;
  if (!device && op >= 8) {
    std::vector<double> res((size_t)W * n);
    for (int64_t t = 0; t < n; ++t) {
      double wo[4];
      to_words(op == 8 ? dot11(a, b, out, n, t) : op == 9 ? ix_dot11(a, b, out, n, t) : ix_addsub(op, a, b, n, t),
               wo);
      for (int k = 0; k < W; ++k) res[k * n + t] = wo[k];
    }
    std::memcpy(out, res.data(), res.size() * sizeof(double));
    return TEUK_OK;
  }
  if (!device) {
    for (int64_t t = 0; t < n; ++t) {
      double wa[4] = {0, 0, 0, 0}, wb[4] = {0, 0, 0, 0}, wo[4] = {0, 0, 0, 0};
      for (int k = 0; k < W; ++k) { wa[k] = a[k * n + t]; wb[k] = b[k * n + t]; wo[k] = out[k * n + t]; }
      const R r = apply_op<R>(op, from_words<R>(wa), from_words<R>(wb), from_words<R>(wo), ln2);
      to_words(r, wo);
      for (int k = 0; k < W; ++k) out[k * n + t] = wo[k];
    }
    return TEUK_OK;
  }
  double *da = nullptr, *db = nullptr, *dout = nullptr, *dres = nullptr;
  const size_t bytes = (size_t)W * n * sizeof(double);
  TEUK_CUDA(nullptr, cudaMalloc(&da, bytes));
  TEUK_CUDA(nullptr, cudaMalloc(&db, bytes));
  TEUK_CUDA(nullptr, cudaMalloc(&dout, bytes));
  TEUK_CUDA(nullptr, cudaMalloc(&dres, bytes));
  cudaMemcpy(da, a, bytes, cudaMemcpyHostToDevice);
  cudaMemcpy(db, b, bytes, cudaMemcpyHostToDevice);
  cudaMemcpy(dout, out, bytes, cudaMemcpyHostToDevice);
  mw_eval_kernel<<<(unsigned)((n + 127) / 128), 128>>>(op, da, db, dout, dres, n, ln2);
  cudaError_t e = cudaMemcpy(out, dres, bytes, cudaMemcpyDeviceToHost);
  cudaFree(da);
  cudaFree(db);
  cudaFree(dout);
  cudaFree(dres);
  return e == cudaSuccess ? TEUK_OK : TEUK_ERR_CUDA;
}

}  // namespace prec_wN
using namespace TEUK_SUFFIX(prec_w);

int TEUK_SUFFIX(setup_w)(teuk_s* h) { return setup_impl(h); }
int TEUK_SUFFIX(pulse_w)(teuk_s* h, double center, double width, double ar, double ai, int ell) {
  return pulse_impl(h, center, width, ar, ai, ell);
}
int TEUK_SUFFIX(substep_w)(teuk_s* h, bool record, int64_t slot) { return substep_impl(h, record, slot); }
int TEUK_SUFFIX(prepare_w)(teuk_s* h) { return prepare_impl(h); }
int TEUK_SUFFIX(persist_w)(teuk_s* h, int64_t n_outer, long long ring_base) {
  return persist_impl(h, n_outer, ring_base);
}
int TEUK_SUFFIX(engine_w)(teuk_s* h, int engine) { return engine_impl(h, engine); }
int TEUK_SUFFIX(dissipation_w)(teuk_s* h, double sigma) { return dissipation_impl(h, sigma); }
int TEUK_SUFFIX(dissipate_w)(teuk_s* h) { return dissipate_impl(h); }
int TEUK_SUFFIX(filter_tables_w)(teuk_s* h, int l_cut) { return filter_tables_impl(h, l_cut); }
std::vector<double> TEUK_SUFFIX(harmonics_w)(int s, int m, int n_th, int ell_min, int ell_max, bool weighted) {
  return harmonic_table(s, m, n_th, ell_min, ell_max, weighted);
}
int TEUK_SUFFIX(theta_dissipation_w)(teuk_s* h, double sigma, double* max_rate) {
  return theta_dissipation_impl(h, sigma, max_rate);
}
int TEUK_SUFFIX(project_w)(teuk_s* h, int ell_min, int ell_max, double* out, int64_t n, int64_t first) {
  return project_impl(h, ell_min, ell_max, out, n, first);
}
int TEUK_SUFFIX(substep_buffers_w)(teuk_s* h, const double* u_in, double* u_out, double* scratch) {
  return substep_buffers_impl(h, u_in, u_out, scratch);
}
int TEUK_SUFFIX(mw_eval_w)(int op, int device, const double* a, const double* b, double* out, int64_t n) {
  return mw_eval_impl(op, device, a, b, out, n);
}

}  // namespace teuk
