// Double-double and quad-double step kernels on the integer engine (ix.cuh, ixq.cuh): the
// same two kernels per Lax-Wendroff iteration as teuk_kernels.cuh (Eqs. lw1, lw2 with the
// folded coefficient tables and the 10th/2nd-order theta stencil, Sec. 3.B-3.D), with every
// dot product formed in fixed point on the integer pipe (each product cut below 2^-122 (dd) /
// 2^-249 (qd) of itself, the sum of the terms exact) and rounded once to the handle's precision.
// The state and the half-step rows stay multi-word doubles in HBM; the coefficient tables are
// kept in the engine's format: the mantissa as 1 (dd) or 2 (qd) uint4 per value in planes of
// their own, the exponent and sign as one int (e * 2 + neg).
//
// The theta operator is evaluated in its factored form L = A2 D2 + (A1 cot theta) D1 with the
// integer stencils D2 = sum_q d2_q s_{j+q}, D1 = sum_q d1_q s_{j+q} (the weights of the
// 11-point stencil are A2 d2_q + A1 d1_q cot theta_j, d2 and d1 integers): each shared theta
// row is held in block-floating form (one exponent per row, every value a K-limb two's
// complement integer aligned to the row's largest), so D2 and D1 are exact integer
// multiply-adds, and the factors H5 A2, H5 A1 cot theta (N5 ... in the full step) are folded
// into the coefficient tables at set-up.
//
// A block's rows of the coefficient tables (and, where the footprint keeps as many blocks per
// SM resident, its state rows) are brought into shared memory by bulk asynchronous copies
// (cp.async.bulk completing on an mbarrier, issued by one thread at the start) while the block
// builds its theta rows; the wait for them is bounded and reports through the status word.
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
  static constexpr int kBlk = 6;                          // limbs of a block-floating row value
  static IXHD void shift_in(Acc& acc, const uint32_t* p, uint32_t neg, int r) { ix::acc_add(acc, p, neg, r); }
  static IXHD Num load(const double* p, size_t ws, uint32_t& bad) { return ix::from_dd(p[0], p[ws], bad); }
  static IXHD Num add(const Num& a, const Num& b, uint32_t nb) { return ix::add(a, b, nb); }
  static IXHD int pexp(int ec, int ev) { return ix::prod_exp(ec, ev); }
  static IXHD void zero(Acc& acc) { ix::acc_zero(acc); }
  static IXHD void prod(Acc& acc, const uint32_t* cm, const uint32_t* vm, uint32_t neg, int ep, int mx) {
    ix::acc_prod(acc, cm, vm, neg, ep, mx);
  }
  static IXHD void prod_pow2(Acc& acc, const uint32_t* vm, uint32_t neg, int ep, int mx) {
    ix::acc_prod_pow2(acc, vm, neg, ep, mx);
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
  static constexpr int kBlk = 10;
  static IXHD void shift_in(Acc& acc, const uint32_t* p, uint32_t neg, int r) { ix::acc_add10(acc, p, neg, r); }
  static IXHD Num load(const double* p, size_t ws, uint32_t& bad) {
    return ix::from_qd(p[0], p[ws], p[2 * ws], p[3 * ws], bad);
  }
  static IXHD Num add(const Num& a, const Num& b, uint32_t nb) { return ix::add8(a, b, nb); }
  static IXHD int pexp(int ec, int ev) { return ix::prod_exp8(ec, ev); }
  static IXHD void zero(Acc& acc) { ix::acc_zero10(acc); }
  static IXHD void prod(Acc& acc, const uint32_t* cm, const uint32_t* vm, uint32_t neg, int ep, int mx) {
    ix::acc_prod10(acc, cm, vm, neg, ep, mx);
  }
  static IXHD void prod_pow2(Acc& acc, const uint32_t* vm, uint32_t neg, int ep, int mx) {
    ix::acc_prod_pow2_10(acc, vm, neg, ep, mx);
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


// Asynchronous bulk copies global -> shared completing on an mbarrier (sm_90+ PTX).
IXD uint32_t ix_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
IXD void ix_bar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ix_saddr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
IXD void ix_bar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ix_saddr(bar)), "r"(bytes) : "memory");
}
// bytes: a multiple of 16; both addresses 16-byte aligned
IXD void ix_bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   ix_saddr(dst)),
               "l"(src), "r"(bytes), "r"(ix_saddr(bar))
               : "memory");
}
// Waits for phase 0 of bar with an iteration limit of 2^limit_log2 tries; false if the limit
// was reached.
IXD bool ix_bar_wait(uint64_t* bar, int limit_log2) {
  const int limit = 1 << limit_log2;
  for (int it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(ix_saddr(bar))
        : "memory");
    if (done) return true;
  }
  return false;
}

// Where a point reads its coefficients: plane q of value index ci at m[(q kU4 + u) pp + ci],
// e[q pp + ci] (the global tables, or the block's rows of them in shared memory).
struct IxTab {
  const uint4* m;
  const int* e;
  size_t pp;
};
// Where a point reads the state: q = Pi_R (component 2), word 0, at the lower of its two rows
// and the point's column (components W * qw apart, words qw, rows pitch); u (full step only)
// = component 0, word 0 of the state at the point's node (components W * uw apart). Global
// memory, or the block's copies of those rows in shared memory.
struct IxSt {
  const double* q;
  size_t qw;
  const double* u;
  size_t uw;
};

template <class N>
__host__ __device__ __forceinline__ int ix_en(const N& x) { return x.e * 2 + (int)x.neg; }

// Mantissa of value r of plane c in a [C][kU4][per_plane] uint4 array.
template <int W>
IXD void ix_ldm(const uint4* base, size_t per_plane, size_t c, size_t r, uint32_t* m) {
#pragma unroll
  for (int u = 0; u < IxT<W>::kU4; ++u) {
    const uint4 v = base[(c * IxT<W>::kU4 + u) * per_plane + r];  // global or shared
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

// Exact product x y of two engine values, cut to the engine's mantissa.
template <int W>
IXHD typename IxT<W>::Num ix_mul(const typename IxT<W>::Num& x, const typename IxT<W>::Num& y) {
  typename IxT<W>::Acc acc;
  IxT<W>::zero(acc);
  const int ep = IxT<W>::pexp(x.e, y.e);
  IxT<W>::prod(acc, x.m, y.m, x.neg ^ y.neg, ep, ep);
  return IxT<W>::to_num(acc, IxT<W>::base(ep));
}

// Folds the theta operator's factors into plane 5 of a converted table (set-up): plane 5
// becomes c5 A2 and plane 8 c5 A1 cot theta_j, for the values c5 of plane 5 at rows of
// `pitch` columns (lfac: [2][W][n_th] as A2, A1 cot theta_j; padding columns get zero).
template <int W>
__global__ void ix_fold_kernel(uint4* dm, int* de, size_t per_plane, int pitch, int n_th, const double* lfac) {
  using T = IxT<W>;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= per_plane) return;
  const int j = (int)(k % (size_t)pitch);
  typename T::Num p5 = T::zero_num(), p8 = T::zero_num();
  if (j < n_th) {
    typename T::Num c5;
#pragma unroll
    for (int u = 0; u < T::kU4; ++u) {
      const uint4 v = dm[(5 * T::kU4 + u) * per_plane + k];
      c5.m[4 * u] = v.x; c5.m[4 * u + 1] = v.y; c5.m[4 * u + 2] = v.z; c5.m[4 * u + 3] = v.w;
    }
    const int en = de[5 * per_plane + k];
    c5.e = en >> 1;
    c5.neg = (uint32_t)en & 1u;
    uint32_t bad = 0;
    p5 = ix_mul<W>(c5, T::load(lfac + j, n_th, bad));
    p8 = ix_mul<W>(c5, T::load(lfac + (size_t)W * n_th + j, n_th, bad));
  }
#pragma unroll
  for (int u = 0; u < T::kU4; ++u) {
    dm[(5 * T::kU4 + u) * per_plane + k] = make_uint4(p5.m[4 * u], p5.m[4 * u + 1], p5.m[4 * u + 2], p5.m[4 * u + 3]);
    dm[(8 * T::kU4 + u) * per_plane + k] = make_uint4(p8.m[4 * u], p8.m[4 * u + 1], p8.m[4 * u + 2], p8.m[4 * u + 3]);
  }
  de[5 * per_plane + k] = p5.e * 2 + (int)p5.neg;
  de[8 * per_plane + k] = p8.e * 2 + (int)p8.neg;
}

// K-limb two's-complement integers (mod 2^(32 K)): in-place sum, difference and multiply-add
// by a 32-bit constant, as carry chains.
template <int K> struct Kl;
template <> struct Kl<6> {
  static IXD void add_to(uint32_t* d, const uint32_t* b) {
    asm("add.cc.u32 %0, %0, %6;\n\t"
        "addc.cc.u32 %1, %1, %7;\n\t"
        "addc.cc.u32 %2, %2, %8;\n\t"
        "addc.cc.u32 %3, %3, %9;\n\t"
        "addc.cc.u32 %4, %4, %10;\n\t"
        "addc.u32 %5, %5, %11;"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3]), "+r"(d[4]), "+r"(d[5])
        : "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]));
  }
  static IXD void sub_from(uint32_t* d, const uint32_t* b) {
    asm("sub.cc.u32 %0, %0, %6;\n\t"
        "subc.cc.u32 %1, %1, %7;\n\t"
        "subc.cc.u32 %2, %2, %8;\n\t"
        "subc.cc.u32 %3, %3, %9;\n\t"
        "subc.cc.u32 %4, %4, %10;\n\t"
        "subc.u32 %5, %5, %11;"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3]), "+r"(d[4]), "+r"(d[5])
        : "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]));
  }
  static IXD void mac(uint32_t* d, uint32_t c, const uint32_t* p) {
    asm("mad.lo.cc.u32 %0, %6, %7, %0;\n\t"
        "madc.lo.cc.u32 %1, %6, %8, %1;\n\t"
        "madc.lo.cc.u32 %2, %6, %9, %2;\n\t"
        "madc.lo.cc.u32 %3, %6, %10, %3;\n\t"
        "madc.lo.cc.u32 %4, %6, %11, %4;\n\t"
        "madc.lo.u32 %5, %6, %12, %5;\n\t"
        "mad.hi.cc.u32 %1, %6, %7, %1;\n\t"
        "madc.hi.cc.u32 %2, %6, %8, %2;\n\t"
        "madc.hi.cc.u32 %3, %6, %9, %3;\n\t"
        "madc.hi.cc.u32 %4, %6, %10, %4;\n\t"
        "madc.hi.u32 %5, %6, %11, %5;"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3]), "+r"(d[4]), "+r"(d[5])
        : "r"(c), "r"(p[0]), "r"(p[1]), "r"(p[2]), "r"(p[3]), "r"(p[4]), "r"(p[5]));
  }
};
template <> struct Kl<10> {
  static IXD void add_to(uint32_t* d, const uint32_t* b) {
    asm("add.cc.u32 %0, %0, %10;\n\t"
        "addc.cc.u32 %1, %1, %11;\n\t"
        "addc.cc.u32 %2, %2, %12;\n\t"
        "addc.cc.u32 %3, %3, %13;\n\t"
        "addc.cc.u32 %4, %4, %14;\n\t"
        "addc.cc.u32 %5, %5, %15;\n\t"
        "addc.cc.u32 %6, %6, %16;\n\t"
        "addc.cc.u32 %7, %7, %17;\n\t"
        "addc.cc.u32 %8, %8, %18;\n\t"
        "addc.u32 %9, %9, %19;"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3]), "+r"(d[4]), "+r"(d[5]), "+r"(d[6]), "+r"(d[7]), "+r"(d[8]), "+r"(d[9])
        : "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]), "r"(b[9]));
  }
  static IXD void sub_from(uint32_t* d, const uint32_t* b) {
    asm("sub.cc.u32 %0, %0, %10;\n\t"
        "subc.cc.u32 %1, %1, %11;\n\t"
        "subc.cc.u32 %2, %2, %12;\n\t"
        "subc.cc.u32 %3, %3, %13;\n\t"
        "subc.cc.u32 %4, %4, %14;\n\t"
        "subc.cc.u32 %5, %5, %15;\n\t"
        "subc.cc.u32 %6, %6, %16;\n\t"
        "subc.cc.u32 %7, %7, %17;\n\t"
        "subc.cc.u32 %8, %8, %18;\n\t"
        "subc.u32 %9, %9, %19;"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3]), "+r"(d[4]), "+r"(d[5]), "+r"(d[6]), "+r"(d[7]), "+r"(d[8]), "+r"(d[9])
        : "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]), "r"(b[9]));
  }
  static IXD void mac(uint32_t* d, uint32_t c, const uint32_t* p) {
    asm("mad.lo.cc.u32 %0, %10, %11, %0;\n\t"
        "madc.lo.cc.u32 %1, %10, %12, %1;\n\t"
        "madc.lo.cc.u32 %2, %10, %13, %2;\n\t"
        "madc.lo.cc.u32 %3, %10, %14, %3;\n\t"
        "madc.lo.cc.u32 %4, %10, %15, %4;\n\t"
        "madc.lo.cc.u32 %5, %10, %16, %5;\n\t"
        "madc.lo.cc.u32 %6, %10, %17, %6;\n\t"
        "madc.lo.cc.u32 %7, %10, %18, %7;\n\t"
        "madc.lo.cc.u32 %8, %10, %19, %8;\n\t"
        "madc.lo.u32 %9, %10, %20, %9;\n\t"
        "mad.hi.cc.u32 %1, %10, %11, %1;\n\t"
        "madc.hi.cc.u32 %2, %10, %12, %2;\n\t"
        "madc.hi.cc.u32 %3, %10, %13, %3;\n\t"
        "madc.hi.cc.u32 %4, %10, %14, %4;\n\t"
        "madc.hi.cc.u32 %5, %10, %15, %5;\n\t"
        "madc.hi.cc.u32 %6, %10, %16, %6;\n\t"
        "madc.hi.cc.u32 %7, %10, %17, %7;\n\t"
        "madc.hi.cc.u32 %8, %10, %18, %8;\n\t"
        "madc.hi.u32 %9, %10, %19, %9;"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3]), "+r"(d[4]), "+r"(d[5]), "+r"(d[6]), "+r"(d[7]), "+r"(d[8]), "+r"(d[9])
        : "r"(c), "r"(p[0]), "r"(p[1]), "r"(p[2]), "r"(p[3]), "r"(p[4]), "r"(p[5]), "r"(p[6]), "r"(p[7]), "r"(p[8]), "r"(p[9]));
  }
};

// Shared row of one component: the values as engine numbers (mantissas [kU4][gstride] uint4,
// exponent-sign words [gstride] int; only the row's own columns are read), and the ghosted
// block-floating row (b: [kBlk / 2][gstride] uint2, value = b * 2^(E - 32)).
struct IxRow {
  uint4* m;
  int* e;
  uint2* b;
  int E;     // largest exponent of the row (kZeroE for a row of zeros)
  uint4* dm; // the differences of the same two rows (Phi_{h+1} - Phi_h), engine numbers at the
  int* de;   //   row's own columns; exponent word kIxBadEn where an operand was Inf / NaN
};
constexpr int kIxBadEn = (int)0x80000000;  // never an exponent-sign word (those are >= -2^25)
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
// Difference at column idx; sets bad where the prep phase met a non-finite operand.
template <int W>
IXD typename IxT<W>::Num ix_diff_get(const IxRow& row, int gstride, int idx, uint32_t& bad) {
  const int en = row.de[idx];
  if (en == kIxBadEn) {
    bad = 1;
    return IxT<W>::zero_num();
  }
  typename IxT<W>::Num r;
#pragma unroll
  for (int u = 0; u < IxT<W>::kU4; ++u) {
    const uint4 v = row.dm[u * gstride + idx];
    r.m[4 * u] = v.x; r.m[4 * u + 1] = v.y; r.m[4 * u + 2] = v.z; r.m[4 * u + 3] = v.w;
  }
  r.e = en >> 1;
  r.neg = (uint32_t)en & 1u;
  return r;
}
template <int W>
IXD void ix_diff_put(const IxRow& row, int gstride, int idx, const typename IxT<W>::Num& v, uint32_t bad) {
#pragma unroll
  for (int u = 0; u < IxT<W>::kU4; ++u)
    row.dm[u * gstride + idx] = make_uint4(v.m[4 * u], v.m[4 * u + 1], v.m[4 * u + 2], v.m[4 * u + 3]);
  row.de[idx] = bad ? kIxBadEn : v.e * 2 + (int)v.neg;
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
// One term c v with c = 2^k made by ix_pow2 (no multiply: a shift of v's mantissa).
template <int W>
IXD void ix_p2term(typename IxT<W>::Acc& acc, const typename IxT<W>::Num& c, const typename IxT<W>::Num& v,
                   uint32_t flip, int mx) {
  IxT<W>::prod_pow2(acc, v.m, c.neg ^ v.neg ^ flip, IxT<W>::pexp(c.e, v.e), mx);
}

template <int W>
IXD void ix_store(double* p, size_t ws, const typename IxT<W>::Acc& acc, int B, uint32_t bad, double* w) {
  IxT<W>::to_words(acc, B, w);
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
  for (int k = 0; k < W; ++k) p[k * ws] = bad ? nan : w[k];
}

// v as a block-floating value of a row of largest exponent E, sign flipped if flip:
// (-1)^neg (m 2^32) >> (E - e) in kBlk limbs (bits below the last are cut).
template <int W>
IXD void ix_to_block(const typename IxT<W>::Num& v, int E, uint32_t flip, uint32_t* out) {
  using T = IxT<W>;
  uint32_t p[T::kLimbs + 1];
#pragma unroll
  for (int k = 0; k < T::kLimbs; ++k) p[k] = v.m[k];
  p[T::kLimbs] = 0;
  typename T::Acc acc;
  T::zero(acc);
  T::shift_in(acc, p, v.neg ^ flip, E - v.e);
#pragma unroll
  for (int k = 0; k < T::kBlk; ++k) out[k] = acc.a[k];
}
template <int W>
IXD void ix_block_put(const IxRow& row, int gstride, int idx, const uint32_t* s) {
#pragma unroll
  for (int u = 0; u < IxT<W>::kBlk / 2; ++u) row.b[u * gstride + idx] = make_uint2(s[2 * u], s[2 * u + 1]);
}
template <int W>
IXD void ix_block_get(const IxRow& row, int gstride, int idx, uint32_t* s) {
#pragma unroll
  for (int u = 0; u < IxT<W>::kBlk / 2; ++u) {
    const uint2 v = row.b[u * gstride + idx];
    s[2 * u] = v.x;
    s[2 * u + 1] = v.y;
  }
}

// Second phase of a row's set-up: the largest exponent of each component's row from the
// per-warp maxima, then the thread's columns (and their parity images across the poles) into
// the block-floating rows.
template <int W>
IXD void ix_block_rows(const IxArgs& x, int tx, int TX, IxRow& sR, IxRow& sI, int gstride, const int* wmax) {
  const StepArgs& a = x.a;
  const int n_th = a.g.n_th, rad = a.radius, nw = (TX + 31) / 32;
  int ER = ix::kZeroE, EI = ix::kZeroE;
  for (int w = 0; w < nw; ++w) {
    ER = imax(ER, wmax[w]);
    EI = imax(EI, wmax[8 + w]);
  }
  sR.E = ER;
  sI.E = EI;
  const uint32_t pflip = a.g.parity > 0 ? 0u : 1u;
  for (int j = tx; j < n_th; j += TX) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const IxRow& row = c == 0 ? sR : sI;
      const typename IxT<W>::Num v = ix_row_get<W>(row, gstride, j + rad);
      uint32_t b[IxT<W>::kBlk];
      ix_to_block<W>(v, row.E, 0u, b);
      ix_block_put<W>(row, gstride, j + rad, b);
      if (j < rad || j >= n_th - rad) {  // (a narrow row can need both images)
        ix_to_block<W>(v, row.E, pflip, b);
        if (j < rad) ix_block_put<W>(row, gstride, rad - 1 - j, b);
        if (j >= n_th - rad) ix_block_put<W>(row, gstride, 2 * n_th - 1 - j + rad, b);
      }
    }
  }
}

// Integer stencils of the theta operator at column j of a block-floating row: D2 = sum_q
// d2_q s_{j+q}, D1 = sum_q d1_q s_{j+q} (10th order: d2 / 25200, d1 / 2520; 2nd order:
// {1, -2, 1}, {-1, 0, 1} / 2; Sec. 3.B, 3.D), exact, returned as engine numbers. The
// symmetric d2 and antisymmetric d1 take the sums and differences of the pairs j +- q.
template <int W, int RAD>
IXD void ix_stencil(const IxRow& row, int gstride, int j, typename IxT<W>::Num& D2, typename IxT<W>::Num& D1) {
  using T = IxT<W>;
  using L = Kl<T::kBlk>;
  constexpr int K = T::kBlk;
  // d2_0 .. d2_RAD and d1_1 .. d1_RAD
  constexpr int d2[6] = {RAD == 5 ? -73766 : -2, RAD == 5 ? 42000 : 1, -6000, 1000, -125, 8};
  constexpr int d1[6] = {0, RAD == 5 ? 2100 : 1, -600, 150, -25, 2};
  uint32_t pos[K], neg[K], dd1[K], s0[K];
#pragma unroll
  for (int k = 0; k < K; ++k) pos[k] = neg[k] = dd1[k] = 0;
  ix_block_get<W>(row, gstride, j + RAD, s0);
  L::mac(neg, (uint32_t)(-d2[0]), s0);
#pragma unroll
  for (int q = 1; q <= RAD; ++q) {
    uint32_t sp[K], sm[K], t[K];
    ix_block_get<W>(row, gstride, j + RAD + q, sp);
    ix_block_get<W>(row, gstride, j + RAD - q, sm);
#pragma unroll
    for (int k = 0; k < K; ++k) t[k] = sp[k];
    L::add_to(t, sm);
    if (d2[q] > 0) L::mac(pos, (uint32_t)d2[q], t);
    else L::mac(neg, (uint32_t)(-d2[q]), t);
    if (d1[q] > 0) {
      L::sub_from(sp, sm);
      L::mac(dd1, (uint32_t)d1[q], sp);
    } else {
      L::sub_from(sm, sp);
      L::mac(dd1, (uint32_t)(-d1[q]), sm);
    }
  }
  L::sub_from(pos, neg);
  typename T::Acc acc;
#pragma unroll
  for (int k = 0; k < K; ++k) acc.a[k] = pos[k];
  D2 = T::to_num(acc, row.E - 32);
#pragma unroll
  for (int k = 0; k < K; ++k) acc.a[k] = dd1[k];
  D1 = T::to_num(acc, row.E - 32);
}
template <int W>
IXD void ix_stencil(const IxArgs& x, const IxRow& row, int gstride, int j, typename IxT<W>::Num& D2,
                    typename IxT<W>::Num& D1) {
  if (x.a.radius == 5) ix_stencil<W, 5>(row, gstride, j, D2, D1);
  else ix_stencil<W, 1>(row, gstride, j, D2, D1);
}

// Eq. lw1, first phase: s_Phi = Phi_{h+1} + Phi_h of row h into the ghosted rows.
// (the values as engine numbers at their own columns; eR, eI: the thread's largest exponents)
template <int W>
IXD void ix_half_prep(const IxArgs& x, int h, int tx, int TX, const IxRow& sR, const IxRow& sI, int gstride,
                      int& eR, int& eI) {
  const StepArgs& a = x.a;
  const size_t ws = (size_t)a.g.n_r * a.g.pitch;
  for (int j = tx; j < a.g.n_th; j += TX) {
    const size_t i0 = (size_t)h * a.g.pitch + j, i1 = i0 + a.g.pitch;
    uint32_t bad = 0;
    const auto r1 = IxT<W>::load(a.u_in + i1, ws, bad), r0 = IxT<W>::load(a.u_in + i0, ws, bad);
    const auto q1 = IxT<W>::load(a.u_in + W * ws + i1, ws, bad), q0 = IxT<W>::load(a.u_in + W * ws + i0, ws, bad);
    const auto vR = IxT<W>::add(r1, r0, 0u), vI = IxT<W>::add(q1, q0, 0u);
    ix_row_put<W>(sR, gstride, j + a.radius, vR, ix_en(vR));
    ix_row_put<W>(sI, gstride, j + a.radius, vI, ix_en(vI));
    ix_diff_put<W>(sR, gstride, j + a.radius, IxT<W>::add(r1, r0, 1u), bad);
    ix_diff_put<W>(sI, gstride, j + a.radius, IxT<W>::add(q1, q0, 1u), bad);
    eR = imax(eR, vR.e);
    eI = imax(eI, vI.e);
  }
}

// End of a row's first phase: each warp's largest exponents of the two rows into wmax
// ([2][8] per row of the block; the warps of a row never straddle rows).
IXD void ix_warp_max(int eR, int eI, int tx, int* wmax, bool write = true) {
  eR = __reduce_max_sync(0xffffffffu, eR);
  eI = __reduce_max_sync(0xffffffffu, eI);
  if (write && (tx & 31) == 0) {
    wmax[tx >> 5] = eR;
    wmax[8 + (tx >> 5)] = eI;
  }
}

// Eq. lw1 at half node h, column j (same terms as half_point in teuk_kernels.cuh).
// The two components share one loop body (own = this component, other = the other one; the
// signs of the cross terms follow the component): unrolled for double-double, kept as a loop
// for quad-double, whose unrolled kernels outgrow the instruction caches.
template <int W>
struct IxUnroll {
  static constexpr int n = W == 4 ? 1 : 2;
};

template <int W>
IXD void ix_half_point(const IxArgs& x, int h, int j, const IxRow& sR, const IxRow& sI, int gstride,
                       const typename IxT<W>::Num& half, const typename IxT<W>::Num& h4, const IxTab& tb,
                       size_t ci, const IxSt& st) {
  using T = IxT<W>;
  using Num = typename T::Num;
  const StepArgs& a = x.a;
  const int pitch = a.g.pitch, rad = a.radius;
  const size_t hs = (size_t)(a.g.n_r - 1) * pitch;
  uint32_t bad = 0;
  const Num uQR0 = T::load(st.q, st.qw, bad), uQR1 = T::load(st.q + pitch, st.qw, bad);
  const Num uQI0 = T::load(st.q + W * st.qw, st.qw, bad), uQI1 = T::load(st.q + W * st.qw + pitch, st.qw, bad);
  // Phi_{h+1} - Phi_h from the prep phase
  const Num dPR = ix_diff_get<W>(sR, gstride, j + rad, bad), dPI = ix_diff_get<W>(sI, gstride, j + rad, bad);
  const Num sQR = T::add(uQR1, uQR0, 0u), sQI = T::add(uQI1, uQI0, 0u);
  // one exact difference and one product are cheaper here than two products
  const Num dQR = T::add(uQR1, uQR0, 1u), dQI = T::add(uQI1, uQI0, 1u);
  const Num sPR = ix_row_get<W>(sR, gstride, j + rad), sPI = ix_row_get<W>(sI, gstride, j + rad);
  const size_t oi = (size_t)h * pitch + j;  // output index
  int ce[kIxPlanes];
#pragma unroll
  for (int q = 0; q < kIxPlanes; ++q) ce[q] = tb.e[q * tb.pp + ci];
#define TT(q, v, f) ix_tterm<W>(acc, tb.m, tb.pp, q, ci, ce[q], v, f, mx)
#define TE(q, v) ix_texp<W>(ce[q], v)
#pragma unroll(IxUnroll<W>::n)
  for (int c = 0; c < 2; ++c) {
    const bool im = c != 0;
    const uint32_t fc = (uint32_t)c;
    Num D2, D1;
    ix_stencil<W>(x, im ? sI : sR, gstride, j, D2, D1);
    const Num sPo = im ? sPI : sPR, sPx = im ? sPR : sPI, dPo = im ? dPI : dPR, dPx = im ? dPR : dPI;
    const Num sQo = im ? sQI : sQR, sQx = im ? sQR : sQI, dQo = im ? dQI : dQR;
    typename T::Acc acc;
    int mx;
    double w[4];
    // Phi_c = s_Phi_c/2 - H0 d_Phi_c + (h/4) s_Pi_c
    mx = imax(imax(T::pexp(half.e, sPo.e), TE(0, dPo)), T::pexp(h4.e, sQo.e));
    T::zero(acc);
    ix_p2term<W>(acc, half, sPo, 0u, mx);
    TT(0, dPo, 1u);
    ix_nterm<W>(acc, h4, sQo, 0u, mx);
    ix_store<W>(a.uh + c * W * hs + oi, hs, acc, T::base(mx), bad, w);
    // Pi_R = H3 s_PiR + H4 s_PiI + H0 (Pi_R,h+1 - Pi_R,h) + H1 d_PhiR + H2 d_PhiI + H5 L_R + H6 s_PhiR - H7 s_PhiI
    // Pi_I = H3 s_PiI - H4 s_PiR + H0 (Pi_I,h+1 - Pi_I,h) + H1 d_PhiI - H2 d_PhiR + H5 L_I + H6 s_PhiI + H7 s_PhiR
    // with H5 L = (H5 A2) D2 + (H5 A1 cot) D1 (planes 5 and 8)
    mx = imax(imax(imax(TE(3, sQo), TE(4, sQx)), imax(TE(0, dQo), TE(8, D1))),
              imax(imax(TE(1, dPo), TE(2, dPx)), imax(TE(5, D2), imax(TE(6, sPo), TE(7, sPx)))));
    T::zero(acc);
    TT(3, sQo, 0u); TT(4, sQx, fc); TT(0, dQo, 0u); TT(1, dPo, 0u);
    TT(2, dPx, fc); TT(5, D2, 0u); TT(8, D1, 0u); TT(6, sPo, 0u); TT(7, sPx, 1u - fc);
    ix_store<W>(a.uh + (2 + c) * W * hs + oi, hs, acc, T::base(mx), bad, w);
  }
#undef TT
#undef TE
}

// Eq. lw2, first phase: s_Phi = Phi_{i+1/2} + Phi_{i-1/2} into the ghosted rows.
template <int W>
IXD void ix_full_prep(const IxArgs& x, int i, int tx, int TX, const IxRow& sR, const IxRow& sI, int gstride,
                      int& eR, int& eI) {
  const StepArgs& a = x.a;
  const size_t hs = (size_t)(a.g.n_r - 1) * a.g.pitch;
  for (int j = tx; j < a.g.n_th; j += TX) {
    const size_t p = (size_t)i * a.g.pitch + j, m = p - a.g.pitch;
    uint32_t bad = 0;
    const auto r1 = IxT<W>::load(a.uh + p, hs, bad), r0 = IxT<W>::load(a.uh + m, hs, bad);
    const auto q1 = IxT<W>::load(a.uh + W * hs + p, hs, bad), q0 = IxT<W>::load(a.uh + W * hs + m, hs, bad);
    const auto vR = IxT<W>::add(r1, r0, 0u), vI = IxT<W>::add(q1, q0, 0u);
    ix_row_put<W>(sR, gstride, j + a.radius, vR, ix_en(vR));
    ix_row_put<W>(sI, gstride, j + a.radius, vI, ix_en(vI));
    ix_diff_put<W>(sR, gstride, j + a.radius, IxT<W>::add(r1, r0, 1u), bad);
    ix_diff_put<W>(sI, gstride, j + a.radius, IxT<W>::add(q1, q0, 1u), bad);
    eR = imax(eR, vR.e);
    eI = imax(eI, vI.e);
  }
}

// Eq. lw2 at node i, column j (same terms as full_point); returns true for a non-finite value.
template <int W>
IXD bool ix_full_point(const IxArgs& x, int i, int j, const IxRow& sR, const IxRow& sI, int gstride,
                       const typename IxT<W>::Num& one, const typename IxT<W>::Num& h2, long long slot,
                       const IxTab& tb, size_t cti, const IxSt& st) {
  using T = IxT<W>;
  using Num = typename T::Num;
  const StepArgs& a = x.a;
  const int pitch = a.g.pitch, rad = a.radius, n_th = a.g.n_th;
  const size_t ws = (size_t)a.g.n_r * pitch;
  uint32_t bad = 0;
  // half-step Pi rows i - 1/2 (q) and i + 1/2 (q + pitch)
  const Num hQR0 = T::load(st.q, st.qw, bad), hQR1 = T::load(st.q + pitch, st.qw, bad);
  const Num hQI0 = T::load(st.q + W * st.qw, st.qw, bad), hQI1 = T::load(st.q + W * st.qw + pitch, st.qw, bad);
  // h_Phi,i+1/2 - h_Phi,i-1/2 from the prep phase
  const Num dPR = ix_diff_get<W>(sR, gstride, j + rad, bad), dPI = ix_diff_get<W>(sI, gstride, j + rad, bad);
  const Num sQR = T::add(hQR1, hQR0, 0u), sQI = T::add(hQI1, hQI0, 0u);
  const Num dQR = T::add(hQR1, hQR0, 1u), dQI = T::add(hQI1, hQI0, 1u);
  const Num sPR = ix_row_get<W>(sR, gstride, j + rad), sPI = ix_row_get<W>(sI, gstride, j + rad);
  const size_t ci = (size_t)i * pitch + j;
  const Num PR = T::load(st.u, st.uw, bad), PI = T::load(st.u + W * st.uw, st.uw, bad);
  const Num QR = T::load(st.u + 2 * W * st.uw, st.uw, bad), QI = T::load(st.u + 3 * W * st.uw, st.uw, bad);
  int ce[kIxPlanes];
#pragma unroll
  for (int q = 0; q < kIxPlanes; ++q) ce[q] = tb.e[q * tb.pp + cti];
#define TT(q, v, f) ix_tterm<W>(acc, tb.m, tb.pp, q, cti, ce[q], v, f, mx)
#define TE(q, v) ix_texp<W>(ce[q], v)
  bool nf = false;
#pragma unroll(IxUnroll<W>::n)
  for (int c = 0; c < 2; ++c) {
    const bool im = c != 0;
    const uint32_t fc = (uint32_t)c;
    Num D2, D1;
    ix_stencil<W>(x, im ? sI : sR, gstride, j, D2, D1);
    const Num sPo = im ? sPI : sPR, sPx = im ? sPR : sPI, dPo = im ? dPI : dPR, dPx = im ? dPR : dPI;
    const Num sQo = im ? sQI : sQR, sQx = im ? sQR : sQI, dQo = im ? dQI : dQR;
    const Num Po = im ? PI : PR, Qo = im ? QI : QR;
    typename T::Acc acc;
    int mx;
    double o[4], w[4];
    // Phi_c' = Phi_c - N0 d_Phi_c + (h/2) s_Pi_c
    mx = imax(imax(T::pexp(one.e, Po.e), TE(0, dPo)), T::pexp(h2.e, sQo.e));
    T::zero(acc);
    ix_p2term<W>(acc, one, Po, 0u, mx);
    TT(0, dPo, 1u);
    ix_nterm<W>(acc, h2, sQo, 0u, mx);
    ix_store<W>(a.u_out + c * W * ws + ci, ws, acc, T::base(mx), bad, o);
    if (slot >= 0 && i == a.i_obs && !bad) {  // the observer's sample of Phi_c
      double* dst = a.ring + (size_t)slot * 2 * W * n_th;
#pragma unroll
      for (int k = 0; k < W; ++k) dst[(c * W + k) * n_th + j] = o[k];
    }
    // Pi_R' = Pi_R + N0 (h_PiR,i+1/2 - h_PiR,i-1/2) + N1 d_PhiR + N2 d_PhiI + N3 s_PiR + N4 s_PiI + N5 L_R
    //         + N6 s_PhiR - N7 s_PhiI
    // Pi_I' = Pi_I + N0 (h_PiI,i+1/2 - h_PiI,i-1/2) + N1 d_PhiI - N2 d_PhiR + N3 s_PiI - N4 s_PiR + N5 L_I
    //         + N6 s_PhiI + N7 s_PhiR, with N5 L = (N5 A2) D2 + (N5 A1 cot) D1 (planes 5 and 8)
    mx = imax(imax(imax(T::pexp(one.e, Qo.e), TE(8, D1)), imax(TE(0, dQo), TE(1, dPo))),
              imax(imax(TE(2, dPx), TE(3, sQo)), imax(imax(TE(4, sQx), TE(5, D2)), imax(TE(6, sPo), TE(7, sPx)))));
    T::zero(acc);
    ix_p2term<W>(acc, one, Qo, 0u, mx);
    TT(0, dQo, 0u); TT(1, dPo, 0u); TT(2, dPx, fc); TT(3, sQo, 0u);
    TT(4, sQx, fc); TT(5, D2, 0u); TT(8, D1, 0u); TT(6, sPo, 0u); TT(7, sPx, 1u - fc);
    ix_store<W>(a.u_out + (2 + c) * W * ws + ci, ws, acc, T::base(mx), bad, w);
    nf = nf || nonfinite(o[0]) || nonfinite(w[0]);
  }
#undef TT
#undef TE
  return bad || nf;
}

// Shared memory of the engine kernels, for blockDim.y rows: with staging, the block's rows of
// the coefficient tables first (mantissas [kIxPlanes][kU4][rows][pitch] uint4, exponent-sign
// words [kIxPlanes][rows][pitch] int); then the value mantissas [rows][2][kU4][gstride]
// (uint4), the difference mantissas (same shape), the values' and the differences'
// exponent-sign words [rows][2][gstride] (int) each, the block-floating rows
// [rows][2][kBlk / 2][gstride] (uint2), the per-warp exponent maxima [rows][16] (int) and the
// copies' mbarrier.
struct IxSmem {
  uint4* tm;
  int* te;
  double* st;  // staged state rows (stage bit 2)
  int* wmax;
  uint64_t* bar;
};
// Doubles of staged state rows for `rows` rows: the half step's Pi rows h0 .. h0 + rows
// ([2][W][rows + 1][pitch]); the full step's half-step Pi rows i0 - 1 .. i0 + rows - 1 (same
// shape) and its state rows i0 .. i0 + rows - 1 ([4][W][rows][pitch]).
template <int W>
IXHD size_t ix_state_doubles(int rows, int pitch, bool full) {
  return (size_t)2 * W * (rows + 1) * pitch + (full ? (size_t)4 * W * rows * pitch : 0);
}
template <int W>
IXD IxSmem ix_rows(int gstride, int pitch, int stage, IxRow& sR, IxRow& sI, int rows, int y, bool full) {
  extern __shared__ uint4 ixsm[];
  constexpr int U = IxT<W>::kU4, KB = IxT<W>::kBlk / 2;
  IxSmem sm;
  sm.tm = ixsm;
  sm.te = reinterpret_cast<int*>(ixsm + (size_t)kIxPlanes * U * rows * pitch);
  sm.st = reinterpret_cast<double*>(sm.te + (size_t)kIxPlanes * rows * pitch);
  uint4* rbase = (stage & 2) ? reinterpret_cast<uint4*>(sm.st + ix_state_doubles<W>(rows, pitch, full))
                 : (stage & 1) ? reinterpret_cast<uint4*>(sm.st)
                               : ixsm;
  // values, then differences: mantissas, then exponent-sign words
  int* ebase = reinterpret_cast<int*>(rbase + (size_t)rows * 2 * U * gstride * 2);
  uint2* bbase = reinterpret_cast<uint2*>(ebase + (size_t)rows * 2 * gstride * 2);
  int* mbase = reinterpret_cast<int*>(bbase + (size_t)rows * 2 * KB * gstride);
  sR.m = rbase + (size_t)y * 2 * U * gstride;
  sI.m = sR.m + (size_t)U * gstride;
  sR.e = ebase + (size_t)y * 2 * gstride;
  sI.e = sR.e + gstride;
  sR.dm = rbase + (size_t)rows * 2 * U * gstride + (size_t)y * 2 * U * gstride;
  sI.dm = sR.dm + (size_t)U * gstride;
  sR.de = ebase + (size_t)rows * 2 * gstride + (size_t)y * 2 * gstride;
  sI.de = sR.de + gstride;
  sR.b = bbase + (size_t)y * 2 * KB * gstride;
  sI.b = sR.b + (size_t)KB * gstride;
  sR.E = sI.E = ix::kZeroE;
  sm.wmax = mbase + 16 * y;
  sm.bar = reinterpret_cast<uint64_t*>(mbase + 16 * rows);
  return sm;
}
// Bytes of shared memory for `rows` rows of gstride columns (stage bit 1: with the table
// rows; bit 2: also the state rows, which only go with the table rows).
template <int W>
inline size_t ix_smem_bytes(int rows, int gstride, int pitch, int stage, bool full) {
  const size_t tab = stage ? (size_t)kIxPlanes * rows * pitch * (IxT<W>::kU4 * sizeof(uint4) + sizeof(int)) : 0;
  const size_t sta = (stage & 2) ? ix_state_doubles<W>(rows, pitch, full) * sizeof(double) : 0;
  return tab + sta +
         (size_t)rows * 2 * gstride *
             (2 * (IxT<W>::kU4 * sizeof(uint4) + sizeof(int)) + IxT<W>::kBlk * sizeof(uint32_t)) +
         (size_t)rows * 16 * sizeof(int) + sizeof(uint64_t);
}

// One thread of the block starts the copies of the block's table rows r0 .. r0 + nv - 1
// (planes of per_plane values at row pitch `pitch`; 16-byte aligned since pitch is a multiple
// of 16) into shared memory.
// With stage bit 2 also the state rows: Pi rows q0 .. q0 + nv of qsrc (planes qs doubles
// apart) into [2][W][rows + 1][pitch], and (full step, usrc != null) rows r0 .. r0 + nv - 1
// of all four components of usrc (planes us apart) into [4][W][rows][pitch] after them.
// stall: this block arms the barrier with the expected byte count and issues no copy (a test
// of the bounded wait's give-up path: nothing is in flight when the block gives up).
template <int W>
IXD void ix_stage(const IxSmem& sm, int stage, const uint4* gm, const int* ge, size_t per_plane, int pitch, int r0,
                  int nv, const double* qsrc, size_t qs, int q0, const double* usrc, size_t us, bool stall) {
  constexpr int U = IxT<W>::kU4;
  const int rows = blockDim.y;
  const uint32_t mb = (uint32_t)nv * pitch * sizeof(uint4), eb = (uint32_t)nv * pitch * sizeof(int);
  const uint32_t qb = (uint32_t)(nv + 1) * pitch * sizeof(double), ub = (uint32_t)nv * pitch * sizeof(double);
  uint32_t bytes = kIxPlanes * (U * mb + eb);
  if (stage & 2) bytes += 2 * W * qb + (usrc ? 4 * W * ub : 0);
  ix_bar_init(sm.bar);
  ix_bar_expect(sm.bar, bytes);
  if (stall) return;
  for (int q = 0; q < kIxPlanes; ++q) {
    for (int u = 0; u < U; ++u)
      ix_bulk_copy(sm.tm + ((size_t)(q * U + u) * rows) * pitch, gm + (q * U + u) * per_plane + (size_t)r0 * pitch,
                   mb, sm.bar);
    ix_bulk_copy(sm.te + (size_t)q * rows * pitch, ge + q * per_plane + (size_t)r0 * pitch, eb, sm.bar);
  }
  if (!(stage & 2)) return;
  for (int k = 0; k < 2 * W; ++k)  // components 2, 3: planes 2 W .. 4 W - 1
    ix_bulk_copy(sm.st + (size_t)k * (rows + 1) * pitch, qsrc + (size_t)(2 * W + k) * qs + (size_t)q0 * pitch, qb,
                 sm.bar);
  if (!usrc) return;
  double* ud = sm.st + (size_t)2 * W * (rows + 1) * pitch;
  for (int k = 0; k < 4 * W; ++k)
    ix_bulk_copy(ud + (size_t)k * rows * pitch, usrc + (size_t)k * us + (size_t)r0 * pitch, ub, sm.bar);
}

template <int W, int V>
__global__ void __launch_bounds__(RowBounds<V>::threads, RowBounds<V>::blocks) half_ix_kernel(IxArgs x) {
  const int gstride = x.a.g.n_th + 2 * x.a.radius, pitch = x.a.g.pitch, nh = x.a.g.n_r - 1;
  const size_t hs = (size_t)nh * pitch, ws = (size_t)x.a.g.n_r * pitch;
  IxRow sR, sI;
  const IxSmem sm = ix_rows<W>(gstride, pitch, x.stage, sR, sI, blockDim.y, threadIdx.y, false);
  const int h0 = blockIdx.x * blockDim.y, h = h0 + threadIdx.y;
  if (x.stage && threadIdx.x == 0 && threadIdx.y == 0)
    ix_stage<W>(sm, x.stage, x.chm, x.che, hs, pitch, h0, min((int)blockDim.y, nh - h0), x.a.u_in, ws, h0, nullptr,
                0, (int)blockIdx.x == x.stall_block);
  const bool ok = h < nh;
  int eR = ix::kZeroE, eI = ix::kZeroE;
  if (ok) ix_half_prep<W>(x, h, threadIdx.x, blockDim.x, sR, sI, gstride, eR, eI);
  ix_warp_max(eR, eI, threadIdx.x, sm.wmax);
  __syncthreads();
  if (ok) ix_block_rows<W>(x, threadIdx.x, blockDim.x, sR, sI, gstride, sm.wmax);
  __syncthreads();
  if (!ok) return;
  IxTab tb{x.chm, x.che, hs};
  size_t base = (size_t)h * pitch;
  IxSt st{x.a.u_in + 2 * W * ws + (size_t)h * pitch, ws, nullptr, 0};
  if (x.stage) {
    if (!ix_bar_wait(sm.bar, x.wait_log2)) {
      atomicOr(x.a.status, 2u);
      return;
    }
    tb = IxTab{sm.tm, sm.te, (size_t)blockDim.y * pitch};
    base = (size_t)threadIdx.y * pitch;
    if (x.stage & 2) st = IxSt{sm.st + (size_t)threadIdx.y * pitch, (size_t)(blockDim.y + 1) * pitch, nullptr, 0};
  }
  uint32_t bad = 0;
  const auto half = ix_pow2<W>(-1);
  const auto h4 = IxT<W>::load(x.a.h4, 1, bad);
  for (int j = threadIdx.x; j < x.a.g.n_th; j += blockDim.x)
    ix_half_point<W>(x, h, j, sR, sI, gstride, half, h4, tb, base + j, IxSt{st.q + j, st.qw, nullptr, 0});
}

template <int W, int V>
__global__ void __launch_bounds__(RowBounds<V>::threads, RowBounds<V>::blocks) full_ix_kernel(IxArgs x) {
  const int gstride = x.a.g.n_th + 2 * x.a.radius, pitch = x.a.g.pitch, n_r = x.a.g.n_r;
  const size_t ws = (size_t)n_r * pitch, hs = (size_t)(n_r - 1) * pitch;
  IxRow sR, sI;
  const IxSmem sm = ix_rows<W>(gstride, pitch, x.stage, sR, sI, blockDim.y, threadIdx.y, true);
  const int i0 = 1 + blockIdx.x * blockDim.y, i = i0 + threadIdx.y;
  if (x.stage && threadIdx.x == 0 && threadIdx.y == 0)
    ix_stage<W>(sm, x.stage, x.cnm, x.cne, ws, pitch, i0, min((int)blockDim.y, n_r - 1 - i0), x.a.uh, hs, i0 - 1,
                x.a.u_in, ws, (int)blockIdx.x == x.stall_block);
  const bool ok = i < n_r - 1;
  int eR = ix::kZeroE, eI = ix::kZeroE;
  if (ok) ix_full_prep<W>(x, i, threadIdx.x, blockDim.x, sR, sI, gstride, eR, eI);
  ix_warp_max(eR, eI, threadIdx.x, sm.wmax);
  __syncthreads();
  if (ok) ix_block_rows<W>(x, threadIdx.x, blockDim.x, sR, sI, gstride, sm.wmax);
  __syncthreads();
  if (!ok) return;
  IxTab tb{x.cnm, x.cne, ws};
  size_t base = (size_t)i * pitch;
  IxSt st{x.a.uh + 2 * W * hs + (size_t)(i - 1) * pitch, hs, x.a.u_in + (size_t)i * pitch, ws};
  if (x.stage) {
    if (!ix_bar_wait(sm.bar, x.wait_log2)) {
      atomicOr(x.a.status, 2u);
      return;
    }
    tb = IxTab{sm.tm, sm.te, (size_t)blockDim.y * pitch};
    base = (size_t)threadIdx.y * pitch;
    if (x.stage & 2) {
      const size_t qw = (size_t)(blockDim.y + 1) * pitch;
      st = IxSt{sm.st + (size_t)threadIdx.y * pitch, qw, sm.st + 2 * W * qw + (size_t)threadIdx.y * pitch,
                (size_t)blockDim.y * pitch};
    }
  }
  uint32_t bad = 0;
  const auto one = ix_pow2<W>(0);
  const auto h2 = IxT<W>::load(x.a.h2, 1, bad);
  long long slot = -1;
  if (x.a.record) slot = x.a.ring_slot >= 0 ? x.a.ring_slot : (*x.a.ring_counter) % x.a.ring_cap;
  bool anybad = false;
  for (int j = threadIdx.x; j < x.a.g.n_th; j += blockDim.x)
    anybad |= ix_full_point<W>(x, i, j, sR, sI, gstride, one, h2, slot, tb, base + j,
                               IxSt{st.q + j, st.qw, st.u + j, st.uw});
  if (anybad) atomicOr(x.a.status, 1u);
}

// Batched execution on the integer engine: batch_kernel's rounds (every member with k > q
// performs iteration q; half-step phase, grid barrier, full-step phase, grid barrier) with the
// engine's row set-up and point functions per work item (rows x theta threads of the block;
// tables read from global memory). ix: the members' engine arguments, indexed like b.m.
template <int W>
__global__ void __launch_bounds__(256, 2) batch_ix_kernel(BatchArgs b, const IxArgs* ix) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  for (int s = 0; s < b.n_outer; ++s) {
    for (int q = 0; q < b.k_max; ++q) {
      const int n_act = b.active_items[q];
      for (int it = blockIdx.x; it < n_act; it += gridDim.x) {
        const int mi = b.item_member[it];
        const BatchMember& M = b.m[mi];
        const IxArgs& x = ix[mi];
        const int tx = threadIdx.x % M.tx, ty = threadIdx.x / M.tx;
        const bool row = ty < M.rows;
        const int h = (it - M.item_begin) * M.rows + ty, nh = M.a.g.n_r - 1, pitch = M.a.g.pitch;
        const size_t ws = (size_t)M.a.g.n_r * pitch;
        const bool ok = row && h < nh;
        const int gstride = M.a.g.n_th + 2 * M.a.radius;
        IxRow sR, sI;
        const IxSmem sm = ix_rows<W>(gstride, pitch, 0, sR, sI, M.rows, row ? ty : 0, false);
        int eR = ix::kZeroE, eI = ix::kZeroE;
        if (ok) ix_half_prep<W>(x, h, tx, M.tx, sR, sI, gstride, eR, eI);
        ix_warp_max(eR, eI, tx, sm.wmax, row);
        __syncthreads();
        if (ok) ix_block_rows<W>(x, tx, M.tx, sR, sI, gstride, sm.wmax);
        __syncthreads();
        if (ok) {
          uint32_t bad = 0;
          const auto half = ix_pow2<W>(-1);
          const auto h4 = IxT<W>::load(M.a.h4, 1, bad);
          const IxTab tb{x.chm, x.che, (size_t)nh * pitch};
          for (int j = tx; j < M.a.g.n_th; j += M.tx)
            ix_half_point<W>(x, h, j, sR, sI, gstride, half, h4, tb, (size_t)h * pitch + j,
                             IxSt{M.a.u_in + 2 * W * ws + (size_t)h * pitch + j, ws, nullptr, 0});
        }
        __syncthreads();
      }
      grid.sync();
      for (int it = blockIdx.x; it < n_act; it += gridDim.x) {
        const int mi = b.item_member[it];
        const BatchMember& M = b.m[mi];
        const IxArgs& x = ix[mi];
        const int tx = threadIdx.x % M.tx, ty = threadIdx.x / M.tx;
        const bool row = ty < M.rows;
        const int i = 1 + (it - M.item_begin) * M.rows + ty, n_r = M.a.g.n_r, pitch = M.a.g.pitch;
        const size_t ws = (size_t)n_r * pitch, hs = (size_t)(n_r - 1) * pitch;
        const bool ok = row && i < n_r - 1;
        const int gstride = M.a.g.n_th + 2 * M.a.radius;
        IxRow sR, sI;
        const IxSmem sm = ix_rows<W>(gstride, pitch, 0, sR, sI, M.rows, row ? ty : 0, true);
        int eR = ix::kZeroE, eI = ix::kZeroE;
        if (ok) ix_full_prep<W>(x, i, tx, M.tx, sR, sI, gstride, eR, eI);
        ix_warp_max(eR, eI, tx, sm.wmax, row);
        __syncthreads();
        if (ok) ix_block_rows<W>(x, tx, M.tx, sR, sI, gstride, sm.wmax);
        __syncthreads();
        if (ok) {
          uint32_t bad = 0;
          const auto one = ix_pow2<W>(0);
          const auto h2 = IxT<W>::load(M.a.h2, 1, bad);
          const long long slot = (q == M.k - 1 && M.ring_cap > 0) ? (M.ring_base + s) % M.ring_cap : -1;
          const IxTab tb{x.cnm, x.cne, (size_t)n_r * pitch};
          bool anybad = false;
          for (int j = tx; j < M.a.g.n_th; j += M.tx)
            anybad |= ix_full_point<W>(x, i, j, sR, sI, gstride, one, h2, slot, tb, (size_t)i * pitch + j,
                                       IxSt{M.a.uh + 2 * W * hs + (size_t)(i - 1) * pitch + j, hs,
                                            M.a.u_in + (size_t)i * pitch + j, ws});
          if (anybad) atomicOr(M.a.status, 1u);
        }
        __syncthreads();
      }
      grid.sync();
    }
  }
}

#undef IXD
#undef IXHD

}  // namespace teuk
