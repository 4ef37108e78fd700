// Integer engine for quad-double dot products: the construction of ix.cuh (double-double)
// with 256-bit mantissas, for the paper's "octal" precision (Sec. 3.D).
//
// A quad-double (x0, x1, x2, x3) becomes an 8-limb (256-bit) fixed-point mantissa with the
// leading bit of x0 at position 254 and an exponent; products keep all partial products of
// weight >= 2^224 of the 512-bit product (the dropped columns 0-6 sum to less than 7.2 *
// 2^256, i.e. 2^-249.1 of a product of two mantissas >= 2^254); the terms of a dot product
// are added, aligned to the largest, in a 320-bit two's-complement accumulator; the result's
// top 212 bits are cut into four doubles and renormalised (HLB01 renormalisation, FP64). An
// N-term dot product is within about 2^-208 of its own magnitude plus N 2^-249.1 of its
// largest term (2^-245.6 for 12 terms).
// Subnormal words are treated as zero; Inf/NaN words set `bad`.
#pragma once

#include "ix.cuh"

namespace ix {

struct Num8 {
  uint32_t m[8];
  int32_t e;
  uint32_t neg;
};
struct Acc10 {
  uint32_t a[10];
};

MW_HD Num8 zero8() {
  Num8 r;
#pragma unroll
  for (int k = 0; k < 8; ++k) r.m[k] = 0;
  r.e = kZeroE;
  r.neg = 0;
  return r;
}

// m (8 limbs) +- x 2^p for a 53-bit x and any p (bits below position 0 are cut).
MW_HD void add_shifted8(uint32_t* m, uint64_t x, int p, uint32_t subtract) {
  uint32_t X[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int s = 32 * k - p;  // position of limb k's bit 0 in x
    X[k] = s >= 64 ? 0u : (s >= 0 ? lo32(x >> s) : (s > -32 ? lo32(x << (-s)) : 0u));
  }
  const uint32_t mask = 0u - subtract;
  uint64_t c = subtract;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint64_t t = (uint64_t)m[k] + (X[k] ^ mask) + c;
    m[k] = lo32(t);
    c = t >> 32;
  }
}

// A normalised quad-double (|x_{k+1}| <= ulp(x_k)/2) as a Num8, leading bit of x0 at 254.
MW_HD Num8 from_qd(double x0, double x1, double x2, double x3, uint32_t& bad) {
  const uint64_t b0 = bits_of(x0);
  const int e0 = (int)((b0 >> 52) & 0x7ff);
  const double w[3] = {x1, x2, x3};
  bad |= (uint32_t)(e0 == 0x7ff);
#pragma unroll
  for (int k = 0; k < 3; ++k) bad |= (uint32_t)(((bits_of(w[k]) >> 52) & 0x7ff) == 0x7ff);
  if (e0 == 0 || e0 == 0x7ff) return zero8();
  Num8 r;
#pragma unroll
  for (int k = 0; k < 8; ++k) r.m[k] = 0;
  const uint64_t m0 = (b0 & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  add_shifted8(r.m, m0, 202, 0u);  // bits 202..254
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint64_t bk = bits_of(w[k]);
    const int ek = (int)((bk >> 52) & 0x7ff);
    if (ek == 0 || ek == 0x7ff) continue;
    const uint64_t mk = (bk & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    add_shifted8(r.m, mk, 202 - (e0 - ek), (uint32_t)((bk >> 63) != (b0 >> 63)));
  }
  r.e = e0 - 1277;  // (e0 - 1023) - 52 - 202
  r.neg = (uint32_t)(b0 >> 63);
  return r;
}

// Window of the product of two 8-limb mantissas: partial products a_i b_j with i + j >= 7,
// divided by 2^224 (9 limbs).
MW_HD void mul_window8(const uint32_t* a, const uint32_t* b, uint32_t* p) {
  uint32_t t0 = 0, t1 = 0, t2 = 0;
#pragma unroll
  for (int col = 7; col <= 14; ++col) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int j = col - i;
      if (j < 0 || j > 7) continue;
#if defined(__CUDA_ARCH__)
      asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\tmadc.hi.cc.u32 %1, %3, %4, %1;\n\taddc.u32 %2, %2, 0;"
          : "+r"(t0), "+r"(t1), "+r"(t2)
          : "r"(a[i]), "r"(b[j]));
#else
      const uint64_t q = (uint64_t)a[i] * b[j];
      const uint64_t lo = (uint64_t)t0 + lo32(q);
      const uint64_t hi = (uint64_t)t1 + hi32(q) + (lo >> 32);
      t0 = lo32(lo);
      t1 = lo32(hi);
      t2 += hi32(hi);
#endif
    }
    p[col - 7] = t0;
    t0 = t1;
    t1 = t2;
    t2 = 0;
  }
  p[8] = t0;  // column 15: the remaining carry
}

// acc += (-1)^neg * (P * 2^32) >> r for the 9-limb window P; r >= 320 adds nothing.
MW_HD void acc_add10(Acc10& acc, const uint32_t* p, uint32_t neg, int r) {
  if (r >= 320) return;
  uint32_t q[10];
  q[0] = 0;
#pragma unroll
  for (int k = 0; k < 9; ++k) q[k + 1] = p[k];
  const bool s256 = (r & 256) != 0, s128 = (r & 128) != 0, s64 = (r & 64) != 0, s32 = (r & 32) != 0;
#pragma unroll
  for (int k = 0; k < 10; ++k) q[k] = s256 ? (k + 8 < 10 ? q[k + 8] : 0u) : q[k];
#pragma unroll
  for (int k = 0; k < 10; ++k) q[k] = s128 ? (k + 4 < 10 ? q[k + 4] : 0u) : q[k];
#pragma unroll
  for (int k = 0; k < 10; ++k) q[k] = s64 ? (k + 2 < 10 ? q[k + 2] : 0u) : q[k];
#pragma unroll
  for (int k = 0; k < 10; ++k) q[k] = s32 ? (k + 1 < 10 ? q[k + 1] : 0u) : q[k];
  const uint32_t bsh = (uint32_t)r & 31u, mask = 0u - neg;
  uint64_t c = neg;
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    const uint32_t t = fshr(q[k], k + 1 < 10 ? q[k + 1] : 0u, bsh) ^ mask;
    const uint64_t s = (uint64_t)acc.a[k] + t + c;
    acc.a[k] = lo32(s);
    c = s >> 32;
  }
}

MW_HD void acc_zero10(Acc10& acc) {
#pragma unroll
  for (int k = 0; k < 10; ++k) acc.a[k] = 0;
}

// Product exponent of the window of c v (2 kZeroE if either is zero).
MW_HD int prod_exp8(int ec, int ev) { return (ec == kZeroE || ev == kZeroE) ? 2 * kZeroE : ec + ev + 224; }
MW_HD void acc_prod10(Acc10& acc, const uint32_t* cm, const uint32_t* vm, uint32_t neg, int ep, int maxE) {
  const int r = maxE + 6 - ep;
  if (r >= 320) return;
  uint32_t p[9];
  mul_window8(cm, vm, p);
  acc_add10(acc, p, neg, r < 0 ? 0 : r);
}
// acc += (-1)^neg c v for c a power of two (mantissa 2^254): v's mantissa shifted left by 30,
// the same bits mul_window8 gives.
MW_HD void acc_prod_pow2_10(Acc10& acc, const uint32_t* vm, uint32_t neg, int ep, int maxE) {
  const int r = maxE + 6 - ep;
  if (r >= 320) return;
  uint32_t p[9];
  p[0] = vm[0] << 30;
#pragma unroll
  for (int k = 1; k < 8; ++k) p[k] = fshl(vm[k - 1], vm[k], 30);
  p[8] = vm[7] >> 2;
  acc_add10(acc, p, neg, r < 0 ? 0 : r);
}
// exponent of the accumulator's bit 0 (the largest window's top lands at bit 312)
MW_HD int acc_base10(int maxE) { return maxE - 26; }

MW_HD void acc_abs10(const Acc10& acc, uint32_t* m, uint32_t& neg, int& top) {
  neg = acc.a[9] >> 31;
  const uint32_t mask = 0u - neg;
  uint64_t c = neg;
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    const uint64_t s = (uint64_t)(acc.a[k] ^ mask) + c;
    m[k] = lo32(s);
    c = s >> 32;
  }
  top = -1;
#pragma unroll
  for (int k = 0; k < 10; ++k)
    if (m[k] != 0) top = 32 * k + 31 - clz32(m[k]);
}

MW_HD void shl320(uint32_t* m, int z) {  // 0 <= z < 320
  const bool s256 = (z & 256) != 0, s128 = (z & 128) != 0, s64 = (z & 64) != 0, s32 = (z & 32) != 0;
#pragma unroll
  for (int k = 9; k >= 0; --k) m[k] = s256 ? (k - 8 >= 0 ? m[k - 8] : 0u) : m[k];
#pragma unroll
  for (int k = 9; k >= 0; --k) m[k] = s128 ? (k - 4 >= 0 ? m[k - 4] : 0u) : m[k];
#pragma unroll
  for (int k = 9; k >= 0; --k) m[k] = s64 ? (k - 2 >= 0 ? m[k - 2] : 0u) : m[k];
#pragma unroll
  for (int k = 9; k >= 0; --k) m[k] = s32 ? (k - 1 >= 0 ? m[k - 1] : 0u) : m[k];
  const uint32_t b = (uint32_t)z & 31u;
#pragma unroll
  for (int k = 9; k >= 0; --k) m[k] = fshl(k - 1 >= 0 ? m[k - 1] : 0u, m[k], b);
}

// 53 bits of the normalised 320-bit value starting at bit `hi` (hi - 52 .. hi), hi >= 52.
MW_HD uint64_t bits53(const uint32_t* m, int hi) {
  const int lo = hi - 52;
  const int w = lo >> 5, b = lo & 31;
  // three consecutive limbs from w cover bits lo .. lo + 95
  const uint32_t l0 = m[w], l1 = w + 1 < 10 ? m[w + 1] : 0u, l2 = w + 2 < 10 ? m[w + 2] : 0u;
  const uint64_t x = ((uint64_t)fshr(l1, l2, b) << 32) | fshr(l0, l1, b);
  return x & ((1ull << 53) - 1);
}

// Result of a dot product as a quad-double: the top 212 bits cut into four doubles, then
// renormalised. B is the exponent of the accumulator's bit 0.
MW_HD mw::qd to_qd(const Acc10& acc, int B) {
  uint32_t m[10], neg;
  int top;
  acc_abs10(acc, m, neg, top);
  if (top < 0) return mw::qd{0.0, 0.0, 0.0, 0.0};
  shl320(m, 319 - top);  // leading bit at 319
  const int E = B + top;
  double w[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) w[k] = make_double(bits53(m, 319 - 53 * k), E - 52 - 53 * k, neg);
  return mw::qd_renorm(w[0], w[1], w[2], w[3], 0.0);
}

// Result of a dot product as a Num8 (leading bit at 254, the bits below cut).
MW_HD Num8 to_num8(const Acc10& acc, int B) {
  uint32_t m[10], neg;
  int top;
  acc_abs10(acc, m, neg, top);
  if (top < 0) return zero8();
  shl320(m, 319 - top);
  Num8 r;
  // bits 319..64 shifted right by one: leading bit at 254
#pragma unroll
  for (int k = 0; k < 8; ++k) r.m[k] = fshr(m[k + 2], k + 3 < 10 ? m[k + 3] : 0u, 1);
  r.e = B + top - 254;
  r.neg = neg;
  return r;
}

// Sum / difference of two Num8 with mantissas below 2^255 (made from quad-doubles): the
// operand of smaller exponent is shifted to the larger exponent (cut below it: relative error
// < 2^-254 of the larger) and the mantissas are added or subtracted.
MW_HD Num8 add8(const Num8& a, const Num8& b, uint32_t negate_b) {
  const uint32_t bneg = b.neg ^ negate_b;
  if (b.e == kZeroE) return a;
  if (a.e == kZeroE) { Num8 r = b; r.neg = bneg; return r; }
  const bool swap = b.e > a.e;
  uint32_t big[8], sm[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    big[k] = swap ? b.m[k] : a.m[k];
    sm[k] = swap ? a.m[k] : b.m[k];
  }
  const int e = swap ? b.e : a.e;
  const uint32_t nbig = swap ? bneg : a.neg, nsm = swap ? a.neg : bneg;
  const int s = swap ? b.e - a.e : a.e - b.e;
  const bool s256 = s >= 256, s128 = (s & 128) != 0, s64 = (s & 64) != 0, s32 = (s & 32) != 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) sm[k] = s256 ? 0u : sm[k];
#pragma unroll
  for (int k = 0; k < 8; ++k) sm[k] = s128 ? (k + 4 < 8 ? sm[k + 4] : 0u) : sm[k];
#pragma unroll
  for (int k = 0; k < 8; ++k) sm[k] = s64 ? (k + 2 < 8 ? sm[k + 2] : 0u) : sm[k];
#pragma unroll
  for (int k = 0; k < 8; ++k) sm[k] = s32 ? (k + 1 < 8 ? sm[k + 1] : 0u) : sm[k];
  const uint32_t bs = (uint32_t)s & 31u;
#pragma unroll
  for (int k = 0; k < 8; ++k) sm[k] = fshr(sm[k], k + 1 < 8 ? sm[k + 1] : 0u, bs);
  const uint32_t sub = nbig ^ nsm, mask = 0u - sub;
  uint32_t r[9];
  uint64_t c = sub;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint64_t t = (uint64_t)big[k] + (sm[k] ^ mask) + c;
    r[k] = lo32(t);
    c = t >> 32;
  }
  r[8] = lo32(c + mask);
  const uint32_t flip = r[8] >> 31, fm = 0u - flip;
  Num8 out;
  uint64_t cc = flip;
  uint32_t any = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint64_t t = (uint64_t)(r[k] ^ fm) + cc;
    out.m[k] = lo32(t);
    cc = t >> 32;
    any |= out.m[k];
  }
  out.e = e;
  out.neg = nbig ^ flip;
  if (any == 0) return zero8();
  return out;
}

// Dot product of N pairs held in registers.
template <int N>
MW_HD void dot8(const Num8* c, const Num8* v, Acc10& acc, int& B) {
  int maxE = 2 * kZeroE;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int ep = prod_exp8(c[k].e, v[k].e);
    maxE = ep > maxE ? ep : maxE;
  }
  acc_zero10(acc);
#pragma unroll
  for (int k = 0; k < N; ++k) acc_prod10(acc, c[k].m, v[k].m, c[k].neg ^ v[k].neg, prod_exp8(c[k].e, v[k].e), maxE);
  B = acc_base10(maxE);
}

}  // namespace ix
