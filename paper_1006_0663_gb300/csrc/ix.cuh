// Integer engine for double-double dot products.
//
// GB300 executes 2 FP64 operations per SM per cycle but about 60-80 integer instructions, so
// the multi-word arithmetic of the Lax-Wendroff step (Sec. 3.D, Sec. 4: "quadruple" precision)
// runs here on the integer pipe: every operand becomes a 128-bit fixed-point mantissa with an
// exponent, products are formed from 32-bit limbs (multiply-add with carry chains), and the
// terms of a dot product are added, aligned to the largest, in a 192-bit two's-complement
// accumulator. Only the final split into two doubles uses three FP64 operations (Fast2Sum).
//
// Accuracy (worst case): a product keeps the partial products of weight >= 2^96 of the
// 256-bit product; the dropped ones (columns 0-2 of 32-bit limbs) sum to less than 3 * 2^128,
// i.e. less than 2^-122.4 of a product of two mantissas >= 2^126. Terms below the
// accumulator's last bit (2^-185 of the largest) are truncated, and the result is cut to 106
// bits before the final rounding: an N-term dot product is within about 2^-105 of its own
// magnitude plus N 2^-122.4 of its largest term (2^-118.8 for 12 terms), tighter than the
// FP64 error-free-transform accumulator it replaces (2^-104 of the sum of |terms|). Subnormal
// inputs are treated as zero; Inf/NaN inputs set `bad`.
//
// The same code runs on the host (tests) and the device; integer arithmetic makes them agree
// bit for bit.
#pragma once

#include <cstdint>
#include <cstring>

#include "mw.cuh"

namespace ix {

constexpr int32_t kZeroE = -(1 << 24);  // exponent given to zero: never the largest term

// (-1)^neg * M * 2^e with M = m[3]:m[2]:m[1]:m[0] < 2^128 (numbers made from a double-double
// have their leading bit at position 126).
struct Num {
  uint32_t m[4];
  int32_t e;
  uint32_t neg;
};

// 192-bit two's-complement accumulator, value = A * 2^B.
struct Acc {
  uint32_t a[6];
};

MW_HD uint64_t bits_of(double x) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  std::memcpy(&b, &x, 8);
  return b;
#endif
}
MW_HD double double_of(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double x;
  std::memcpy(&x, &b, 8);
  return x;
#endif
}
MW_HD uint32_t lo32(uint64_t x) { return (uint32_t)x; }
MW_HD uint32_t hi32(uint64_t x) { return (uint32_t)(x >> 32); }
// (hi:lo) >> s for 0 <= s < 32 (the high word's bits enter from the left)
MW_HD uint32_t fshr(uint32_t lo, uint32_t hi, uint32_t s) {
#if defined(__CUDA_ARCH__)
  return __funnelshift_r(lo, hi, s);
#else
  return s == 0 ? lo : (lo >> s) | (hi << (32 - s));
#endif
}
// (hi:lo) << s for 0 <= s < 32, high word of the result
MW_HD uint32_t fshl(uint32_t lo, uint32_t hi, uint32_t s) {
#if defined(__CUDA_ARCH__)
  return __funnelshift_l(lo, hi, s);
#else
  return s == 0 ? hi : (hi << s) | (lo >> (32 - s));
#endif
}
MW_HD int clz32(uint32_t x) {
#if defined(__CUDA_ARCH__)
  return __clz(x);
#else
  return x == 0 ? 32 : __builtin_clz(x);
#endif
}

MW_HD Num zero() { return Num{{0, 0, 0, 0}, kZeroE, 0}; }

// 128-bit helpers on (hi, lo) 64-bit halves
MW_HD void shl128(uint64_t x, int s, uint64_t& hi, uint64_t& lo) {  // x << s, 0 <= s < 128
  lo = s < 64 ? x << s : 0;
  hi = s == 0 ? 0 : (s < 64 ? x >> (64 - s) : x << (s - 64));
}

// A double-double (h, l), |l| <= ulp(h)/2, as a Num with the leading bit of h at position 126.
MW_HD Num from_dd(double h, double l, uint32_t& bad) {
  const uint64_t bh = bits_of(h), bl = bits_of(l);
  const int eh = (int)((bh >> 52) & 0x7ff), el = (int)((bl >> 52) & 0x7ff);
  bad |= (uint32_t)(eh == 0x7ff) | (uint32_t)(el == 0x7ff);
  if (eh == 0 || eh == 0x7ff) return zero();
  const uint64_t mh = (bh & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  uint64_t hi = mh << 10, lo = 0;  // mh << 74
  if (el != 0 && el != 0x7ff) {
    const uint64_t ml = (bl & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = 74 - (eh - el);
    uint64_t Lhi = 0, Llo = 0;
    if (sh >= 0) {
      shl128(ml, sh, Lhi, Llo);
    } else if (sh > -64) {
      Llo = ml >> (-sh);
    }
    if ((bl >> 63) == (bh >> 63)) {
      lo += Llo;
      hi += Lhi + (lo < Llo);
    } else {
      const uint64_t b = lo < Llo;
      lo -= Llo;
      hi -= Lhi + b;
    }
  }
  Num r;
  r.m[0] = lo32(lo); r.m[1] = hi32(lo); r.m[2] = lo32(hi); r.m[3] = hi32(hi);
  r.e = eh - 1149;  // (eh - 1023) - 52 - 74
  r.neg = (uint32_t)(bh >> 63);
  return r;
}

MW_HD bool is_zero(const Num& x) { return (x.m[0] | x.m[1] | x.m[2] | x.m[3]) == 0; }

// Window of the product of two mantissas: p = sum over i + j >= 3 of a_i b_j 2^(32(i+j) - 96),
// i.e. the 256-bit product divided by 2^96, without the partial products of lower weight.
MW_HD void mul_window(const uint32_t* a, const uint32_t* b, uint32_t* p) {
#if defined(__CUDA_ARCH__)
  uint32_t t0 = 0, t1 = 0, t2 = 0;
  // column 3: (0,3) (1,2) (2,1) (3,0)
  asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\tmadc.hi.cc.u32 %1, %3, %4, %1;\n\taddc.u32 %2, %2, 0;\n\t"
      "mad.lo.cc.u32 %0, %5, %6, %0;\n\tmadc.hi.cc.u32 %1, %5, %6, %1;\n\taddc.u32 %2, %2, 0;\n\t"
      "mad.lo.cc.u32 %0, %7, %8, %0;\n\tmadc.hi.cc.u32 %1, %7, %8, %1;\n\taddc.u32 %2, %2, 0;\n\t"
      "mad.lo.cc.u32 %0, %9, %10, %0;\n\tmadc.hi.cc.u32 %1, %9, %10, %1;\n\taddc.u32 %2, %2, 0;"
      : "+r"(t0), "+r"(t1), "+r"(t2)
      : "r"(a[0]), "r"(b[3]), "r"(a[1]), "r"(b[2]), "r"(a[2]), "r"(b[1]), "r"(a[3]), "r"(b[0]));
  p[0] = t0; t0 = t1; t1 = t2; t2 = 0;
  // column 4: (1,3) (2,2) (3,1)
  asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\tmadc.hi.cc.u32 %1, %3, %4, %1;\n\taddc.u32 %2, %2, 0;\n\t"
      "mad.lo.cc.u32 %0, %5, %6, %0;\n\tmadc.hi.cc.u32 %1, %5, %6, %1;\n\taddc.u32 %2, %2, 0;\n\t"
      "mad.lo.cc.u32 %0, %7, %8, %0;\n\tmadc.hi.cc.u32 %1, %7, %8, %1;\n\taddc.u32 %2, %2, 0;"
      : "+r"(t0), "+r"(t1), "+r"(t2)
      : "r"(a[1]), "r"(b[3]), "r"(a[2]), "r"(b[2]), "r"(a[3]), "r"(b[1]));
  p[1] = t0; t0 = t1; t1 = t2; t2 = 0;
  // column 5: (2,3) (3,2)
  asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\tmadc.hi.cc.u32 %1, %3, %4, %1;\n\taddc.u32 %2, %2, 0;\n\t"
      "mad.lo.cc.u32 %0, %5, %6, %0;\n\tmadc.hi.cc.u32 %1, %5, %6, %1;\n\taddc.u32 %2, %2, 0;"
      : "+r"(t0), "+r"(t1), "+r"(t2)
      : "r"(a[2]), "r"(b[3]), "r"(a[3]), "r"(b[2]));
  p[2] = t0; t0 = t1; t1 = t2;
  // column 6: (3,3); column 7 is the carry
  asm("mad.lo.cc.u32 %0, %2, %3, %0;\n\tmadc.hi.u32 %1, %2, %3, %1;"
      : "+r"(t0), "+r"(t1)
      : "r"(a[3]), "r"(b[3]));
  p[3] = t0;
  p[4] = t1;
#else
  // column sums with a 96-bit running total (lo 64 bits + carry word)
  uint64_t acc = 0, carry = 0;
  auto add = [&](uint32_t x, uint32_t y) {
    const uint64_t q = (uint64_t)x * y;
    acc += q;
    carry += acc < q;
  };
  auto shift = [&]() {
    acc = (acc >> 32) | (carry << 32);
    carry = 0;
  };
  add(a[0], b[3]); add(a[1], b[2]); add(a[2], b[1]); add(a[3], b[0]);
  p[0] = lo32(acc); shift();
  add(a[1], b[3]); add(a[2], b[2]); add(a[3], b[1]);
  p[1] = lo32(acc); shift();
  add(a[2], b[3]); add(a[3], b[2]);
  p[2] = lo32(acc); shift();
  add(a[3], b[3]);
  p[3] = lo32(acc);
  p[4] = hi32(acc);
#endif
}

// acc += (-1)^neg * (P * 2^32) >> r, for the 5-limb window P; r >= 192 adds nothing.
MW_HD void acc_add(Acc& acc, const uint32_t* p, uint32_t neg, int r) {
  if (r >= 192) return;
  uint32_t q[6] = {0, p[0], p[1], p[2], p[3], p[4]};
  // barrel shift right by r: whole limbs by 4, 2, 1, then the bits
  const bool s128 = (r & 128) != 0, s64 = (r & 64) != 0, s32 = (r & 32) != 0;
#pragma unroll
  for (int k = 0; k < 6; ++k) q[k] = s128 ? (k + 4 < 6 ? q[k + 4] : 0u) : q[k];
#pragma unroll
  for (int k = 0; k < 6; ++k) q[k] = s64 ? (k + 2 < 6 ? q[k + 2] : 0u) : q[k];
#pragma unroll
  for (int k = 0; k < 6; ++k) q[k] = s32 ? (k + 1 < 6 ? q[k + 1] : 0u) : q[k];
  const uint32_t b = (uint32_t)r & 31u;
  uint32_t t[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) t[k] = fshr(q[k], k + 1 < 6 ? q[k + 1] : 0u, b);
  // add t or its two's complement (~t + 1)
  const uint32_t mask = 0u - neg;
#if defined(__CUDA_ARCH__)
  uint32_t junk;  // only the carry of this first addition is used (the sum itself is dropped)
  asm("add.cc.u32 %6, %7, 0xffffffff;\n\t"
      "addc.cc.u32 %0, %0, %8;\n\taddc.cc.u32 %1, %1, %9;\n\taddc.cc.u32 %2, %2, %10;\n\t"
      "addc.cc.u32 %3, %3, %11;\n\taddc.cc.u32 %4, %4, %12;\n\taddc.u32 %5, %5, %13;"
      : "+r"(acc.a[0]), "+r"(acc.a[1]), "+r"(acc.a[2]), "+r"(acc.a[3]), "+r"(acc.a[4]), "+r"(acc.a[5]),
        "=r"(junk)
      : "r"(neg), "r"(t[0] ^ mask), "r"(t[1] ^ mask), "r"(t[2] ^ mask), "r"(t[3] ^ mask), "r"(t[4] ^ mask),
        "r"(t[5] ^ mask));
  (void)junk;
#else
  uint64_t c = neg;
  for (int k = 0; k < 6; ++k) {
    const uint64_t s = (uint64_t)acc.a[k] + (t[k] ^ mask) + c;
    acc.a[k] = lo32(s);
    c = s >> 32;
  }
#endif
}

// Magnitude and sign of the accumulator, with the index of the top set bit (-1 for zero).
MW_HD void acc_abs(const Acc& acc, uint32_t* m, uint32_t& neg, int& top) {
  neg = acc.a[5] >> 31;
  const uint32_t mask = 0u - neg;
  uint64_t c = neg;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const uint64_t s = (uint64_t)(acc.a[k] ^ mask) + c;
    m[k] = lo32(s);
    c = s >> 32;
  }
  top = -1;
#pragma unroll
  for (int k = 0; k < 6; ++k)
    if (m[k] != 0) top = 32 * k + 31 - clz32(m[k]);
}

// m (6 limbs) shifted left by z, 0 <= z < 192, in place
MW_HD void shl192(uint32_t* m, int z) {
  const bool s128 = (z & 128) != 0, s64 = (z & 64) != 0, s32 = (z & 32) != 0;
#pragma unroll
  for (int k = 5; k >= 0; --k) m[k] = s128 ? (k - 4 >= 0 ? m[k - 4] : 0u) : m[k];
#pragma unroll
  for (int k = 5; k >= 0; --k) m[k] = s64 ? (k - 2 >= 0 ? m[k - 2] : 0u) : m[k];
#pragma unroll
  for (int k = 5; k >= 0; --k) m[k] = s32 ? (k - 1 >= 0 ? m[k - 1] : 0u) : m[k];
  const uint32_t b = (uint32_t)z & 31u;
#pragma unroll
  for (int k = 5; k >= 0; --k) m[k] = fshl(k - 1 >= 0 ? m[k - 1] : 0u, m[k], b);
}

// A double from a 53-bit-or-shorter integer x (< 2^53) times 2^ex, sign s (0 if x == 0 or
// the result underflows the normal range).
MW_HD double make_double(uint64_t x, int ex, uint32_t s) {
  if (x == 0) return 0.0;
  const int lz = (x >> 32) != 0 ? clz32(hi32(x)) : 32 + clz32(lo32(x));
  const int sh = lz - 11;  // bring the leading bit to position 52
  const uint64_t m = x << sh;
  const int be = ex - sh + 52 + 1023;  // biased exponent of the leading bit
  if (be <= 0) return 0.0;
  const uint64_t bits = ((uint64_t)s << 63) | ((uint64_t)(be >= 2047 ? 2047 : be) << 52) |
                        (be >= 2047 ? 0ull : (m & 0xFFFFFFFFFFFFFull));
  return double_of(bits);
}

// Result of a dot product as a double-double: the top 106 bits of |A| as two doubles (exact),
// normalised by Fast2Sum. B is the exponent of the accumulator's bit 0.
MW_HD mw::dd to_dd(const Acc& acc, int B) {
  uint32_t m[6], neg;
  int top;
  acc_abs(acc, m, neg, top);
  if (top < 0) return mw::dd{0.0, 0.0};
  shl192(m, 191 - top);  // leading bit at 191
  const uint64_t hi53 = (((uint64_t)m[5] << 32) | m[4]) >> 11;  // bits 191..139
  const uint64_t x = ((uint64_t)m[4] << 32) | m[3];               // bits 159..96
  const uint64_t lo53 = ((x << 10) | (m[2] >> 22)) & ((1ull << 53) - 1);  // bits 138..86
  const int E = B + top;  // exponent of the leading bit
  const double h = make_double(hi53, E - 52, neg);
  const double l = make_double(lo53, E - 105, neg);
  mw::dd r;
  mw::fast_two_sum(h, l, r.h, r.l);
  return r;
}

// Result of a dot product as a Num (leading bit at 126, the bits below cut).
MW_HD Num to_num(const Acc& acc, int B) {
  uint32_t m[6], neg;
  int top;
  acc_abs(acc, m, neg, top);
  if (top < 0) return zero();
  shl192(m, 191 - top);
  Num r;
  // bits 191..64 shifted right by one: leading bit at 126
#pragma unroll
  for (int k = 0; k < 4; ++k) r.m[k] = fshr(m[k + 2], k + 3 < 6 ? m[k + 3] : 0u, 1);
  r.e = B + top - 126;
  r.neg = neg;
  return r;
}

// ---- dot products in two passes: the exponents of all terms first (the largest sets the
// accumulator's alignment), then the products one at a time (only one term's limbs live).

// Exponent of the product window of c v (2 kZeroE if either is zero: never aligned in).
MW_HD int prod_exp(int ec, int ev) { return (ec == kZeroE || ev == kZeroE) ? 2 * kZeroE : ec + ev + 96; }
MW_HD void acc_zero(Acc& acc) {
#pragma unroll
  for (int k = 0; k < 6; ++k) acc.a[k] = 0;
}
// acc += (-1)^neg c v, for the product exponent ep = prod_exp(.) and the largest one maxE.
MW_HD void acc_prod(Acc& acc, const uint32_t* cm, const uint32_t* vm, uint32_t neg, int ep, int maxE) {
  const int r = maxE + 6 - ep;
  if (r >= 192) return;
  uint32_t p[5];
  mul_window(cm, vm, p);
  acc_add(acc, p, neg, r < 0 ? 0 : r);
}
// acc += (-1)^neg c v for c a power of two (mantissa 2^126, as made by a constant 2^k): the
// product window is v's mantissa shifted left by 30, the same bits mul_window gives.
MW_HD void acc_prod_pow2(Acc& acc, const uint32_t* vm, uint32_t neg, int ep, int maxE) {
  const int r = maxE + 6 - ep;
  if (r >= 192) return;
  uint32_t p[5];
  p[0] = vm[0] << 30;
#pragma unroll
  for (int k = 1; k < 4; ++k) p[k] = fshl(vm[k - 1], vm[k], 30);
  p[4] = vm[3] >> 2;
  acc_add(acc, p, neg, r < 0 ? 0 : r);
}
// Exponent of the accumulator's bit 0 for the largest product exponent maxE.
MW_HD int acc_base(int maxE) { return maxE - 26; }

// Dot product of N pairs held in registers: sum_k (-1)^{neg} c_k v_k.
template <int N>
MW_HD void dot(const Num* c, const Num* v, Acc& acc, int& B) {
  int maxE = 2 * kZeroE;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int ep = prod_exp(c[k].e, v[k].e);
    maxE = ep > maxE ? ep : maxE;
  }
  acc_zero(acc);
#pragma unroll
  for (int k = 0; k < N; ++k) acc_prod(acc, c[k].m, v[k].m, c[k].neg ^ v[k].neg, prod_exp(c[k].e, v[k].e), maxE);
  B = acc_base(maxE);
}

// Sum or difference a + (-1)^negate_b b of two Nums with mantissas below 2^127 (made from
// double-doubles): the operand of smaller exponent is shifted to the larger one's exponent
// (bits below its last are cut: relative error < 2^-126 of the larger) and the mantissas are
// added or subtracted; the result keeps the larger exponent (mantissa below 2^128).
MW_HD Num add(const Num& a, const Num& b, uint32_t negate_b) {
  const uint32_t bneg = b.neg ^ negate_b;
  if (b.e == kZeroE) { Num r = a; return r; }
  if (a.e == kZeroE) { Num r = b; r.neg = bneg; return r; }
  const bool swap = b.e > a.e;
  uint32_t big[4], sm[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    big[k] = swap ? b.m[k] : a.m[k];
    sm[k] = swap ? a.m[k] : b.m[k];
  }
  const int e = swap ? b.e : a.e;
  const uint32_t nbig = swap ? bneg : a.neg, nsm = swap ? a.neg : bneg;
  const int s = swap ? b.e - a.e : a.e - b.e;
  // sm >>= s (s >= 128 clears it)
  const bool s128 = s >= 128, s64 = (s & 64) != 0, s32 = (s & 32) != 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) sm[k] = s128 ? 0u : sm[k];
#pragma unroll
  for (int k = 0; k < 4; ++k) sm[k] = s64 ? (k + 2 < 4 ? sm[k + 2] : 0u) : sm[k];
#pragma unroll
  for (int k = 0; k < 4; ++k) sm[k] = s32 ? (k + 1 < 4 ? sm[k + 1] : 0u) : sm[k];
  const uint32_t bs = (uint32_t)s & 31u;
#pragma unroll
  for (int k = 0; k < 4; ++k) sm[k] = fshr(sm[k], k + 1 < 4 ? sm[k + 1] : 0u, bs);
  // big +- sm as a signed 160-bit value
  const uint32_t sub = nbig ^ nsm, mask = 0u - sub;
  uint32_t r[5];
  uint64_t c = sub;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint64_t t = (uint64_t)big[k] + (sm[k] ^ mask) + c;
    r[k] = lo32(t);
    c = t >> 32;
  }
  r[4] = lo32(c + mask);  // 0 or 1 for a sum; 0 (no borrow) or 0xffffffff (negative) for a difference
  const uint32_t flip = r[4] >> 31, fm = 0u - flip;
  Num out;
  uint64_t cc = flip;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint64_t t = (uint64_t)(r[k] ^ fm) + cc;
    out.m[k] = lo32(t);
    cc = t >> 32;
  }
  out.e = e;
  out.neg = nbig ^ flip;
  if ((out.m[0] | out.m[1] | out.m[2] | out.m[3]) == 0) return zero();
  return out;
}

}  // namespace ix
