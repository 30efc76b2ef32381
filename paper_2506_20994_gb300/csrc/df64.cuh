// Double-float arithmetic: a value is carried as an unevaluated sum hi + lo
// of two fp32 numbers (Dekker 1971, "A floating-point technique for
// extending the available precision"; the error-free transformations
// TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and TwoProduct-by-FMA (Ogita, Rump,
// Oishi 2005, "Accurate sum and dot product")).  About 48 significant bits,
// fp32 exponent range.
//
// Conversions to and from IEEE fp64 use integer operations on the bit
// patterns only, so a kernel built on these helpers issues no fp64
// instruction.  All fp32 operations are written with the explicitly rounded
// intrinsics so that the compiler cannot contract or reassociate them.
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define DF_HD __host__ __device__ __forceinline__
#else
#define DF_HD inline
#endif

namespace ax {
namespace df {

struct df2 {
  float hi, lo;
};

// --- bit casts and explicitly rounded fp32 ops usable on host and device --
DF_HD uint32_t f2u(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
#endif
}
DF_HD float u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}
DF_HD uint64_t d2u(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t u;
  memcpy(&u, &d, 8);
  return u;
#endif
}
DF_HD double u2d(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  memcpy(&d, &u, 8);
  return d;
#endif
}
#ifdef __CUDA_ARCH__
DF_HD float add(float a, float b) { return __fadd_rn(a, b); }
DF_HD float sub(float a, float b) { return __fsub_rn(a, b); }
DF_HD float mul(float a, float b) { return __fmul_rn(a, b); }
DF_HD float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
DF_HD int f2i_rn(float a) { return __float2int_rn(a); }
#else
// Host twins (used by the host-side self-test entry point only); volatile
// keeps the host compiler from contracting the error-free transformations.
DF_HD float add(float a, float b) { volatile float r = a + b; return r; }
DF_HD float sub(float a, float b) { volatile float r = a - b; return r; }
DF_HD float mul(float a, float b) { volatile float r = a * b; return r; }
DF_HD float fma(float a, float b, float c) { return __builtin_fmaf(a, b, c); }
DF_HD int f2i_rn(float a) { return (int)__builtin_nearbyintf(a); }
#endif

// --- fp64 -> double-float split, integer ops only ---------------------------
// hi = x truncated to 24 significant bits; lo = the next 23 bits of x, so
// |x - (hi + lo)| < 2^-46 |x| for 2^-80 <= |x| < 2^128.  Smaller magnitudes
// keep an absolute error below 2^-100 (hi flushes toward zero below 2^-126).
DF_HD df2 split(double x) {
  const uint64_t b = d2u(x);
  const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
  const uint32_t sgn = hw & 0x80000000u;
  uint32_t mag = hw & 0x7FFFFFFFu;            // exponent(11) | mantissa-high(20)
  const uint32_t bias = 896u << 20;           // 1023 - 127
  mag = mag < bias ? bias : mag;              // flush below the fp32 normal range
  // ((mag - bias) << 3) | (lw >> 29): fp32 exponent(8) | 23 mantissa bits
  const uint32_t fh = (((mag - bias) << 3) | (lw >> 29)) | sgn;
  // remaining 29 bits r of the mantissa, value r * 2^(e-1075); keep the top 23
  const uint32_t r23 = (lw >> 6) & 0x7FFFFFu;
  const float rf = sub(u2f(0x4B000000u | r23), 8388608.0f);  // exact integer r >> 6
  const uint32_t e = (hw >> 20) & 0x7FFu;
  // +-2^(e-1069), or zero (lo dropped) below |x| = 2^-80
  const uint32_t sc = e >= 943u ? (((e - 942u) << 23) | sgn) : 0u;
  df2 o;
  o.hi = u2f(fh);
  o.lo = mul(rf, u2f(sc));
  return o;
}

// Round-to-nearest split for data converted once (prepared geometry,
// coefficients): hi = fl32(x), lo = fl32(x - hi), |x - (hi + lo)| <= 2^-48 |x|
// for 2^-100 <= |x| < 2^127 (half the error of `split`; it costs fp64 and
// conversion instructions, so the kernels' per-apply splits use `split`).
DF_HD df2 split_rn(double x) {
  df2 o;
  o.hi = (float)x;
  o.lo = (float)(x - (double)o.hi);
  return o;
}

// --- double-float -> fp64, integer ops plus one fp32->int conversion -------
// Requires |lo| <= ulp(hi)/2 (a normalised pair, see `norm`).  Exact to
// within half an fp64 ulp of (hi + lo) for |hi| >= 2^-75; below that lo is
// dropped.  hi == 0 or fp32-subnormal gives (signed) zero.
DF_HD double join(float hi, float lo) {
  const uint32_t hb = f2u(hi);
  const uint32_t sgn = hb & 0x80000000u;
  const uint32_t eh = (hb >> 23) & 0xFFu;
  // |hi| as fp64 bits: exponent + 896, mantissa shifted up by 29
  const uint32_t mh = hb & 0x7FFFFFFFu;
  uint32_t whi = (mh >> 3) + (896u << 20);
  uint32_t wlo = mh << 29;
  // lo in units of the fp64 ulp at hi's exponent: round(lo * 2^(179 - eh))
  const uint32_t se = eh >= 52u ? (306u - eh) : 254u;
  int n = f2i_rn(mul(lo, u2f(se << 23)));
  if (eh < 52u) n = 0;
  n = sgn ? -n : n;                           // add to the magnitude
  // crossing down into the lower binade halves the ulp: count twice
  if ((mh & 0x7FFFFFu) == 0u && n < 0) n *= 2;
  uint64_t m = ((uint64_t)whi << 32) | wlo;
  m += (uint64_t)(int64_t)n;
  m |= (uint64_t)sgn << 32;
  if (eh == 0u) m = (uint64_t)sgn << 32;
  return u2d(m);
}

// --- error-free building blocks -------------------------------------------
// FastTwoSum: renormalise a pair whose hi dominates.
DF_HD df2 norm(float s, float c) {
  const float h = add(s, c);
  df2 o;
  o.hi = h;
  o.lo = sub(c, sub(h, s));
  return o;
}

// Running sum of products: s carries the exact-sum head, c the tail.
struct acc {
  float s, c;
};

// acc = d * u (first term of a sum).
DF_HD acc prod(df2 d, df2 u) {
  acc a;
  a.s = mul(d.hi, u.hi);
  float e = fma(d.hi, u.hi, -a.s);
  e = fma(d.hi, u.lo, e);
  a.c = fma(d.lo, u.hi, e);
  return a;
}

// acc += d * u: exact head product by FMA, exact head sum by TwoSum, the
// cross terms and both rounding errors folded into the tail.
DF_HD void mac(acc &a, df2 d, df2 u) {
  const float p = mul(d.hi, u.hi);
  float c = fma(d.hi, u.hi, -p);
  c = fma(d.hi, u.lo, c);
  c = fma(d.lo, u.hi, c);
  const float s = add(a.s, p);
  const float bp = sub(s, a.s);
  const float err = add(sub(a.s, sub(s, bp)), sub(p, bp));
  a.c = add(a.c, add(c, err));
  a.s = s;
}

DF_HD df2 result(acc a) { return norm(a.s, a.c); }

// Product of two pairs, left as an (almost normalised) pair.
DF_HD df2 mul2(df2 a, df2 b) {
  df2 o;
  o.hi = mul(a.hi, b.hi);
  float e = fma(a.hi, b.hi, -o.hi);
  e = fma(a.hi, b.lo, e);
  o.lo = fma(a.lo, b.hi, e);
  return o;
}

// --- packed pairs: two independent double-float lanes per 64-bit register --
// sm_100-class parts issue add/sub/mul/fma.rn.f32x2 at the fp32 lane rate but
// in half the issue slots; lane x and lane y are unrelated values.
#ifdef __CUDACC__
#define DF_D __device__ __forceinline__
typedef unsigned long long u64;
DF_D u64 pk(float x, float y) {
  return (u64)__float_as_uint(x) | ((u64)__float_as_uint(y) << 32);
}
DF_D float lx_(u64 v) { return __uint_as_float((unsigned)(v & 0xFFFFFFFFull)); }
DF_D float ly_(u64 v) { return __uint_as_float((unsigned)(v >> 32)); }
DF_D u64 add2(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
DF_D u64 sub2(u64 a, u64 b) {
  u64 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
DF_D u64 mul2p(u64 a, u64 b) {
  u64 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
DF_D u64 fma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Sign flips by integer XOR (integer pipe), keeping them off the fp32 pipe
// that the double-float arithmetic saturates.
DF_D u64 neg2(u64 a) { return a ^ 0x8000000080000000ull; }
DF_D float negf(float a) { return __uint_as_float(__float_as_uint(a) ^ 0x80000000u); }
DF_D u64 pk_pm(float x) { return pk(x, negf(x)); }  // (x, -x)

// Two double-float values, lane by lane: value_x = lx(hi)+lx(lo), etc.
struct __align__(16) dd2 {
  u64 hi, lo;
};
// Two running sums of products (heads s, tails c), lane by lane.
struct acc2 {
  u64 s, c;
};

// acc = d * u per lane (first term); nd = -d.hi (precomputed)
DF_D acc2 prod2(dd2 d, u64 nd, dd2 u) {
  acc2 a;
  a.s = mul2p(d.hi, u.hi);
  const u64 q = fma2(nd, u.hi, a.s);  // s - d.hi*u.hi = -(rounding error)
  u64 c = fma2(d.hi, u.lo, neg2(q));
  a.c = fma2(d.lo, u.hi, c);
  return a;
}

// acc += d * u per lane: TwoProduct by FMA, TwoSum on the heads, cross terms
// and both rounding errors into the tails.  nd = -d.hi.
DF_D void mac2(acc2 &a, dd2 d, u64 nd, dd2 u) {
  const u64 p = mul2p(d.hi, u.hi);
  const u64 q = fma2(nd, u.hi, p);  // p - d.hi*u.hi = -(error of p)
  u64 c = fma2(d.hi, u.lo, a.c);
  c = fma2(d.lo, u.hi, c);
  const u64 s = add2(a.s, p);
  const u64 bp = sub2(s, a.s);
  const u64 err = add2(sub2(a.s, sub2(s, bp)), sub2(p, bp));
  a.c = sub2(add2(c, err), q);
  a.s = s;
}

// (a + b) per lane, heads by TwoSum, not renormalised
DF_D dd2 dsum2(dd2 a, dd2 b) {
  const u64 s = add2(a.hi, b.hi);
  const u64 bp = sub2(s, a.hi);
  const u64 err = add2(sub2(a.hi, sub2(s, bp)), sub2(b.hi, bp));
  dd2 r;
  r.hi = s;
  r.lo = add2(add2(a.lo, b.lo), err);
  return r;
}
#endif

}  // namespace df
}  // namespace ax
