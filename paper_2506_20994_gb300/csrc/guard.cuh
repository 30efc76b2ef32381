// Range guard of the double-float kernels and their exact fallback.
//
// The double-float kernels (df64.cuh) carry an fp64 value as two fp32
// numbers.  That keeps ~47 significant bits only while every value and every
// intermediate of the operator w = D^T (h1 G (D u)) stays inside the fp32
// exponent range with room for the tails: the head of a value must be a
// normal fp32 number and the tail (2^-24 below it) too, and no intermediate
// may overflow.  Each kernel therefore records, per element, the largest
// binary exponent of u, of the six G fields and of h1 (and, per block, of
// the 1-D matrices), and checks the exponents of the products the operator
// forms against that window.  An element outside it (values that are
// infinite or NaN, fp64 magnitudes beyond the fp32 range, or a product chain
// that would underflow the tails) is recomputed by `element_f64` below with
// fp64 units, so that it gets IEEE fp64 semantics.  The same routine serves
// the even-odd kernels when the matrices are not centro-antisymmetric.
//
// Values below 2^-1022 (fp64 subnormals) count as zero in the exponent
// record; inside the window the double-float split flushes any value more
// than ~2^125 below the element's largest one, an absolute change below
// 2^-47 of that element's scale.
#pragma once

#include <stdint.h>

#include "common.cuh"

namespace ax {
namespace guard {

// Ordered key of |x|'s binary exponent: the fp64 high word shifted left by
// one (sign dropped).  max over values, then `field` recovers the biased
// exponent (0: zero or subnormal, 2047: Inf or NaN).
AX_D unsigned key(double x) {
  return (unsigned)(__double_as_longlong(x) >> 31) & 0xFFFFFFFEu;
}
AX_HD int field(unsigned k) { return (int)(k >> 21); }

// Window of the double-float arithmetic, from the biased exponent fields of
// the element maxima of u, G, h1 and of the matrices D (fd).  A zero factor
// gives w = 0 exactly; a non-finite one must go to fp64 units.
AX_HD bool window_ok(int fu, int fg, int fh, int fd) {
  if (fu == 2047 || fg == 2047 || fh == 2047 || fd == 2047) return false;
  if (fu == 0 || fg == 0 || fh == 0 || fd == 0) return true;
  const int a = fu - 1023, b = fg - 1023, c = fh - 1023, d = fd - 1023;
  auto in = [](int x, int lo, int hi) { return x >= lo && x <= hi; };
  // each factor: head and tail normal fp32 numbers
  if (!in(a, -78, 90) || !in(b, -78, 90) || !in(c, -78, 90) || !in(d, -24, 24)) return false;
  // the products in the order the kernels form them: D u, G (D u),
  // h1 G (D u), D^T (h1 G D u); bounded away from the fp32 limits with
  // room for sums of up to 3 * 16 terms
  return in(a + d, -90, 100) && in(a + b + d, -90, 100) && in(a + b + c + d, -90, 100) &&
         in(a + b + c + 2 * d, -90, 100);
}

// For fixed G, h1 and D exponent fields, the u fields window_ok accepts form
// one interval; u_range packs it as {lo | hi << 16, zero_ok} (zero_ok: an
// all-zero u is fine, i.e. nothing is non-finite), u_in_range tests it.
AX_HD void u_range(int fg, int fh, int fd, unsigned &packed, unsigned &zero_ok) {
  int lo = 1, hi = 0;  // empty
  zero_ok = (fg != 2047 && fh != 2047 && fd != 2047) ? 1u : 0u;
  if (zero_ok) {
    if (fg == 0 || fh == 0 || fd == 0) {
      lo = 1;
      hi = 2046;  // a zero factor: any finite u
    } else {
      for (int fu = 1; fu <= 2046; ++fu) {  // the window is an interval in fu
        if (window_ok(fu, fg, fh, fd)) {
          if (lo > hi) lo = fu;
          hi = fu;
        }
      }
    }
  }
  packed = (unsigned)lo | ((unsigned)hi << 16);
}
AX_HD bool u_in_range(uint2 r, int fu) {
  if (fu == 0) return r.y != 0u;
  return fu >= (int)(r.x & 0xFFFFu) && fu <= (int)(r.x >> 16);
}

// Per-block record: per element the three exponent keys (u, G, h1), plus the
// largest |D| key and the largest centro-antisymmetry defect of the matrices.
constexpr int kMaxElems = 64;

// The fp64 geometry arrays an element falls back to (kernels that read a
// prepared copy keep them for that).
struct RawGeo {
  const double *h1, *g11, *g22, *g33, *g12, *g13, *g23;
};
struct Record {
  unsigned ex[kMaxElems][3];
  unsigned long long dmax, ddev;  // fp64 bit patterns of non-negative values
};

AX_D void clear(Record &r, int nel) {
  for (int q = threadIdx.x; q < nel * 3; q += blockDim.x) r.ex[q / 3][q % 3] = 0u;
  if (threadIdx.x == 0) {
    r.dmax = 0ull;
    r.ddev = 0ull;
  }
}
AX_D unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
// |D| entries; the defect |D[i][l] + D[N-i][N-l]| of each mirrored pair
AX_D void note_d(Record &r, double a) { atomicMax(&r.dmax, abs_bits(a)); }
AX_D void note_pair(Record &r, double a, double mirrored) {
  atomicMax(&r.dmax, abs_bits(a) > abs_bits(mirrored) ? abs_bits(a) : abs_bits(mirrored));
  atomicMax(&r.ddev, abs_bits(__dadd_rn(a, mirrored)));
}
// field of the largest |D|
AX_D int d_field(const Record &r) {
  return (int)((r.dmax >> 52) & 0x7FFull);
}
// matrices centro-antisymmetric to 2^-46 of their largest entry (the split of
// the even-odd kernels reads only half the rows; a defect this small changes
// w by less than the double-float rounding)
AX_D bool centro_ok(const Record &r) {
  const double dmax = __longlong_as_double((long long)r.dmax);
  const double dev = __longlong_as_double((long long)r.ddev);
  return dev <= dmax * 0x1p-46;
}
AX_D bool elem_ok(const Record &r, int le) {
  return window_ok(field(r.ex[le][0]), field(r.ex[le][1]), field(r.ex[le][2]), d_field(r));
}

// w_e = D^T (h1 G (D u_e)) of one element with fp64 units, in the loop order
// of Listing 2 (reference gradient, pointwise h1 G, transposed sum).  Run by
// the `nt` threads of the element (rank `r`); `sync()` synchronises at least
// those threads.  `scr` holds 3 lx^3 doubles of shared memory.  u is read with
// coherent loads (a solver kernel may have written it earlier in the same
// launch).  dot (optional): adds this thread's share of u . w.  Threads with
// `on` false only take part in the two barriers.
template <int LX, class Sync>
__device__ __noinline__ void element_f64(bool on, double *__restrict__ w, const double *u, const double *__restrict__ dx,
                      const double *__restrict__ dy, const double *__restrict__ dz,
                      const double *__restrict__ dxt, const double *__restrict__ dyt,
                      const double *__restrict__ dzt, const double *__restrict__ h1,
                      const double *__restrict__ g11, const double *__restrict__ g22,
                      const double *__restrict__ g33, const double *__restrict__ g12,
                      const double *__restrict__ g13, const double *__restrict__ g23,
                      size_t eb, double *scr, int r, int nt, Sync sync, double *dot) {
  constexpr int N2 = LX * LX, N3 = N2 * LX;
  double *sr = scr, *ss = scr + N3, *st = scr + 2 * N3;
  for (int p = r; on && p < N3; p += nt) {
    const int i = p % LX, j = (p / LX) % LX, k = p / N2;
    double ur = 0.0, us = 0.0, ut = 0.0;
#pragma unroll 4
    for (int l = 0; l < LX; ++l) {
      ur = __fma_rn(__ldg(dx + l * LX + i), u[eb + (k * LX + j) * LX + l], ur);
      us = __fma_rn(__ldg(dy + l * LX + j), u[eb + (k * LX + l) * LX + i], us);
      ut = __fma_rn(__ldg(dz + l * LX + k), u[eb + (l * LX + j) * LX + i], ut);
    }
    const size_t q = eb + p;
    const double a11 = __ldg(g11 + q), a22 = __ldg(g22 + q), a33 = __ldg(g33 + q);
    const double a12 = __ldg(g12 + q), a13 = __ldg(g13 + q), a23 = __ldg(g23 + q);
    const double hh = __ldg(h1 + q);
    sr[p] = hh * (a11 * ur + a12 * us + a13 * ut);
    ss[p] = hh * (a12 * ur + a22 * us + a23 * ut);
    st[p] = hh * (a13 * ur + a23 * us + a33 * ut);
  }
  sync();
  for (int p = r; on && p < N3; p += nt) {
    const int i = p % LX, j = (p / LX) % LX, k = p / N2;
    double acc = 0.0;
#pragma unroll 4
    for (int l = 0; l < LX; ++l) {
      acc = __fma_rn(__ldg(dxt + l * LX + i), sr[(k * LX + j) * LX + l], acc);
      acc = __fma_rn(__ldg(dyt + l * LX + j), ss[(k * LX + l) * LX + i], acc);
      acc = __fma_rn(__ldg(dzt + l * LX + k), st[(l * LX + j) * LX + i], acc);
    }
    w[eb + p] = acc;
    if (dot) *dot = __fma_rn(u[eb + p], acc, *dot);
  }
  sync();  // the scratch is reused by the caller
}

}  // namespace guard

// Rewrites per-element geometry keys {G, h1} in place into the u range of
// guard::u_range for matrices whose largest entry has exponent field fd.
__global__ void geo_urange_kernel(unsigned *__restrict__ keys, int nelv, int fd);

// Exponent keys of each element's fp64 geometry: keys[2e] over g11..g23,
// keys[2e+1] over h1 (one warp per element; 8 elements per 256-thread block).
__global__ void geo_keys_kernel(unsigned *__restrict__ keys, const double *__restrict__ h1,
                                const double *__restrict__ g11, const double *__restrict__ g22,
                                const double *__restrict__ g33, const double *__restrict__ g12,
                                const double *__restrict__ g13, const double *__restrict__ g23,
                                int nelv, int n3);

}  // namespace ax
