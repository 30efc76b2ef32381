// The element operator of Listing 2 (Sec. "The Kernel Expressed in DaCe")
// with one arithmetic type T throughout: fp64 on the fp64 units, or fp32 for
// the fp32/bf16 storage modes.
//
// Schedule: the two element maps of Listing 2 fused into one kernel, with u
// and the 1-D matrices kept in shared memory (the paper's "fusion, tiling
// and shared memory" step) - but laid out for sm_103a rather than as the
// paper's lx^3-thread blocks:
//   * a block holds `epb` elements, each served by lx*lx threads, thread
//     (j, i) of an element walking k = 0..lx-1 (a k-loop), so that every
//     global load and store of a k-plane is one contiguous lx*lx run;
//   * u_e is staged in shared memory once; the t-derivative uses the
//     thread's own column of u held in registers;
//   * the t-part of the transposed sum is accumulated in registers during
//     the k-loop; the r- and s-parts read the weighted gradient back from
//     shared memory after one block barrier.
// Algorithmic traffic per element: u, h1, six G factors read and w written
// once (9 * lx^3 values).  The body works on `nel` (<= epb) consecutive
// elements from e0, so the persistent multi-mesh kernel (batch.cu) reuses it.
#pragma once

#include "common.cuh"

namespace ax {

// Bulk L2 prefetch of an element's geometry at the start of the element.
constexpr bool kPrefetchGeometry = true;

AX_D double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
AX_D float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
AX_D float4 row4(const float *r, int q) { return reinterpret_cast<const float4 *>(r)[q]; }

// The single-mesh kernel's row-table form (VEC in kstep_body): fp32
// arithmetic and lx divisible by 4.  Rows padded to RS floats so that the
// 16-byte loads of different rows fall in different banks.
template <int LX, typename T>
constexpr bool kstep_vec() {
  return sizeof(T) == 4 && LX % 4 == 0;
}
template <int LX, bool VEC>
constexpr int kstep_rs() {
  return VEC && LX % 8 == 0 ? LX + 4 : LX;
}

// AHEAD: geometry loads one k-plane ahead (measured faster for the
// single-mesh fp32-storage kernel only).
// XYZ: one matrix per direction (dx, dy, dz forward; dxt, dyt, dzt
// transposed) as in the full signature of Listings 1-2; otherwise dx and
// dxt serve all three directions.
// VEC (fp32 arithmetic, lx divisible by 4, one matrix pair): the matrices
// are staged as row tables padded to RS floats (kstep_rs), so every
// contraction reads its matrix row, and the r-lines of u and wr, as 16-byte
// loads; a quarter of the shared-memory load instructions of the scalar form
// for those operands.  Same summation order as the scalar form.
template <int LX, typename SU, typename S, typename T, typename W, bool AHEAD = false,
          bool XYZ = false, bool VEC = false>
__device__ __forceinline__ void kstep_body(W *__restrict__ w, const SU *__restrict__ u,
                                           const T *__restrict__ dx, const T *__restrict__ dxt,
                                           const S *__restrict__ h1, const S *__restrict__ g11,
                                           const S *__restrict__ g22, const S *__restrict__ g33,
                                           const S *__restrict__ g12, const S *__restrict__ g13,
                                           const S *__restrict__ g23, long long e0, int nel,
                                           int epb, unsigned char *smem_raw,
                                           double *__restrict__ dotp = nullptr,
                                           const T *__restrict__ dy = nullptr,
                                           const T *__restrict__ dz = nullptr,
                                           const T *__restrict__ dyt = nullptr,
                                           const T *__restrict__ dzt = nullptr) {
  constexpr int N2 = LX * LX;
  constexpr int N3 = LX * N2;
  static_assert(!VEC || (sizeof(T) == 4 && LX % 4 == 0 && !XYZ), "VEC: fp32, lx % 4 == 0");
  constexpr int RS = kstep_rs<LX, VEC>();
  T *sdx = reinterpret_cast<T *>(smem_raw);
  T *sdxt = sdx + N2;
  T *sdy = sdx, *sdz = sdx, *sdyt = sdxt, *sdzt = sdxt;
  T *stage = sdxt + N2;
  // VEC tables: Fd[a][l] = dx[l*lx + a], Bd[a][l] = dxt[l*lx + a],
  // Td[a][b] = dxt[a*lx + b]
  T *Fd = sdx, *Bd = sdx, *Td = sdx;
  if constexpr (VEC) {
    Fd = reinterpret_cast<T *>(smem_raw);
    Bd = Fd + LX * RS;
    Td = Bd + LX * RS;
    stage = Td + LX * RS;
  }
  if constexpr (XYZ) {
    sdy = stage;
    sdz = sdy + N2;
    sdyt = sdz + N2;
    sdzt = sdyt + N2;
    stage = sdzt + N2;
  }
  const bool own = (int)threadIdx.x < epb * N2;
  const int le = own ? (int)threadIdx.x / N2 : 0;
  const int p = (int)threadIdx.x - le * N2;
  const int i = p % LX;
  const int j = p / LX;
  T *su = stage + (size_t)le * 3 * N3;
  T *swr = su + N3;
  T *sws = swr + N3;

  for (int t = threadIdx.x; VEC && t < N2; t += blockDim.x) {
    const int a = t / LX, b = t % LX;
    Fd[b * RS + a] = dx[t];
    Bd[b * RS + a] = dxt[t];
    Td[a * RS + b] = dxt[t];
  }
  for (int t = threadIdx.x; !VEC && t < N2; t += blockDim.x) {
    sdx[t] = dx[t];
    sdxt[t] = dxt[t];
    if constexpr (XYZ) {
      sdy[t] = dy[t];
      sdz[t] = dz[t];
      sdyt[t] = dyt[t];
      sdzt[t] = dzt[t];
    }
  }
  const bool active = own && le < nel;
  const size_t base = (size_t)(active ? e0 + le : 0) * N3 + p;
  // the geometry is read plane by plane in the k-loop: start all of it towards L2
  if (kPrefetchGeometry && active && p < 7 && (N3 * sizeof(S)) % 16 == 0) {
    const S *f = p == 0 ? g11 : p == 1 ? g22 : p == 2 ? g33 : p == 3 ? g12 : p == 4 ? g13
               : p == 5 ? g23 : h1;
    prefetch_l2(f + (base - p), (unsigned)(N3 * sizeof(S)));
  }

  T uk[LX];
  if (own) {
#pragma unroll
    for (int k = 0; k < LX; ++k) {
      uk[k] = active ? ld_cvt<T>(u + base + (size_t)k * N2) : T(0);
      su[k * N2 + p] = uk[k];
    }
  }
  __syncthreads();

  // geometry of one k-plane; with AHEAD loaded one plane ahead of its use so
  // that the loads are in flight during the previous plane's contractions
  constexpr bool kAhead = AHEAD;
  auto load_plane = [&](int k, T (&g)[7]) {
    const size_t q = base + (size_t)k * N2;
    g[0] = ld_cvt<T>(g11 + q);
    g[1] = ld_cvt<T>(g22 + q);
    g[2] = ld_cvt<T>(g33 + q);
    g[3] = ld_cvt<T>(g12 + q);
    g[4] = ld_cvt<T>(g13 + q);
    g[5] = ld_cvt<T>(g23 + q);
    g[6] = ld_cvt<T>(h1 + q);
  };
  T gcur[7], gnext[7];
  if (kAhead && active) load_plane(0, gnext);

  T wacc[LX];
  if (own) {
#pragma unroll
    for (int k = 0; k < LX; ++k) wacc[k] = T(0);
#pragma unroll
    for (int k = 0; k < LX; ++k) {
      if constexpr (kAhead) {
#pragma unroll
        for (int f = 0; f < 7; ++f) gcur[f] = gnext[f];
        if (active && k + 1 < LX) load_plane(k + 1, gnext);
      }
      T ur = T(0), us = T(0), ut = T(0);
      if constexpr (VEC) {
#pragma unroll
        for (int q = 0; q < LX / 4; ++q) {
          const float4 fi = row4(Fd + i * RS, q), fj = row4(Fd + j * RS, q);
          const float4 fk = row4(Fd + k * RS, q), v = row4(su + k * N2 + j * LX, q);
          const T *c = su + k * N2 + 4 * q * LX + i;
          ur = fma_t(fi.x, v.x, ur);
          us = fma_t(fj.x, c[0], us);
          ut = fma_t(fk.x, uk[4 * q], ut);
          ur = fma_t(fi.y, v.y, ur);
          us = fma_t(fj.y, c[LX], us);
          ut = fma_t(fk.y, uk[4 * q + 1], ut);
          ur = fma_t(fi.z, v.z, ur);
          us = fma_t(fj.z, c[2 * LX], us);
          ut = fma_t(fk.z, uk[4 * q + 2], ut);
          ur = fma_t(fi.w, v.w, ur);
          us = fma_t(fj.w, c[3 * LX], us);
          ut = fma_t(fk.w, uk[4 * q + 3], ut);
        }
      } else {
#pragma unroll
        for (int l = 0; l < LX; ++l) {
          ur = fma_t(sdx[l * LX + i], su[k * N2 + j * LX + l], ur);
          us = fma_t(sdy[l * LX + j], su[k * N2 + l * LX + i], us);
          ut = fma_t(sdz[l * LX + k], uk[l], ut);
        }
      }
      T wr = T(0), ws = T(0), wt = T(0);
      if (active) {
        if constexpr (!kAhead) load_plane(k, gcur);
        const T a11 = gcur[0], a22 = gcur[1], a33 = gcur[2];
        const T a12 = gcur[3], a13 = gcur[4], a23 = gcur[5], hh = gcur[6];
        wr = hh * (a11 * ur + a12 * us + a13 * ut);
        ws = hh * (a12 * ur + a22 * us + a23 * ut);
        wt = hh * (a13 * ur + a23 * us + a33 * ut);
      }
      swr[k * N2 + p] = wr;
      sws[k * N2 + p] = ws;
      if constexpr (VEC) {
#pragma unroll
        for (int q = 0; q < LX / 4; ++q) {
          const float4 t4 = row4(Td + k * RS, q);
          wacc[4 * q] = fma_t(t4.x, wt, wacc[4 * q]);
          wacc[4 * q + 1] = fma_t(t4.y, wt, wacc[4 * q + 1]);
          wacc[4 * q + 2] = fma_t(t4.z, wt, wacc[4 * q + 2]);
          wacc[4 * q + 3] = fma_t(t4.w, wt, wacc[4 * q + 3]);
        }
      } else {
#pragma unroll
        for (int kk = 0; kk < LX; ++kk) wacc[kk] = fma_t(sdzt[k * LX + kk], wt, wacc[kk]);
      }
    }
  }
  __syncthreads();

  T dsum = T(0);  // u . w of this thread's column (fused dot, if dotp)
  if (own) {
#pragma unroll
    for (int k = 0; k < LX; ++k) {
      T acc = wacc[k];
      if constexpr (VEC) {
#pragma unroll
        for (int q = 0; q < LX / 4; ++q) {
          const float4 bi = row4(Bd + i * RS, q), bj = row4(Bd + j * RS, q);
          const float4 v = row4(swr + k * N2 + j * LX, q);
          const T *c = sws + k * N2 + 4 * q * LX + i;
          acc = fma_t(bi.x, v.x, acc);
          acc = fma_t(bj.x, c[0], acc);
          acc = fma_t(bi.y, v.y, acc);
          acc = fma_t(bj.y, c[LX], acc);
          acc = fma_t(bi.z, v.z, acc);
          acc = fma_t(bj.z, c[2 * LX], acc);
          acc = fma_t(bi.w, v.w, acc);
          acc = fma_t(bj.w, c[3 * LX], acc);
        }
      } else {
#pragma unroll
        for (int l = 0; l < LX; ++l) {
          acc = fma_t(sdxt[l * LX + i], swr[k * N2 + j * LX + l], acc);
          acc = fma_t(sdyt[l * LX + j], sws[k * N2 + l * LX + i], acc);
        }
      }
      if (active) w[base + (size_t)k * N2] = (W)acc;
      if (dotp) dsum = fma_t(uk[k], acc, dsum);
    }
  }
  if (dotp) {  // one partial per block, fixed order (block-uniform branch)
    __shared__ double red[32];
    double v = (double)dsum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < (int)((blockDim.x + 31) / 32); ++k) t += red[k];
      dotp[blockIdx.x] = t;
    }
  }
}

// DOT: also one partial of sum u . w per block (the CG's <p, Ap> before the
// gather-scatter, see the fused solver loops).
template <int LX, typename SU, typename S, typename T, typename W, bool DOT = false>
__global__ void __launch_bounds__(1024)
ax_kstep_kernel(W *__restrict__ w, const SU *__restrict__ u, const T *__restrict__ dx,
                const T *__restrict__ dxt, const S *__restrict__ h1,
                const S *__restrict__ g11, const S *__restrict__ g22,
                const S *__restrict__ g33, const S *__restrict__ g12,
                const S *__restrict__ g13, const S *__restrict__ g23, int nelv, int epb,
                double *__restrict__ dotp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long e0 = (long long)blockIdx.x * epb;
  const long long left = nelv - e0;
  const int nel = left < epb ? (int)left : epb;
  constexpr bool ahead = sizeof(S) == 4 && sizeof(T) == 4;
  kstep_body<LX, SU, S, T, W, ahead, false, kstep_vec<LX, T>()>(
      w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, e0, nel, epb, smem_raw,
      DOT ? dotp : nullptr);
}

// Shared-memory bytes of one block of the k-loop kernel (VEC: the single-mesh
// kernel's padded matrix tables).
template <int LX, typename T, bool XYZ = false, bool VEC = false>
constexpr size_t kstep_smem(int epb) {
  const size_t tables = VEC ? 3 * (size_t)LX * kstep_rs<LX, VEC>() : (XYZ ? 6 : 2) * (size_t)LX * LX;
  return (tables + (size_t)epb * 3 * LX * LX * LX) * sizeof(T);
}

// Default elements per block: about 256 threads, at least one element.
inline int kstep_default_epb(int lx) {
  int e = 256 / (lx * lx);
  return e < 1 ? 1 : e;
}

// dotp (optional): ceil(nelv / epb) partials of sum u . w, one per block.
template <int LX, typename SU, typename S, typename T, typename W>
int launch_kstep(W *w, const SU *u, const T *dx, const T *dxt, const S *h1, const S *g11,
                 const S *g22, const S *g33, const S *g12, const S *g13, const S *g23,
                 int nelv, int epb, cudaStream_t stream, double *dotp = nullptr) {
  if (epb <= 0) epb = kstep_default_epb(LX);
  if (epb * LX * LX > 1024) return AX_EINVAL;
  const size_t smem = kstep_smem<LX, T, false, kstep_vec<LX, T>()>(epb);
  auto kern = dotp ? ax_kstep_kernel<LX, SU, S, T, W, true> : ax_kstep_kernel<LX, SU, S, T, W>;
  static std::atomic<size_t> granted[2][kMaxDevices];  // per kernel
  if (!grant_smem(kern, smem, granted[dotp != nullptr])) return AX_EINVAL;
  const unsigned grid = (unsigned)((nelv + epb - 1) / epb);
  kern<<<grid, epb * LX * LX, smem, stream>>>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23,
                                              nelv, epb, dotp);
  return launch_status();
}

}  // namespace ax
