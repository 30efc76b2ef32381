// fp64-accurate element operator of Listing 2 that issues no fp64
// instruction: fp64 inputs are split into double-float pairs with integer
// operations, every contraction and the pointwise metric step run as
// error-free fp32 transformations (df64.cuh), and w is re-assembled into
// fp64 bits.  The schedule is the k-loop one of ax_kstep.cuh (lx*lx threads
// per element, u and the weighted gradient staged in shared memory).
//
// Why: the fp64 pipe of sm_103a issues at a small fraction of the fp32
// rate, so the fp64 operator on fp64 units is bound by fp64 throughput far
// below the HBM roofline; fp32 pairs trade each fp64 FMA for about a dozen
// fp32 operations, which the fp32 pipe issues much faster.
//
// The body is a device function over `nel` (<= epb) consecutive elements
// starting at element e0 of one mesh, so the per-mesh kernel and the
// persistent multi-mesh kernel (batch.cu) share it.  Threads at or above
// epb*lx*lx only take part in the block barriers.
#pragma once

#include "common.cuh"
#include "df64.cuh"
#include "guard.cuh"

namespace ax {

// XYZ: one matrix per direction as in the full signature of Listings 1-2
// (dx, dy, dz forward; dxt, dyt, dzt transposed), six staged matrices;
// otherwise dx and dxt serve all three directions.
template <int LX, bool XYZ = false>
constexpr size_t df64_smem(int epb) {
  return ((XYZ ? 6 : 2) * (size_t)LX * LX + (size_t)epb * 3 * LX * LX * LX) * sizeof(df::df2);
}

template <int LX, bool XYZ = false>
__device__ __forceinline__ void df64_body(double *__restrict__ w, const double *__restrict__ u,
                                          const double *__restrict__ dx,
                                          const double *__restrict__ dxt,
                                          const double *__restrict__ h1,
                                          const double *__restrict__ g11,
                                          const double *__restrict__ g22,
                                          const double *__restrict__ g33,
                                          const double *__restrict__ g12,
                                          const double *__restrict__ g13,
                                          const double *__restrict__ g23, long long e0, int nel,
                                          int epb, unsigned char *smem_raw,
                                          const double *__restrict__ dy = nullptr,
                                          const double *__restrict__ dz = nullptr,
                                          const double *__restrict__ dyt = nullptr,
                                          const double *__restrict__ dzt = nullptr) {
  using namespace df;
  constexpr int N2 = LX * LX;
  constexpr int N3 = LX * N2;
  df2 *sdx = reinterpret_cast<df2 *>(smem_raw);
  df2 *sdxt = sdx + N2;
  // per-direction matrices (the same two unless XYZ)
  df2 *sdy = sdx, *sdz = sdx, *sdyt = sdxt, *sdzt = sdxt;
  df2 *stage = sdxt + N2;
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
  df2 *su = stage + (size_t)le * 3 * N3;
  df2 *swr = su + N3;
  df2 *sws = swr + N3;

  // range record of this block (guard.cuh)
  __shared__ guard::Record rec;
  guard::clear(rec, epb);
  __syncthreads();

  for (int t = threadIdx.x; t < N2; t += blockDim.x) {
    const double a = __ldg(dx + t), at = __ldg(dxt + t);
    guard::note_d(rec, a);
    guard::note_d(rec, at);
    sdx[t] = split(a);
    sdxt[t] = split(at);
    if constexpr (XYZ) {
      const double b = __ldg(dy + t), c = __ldg(dz + t), bt = __ldg(dyt + t), ct = __ldg(dzt + t);
      guard::note_d(rec, b);
      guard::note_d(rec, c);
      guard::note_d(rec, bt);
      guard::note_d(rec, ct);
      sdy[t] = split(b);
      sdz[t] = split(c);
      sdyt[t] = split(bt);
      sdzt[t] = split(ct);
    }
  }
  const bool active = own && le < nel;
  const size_t base = (size_t)(active ? e0 + le : 0) * N3 + p;
  // the geometry is read plane by plane in the k-loop: start all of it towards L2
  if (active && p < 7 && (N3 * sizeof(double)) % 16 == 0) {
    const double *f = p == 0 ? g11 : p == 1 ? g22 : p == 2 ? g33 : p == 3 ? g12 : p == 4 ? g13
                    : p == 5 ? g23 : h1;
    prefetch_l2(f + (base - p), (unsigned)(N3 * sizeof(double)));
  }

  df2 uk[LX];
  unsigned ukey = 0u, gkey = 0u, hkey = 0u;  // exponent keys of u, G, h1
  if (own) {
#pragma unroll
    for (int k = 0; k < LX; ++k) {
      const double x = active ? __ldg(u + base + (size_t)k * N2) : 0.0;
      ukey = max(ukey, guard::key(x));
      uk[k] = split(x);
      su[k * N2 + p] = uk[k];
    }
    if (active) atomicMax(&rec.ex[le][0], ukey);
  }
  __syncthreads();

  acc wacc[LX];
  if (own) {
#pragma unroll
    for (int k = 0; k < LX; ++k) {
      acc ar = prod(sdx[i], su[k * N2 + j * LX]);
      acc as = prod(sdy[j], su[k * N2 + i]);
      acc at = prod(sdz[k], uk[0]);
#pragma unroll
      for (int l = 1; l < LX; ++l) {
        mac(ar, sdx[l * LX + i], su[k * N2 + j * LX + l]);
        mac(as, sdy[l * LX + j], su[k * N2 + l * LX + i]);
        mac(at, sdz[l * LX + k], uk[l]);
      }
      const df2 ur = result(ar), us = result(as), ut = result(at);
      df2 wr{0.f, 0.f}, ws{0.f, 0.f}, wt{0.f, 0.f};
      if (active) {
        const size_t q = base + (size_t)k * N2;
        const double v11 = __ldg(g11 + q), v22 = __ldg(g22 + q), v33 = __ldg(g33 + q);
        const double v12 = __ldg(g12 + q), v13 = __ldg(g13 + q), v23 = __ldg(g23 + q);
        const double vh = __ldg(h1 + q);
        gkey = max(gkey, max(max(guard::key(v11), guard::key(v22)),
                             max(max(guard::key(v33), guard::key(v12)),
                                 max(guard::key(v13), guard::key(v23)))));
        hkey = max(hkey, guard::key(vh));
        const df2 a11 = split(v11), a22 = split(v22);
        const df2 a33 = split(v33), a12 = split(v12);
        const df2 a13 = split(v13), a23 = split(v23);
        const df2 hh = split(vh);
        acc a = prod(a11, ur);
        mac(a, a12, us);
        mac(a, a13, ut);
        wr = mul2(hh, result(a));
        a = prod(a12, ur);
        mac(a, a22, us);
        mac(a, a23, ut);
        ws = mul2(hh, result(a));
        a = prod(a13, ur);
        mac(a, a23, us);
        mac(a, a33, ut);
        wt = mul2(hh, result(a));
      }
      swr[k * N2 + p] = wr;
      sws[k * N2 + p] = ws;
#pragma unroll
      for (int kk = 0; kk < LX; ++kk) {
        if (k == 0)
          wacc[kk] = prod(sdzt[kk], wt);
        else
          mac(wacc[kk], sdzt[k * LX + kk], wt);
      }
    }
    if (active) {
      atomicMax(&rec.ex[le][1], gkey);
      atomicMax(&rec.ex[le][2], hkey);
    }
  }
  __syncthreads();

  // an element outside the double-float range is recomputed with fp64 units
  const bool bad = active && !guard::elem_ok(rec, le);
  if (own) {
#pragma unroll
    for (int k = 0; k < LX; ++k) {
      acc a = wacc[k];
#pragma unroll
      for (int l = 0; l < LX; ++l) {
        mac(a, sdxt[l * LX + i], swr[k * N2 + j * LX + l]);
        mac(a, sdyt[l * LX + j], sws[k * N2 + l * LX + i]);
      }
      const df2 r = result(a);
      if (active && !bad) w[base + (size_t)k * N2] = join(r.hi, r.lo);
    }
  }
  if (__syncthreads_or(bad)) {  // block-uniform; the barrier also frees the scratch
    const double *ddy = XYZ ? dy : dx, *ddz = XYZ ? dz : dx;
    const double *ddyt = XYZ ? dyt : dxt, *ddzt = XYZ ? dzt : dxt;
    guard::element_f64<LX>(bad, w, u, dx, ddy, ddz, dxt, ddyt, ddzt, h1, g11, g22, g33, g12, g13,
                           g23, (size_t)(active ? e0 + le : 0) * N3,
                           reinterpret_cast<double *>(su), own ? p : 0, N2,
                           [] { __syncthreads(); }, nullptr);
  }
}

template <int LX>
__global__ void __launch_bounds__(256)
ax_df64_kernel(double *__restrict__ w, const double *__restrict__ u,
               const double *__restrict__ dx, const double *__restrict__ dxt,
               const double *__restrict__ h1, const double *__restrict__ g11,
               const double *__restrict__ g22, const double *__restrict__ g33,
               const double *__restrict__ g12, const double *__restrict__ g13,
               const double *__restrict__ g23, int nelv, int epb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long e0 = (long long)blockIdx.x * epb;
  const long long left = nelv - e0;
  const int nel = left < epb ? (int)left : epb;
  df64_body<LX>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, e0, nel, epb, smem_raw);
}

template <int LX>
int launch_df64(double *w, const double *u, const double *dx, const double *dxt,
                const double *h1, const double *g11, const double *g22, const double *g33,
                const double *g12, const double *g13, const double *g23, int nelv, int epb,
                cudaStream_t stream) {
  if (epb <= 0) epb = 256 / (LX * LX) < 1 ? 1 : 256 / (LX * LX);
  if (epb * LX * LX > 256) return AX_EINVAL;
  const size_t smem = df64_smem<LX>(epb);
  auto kern = ax_df64_kernel<LX>;
  static std::atomic<size_t> granted[kMaxDevices];
  if (!grant_smem(kern, smem, granted)) return AX_EINVAL;
  const unsigned grid = (unsigned)((nelv + epb - 1) / epb);
  kern<<<grid, epb * LX * LX, smem, stream>>>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23,
                                              nelv, epb);
  return launch_status();
}

}  // namespace ax
