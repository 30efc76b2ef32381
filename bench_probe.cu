// Benchmark tooling, not part of libaxhelm.so: bench_extras.py compiles this
// file on its own (nvcc -shared) and loads it to report, beside the operator
// timings, the per-SM, per-clock rates of the three multiply-add forms the
// operator kernels are built from (fp64 on the fp64 pipe, fp32, and the
// packed f32x2 form of the double-float kernels).  These rates decide the
// design: an fp64-unit operator is bound by the first, the double-float
// kernels by the other two.
//
// Each thread runs kChains independent multiply-add chains of `iters` steps
// (independent so the pipe, not the latency, limits); every block records
// the SM it ran on and its start and end clocks (the SM's own counter).  Per
// SM: ops of the blocks that ran there / (last end - first start); the probe
// reports the median over SMs, so an uneven placement of blocks does not bias
// it.  The compiler may issue independent fp32 chains as packed f32x2
// instructions, so the fp32 figure is the rate the compiler reaches for
// plain fp32 code.  Results go to a small sink so nothing is optimised away.
#include <algorithm>
#include <vector>

#include "paper_2506_20994_gb300/csrc/common.cuh"
#include "paper_2506_20994_gb300/csrc/df64.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <int KIND>  // 0: fp64 fma, 1: fp32 fma, 2: packed fma.rn.f32x2
__global__ void __launch_bounds__(kThreads) probe_kernel(int iters, double seed,
                                                         long long *stamps, double *sink) {
  __syncthreads();
  long long t0 = clock64();
  double out = 0.0;
  if constexpr (KIND == 0) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + c;
    const double m = 1.0 - 1e-9, b = 1e-9;
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = __fma_rn(a[c], m, b);
#pragma unroll
    for (int c = 0; c < kChains; ++c) out += a[c];
  } else if constexpr (KIND == 1) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (float)seed + c;
    const float m = 1.0f - 1e-6f, b = 1e-6f;
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = __fmaf_rn(a[c], m, b);
#pragma unroll
    for (int c = 0; c < kChains; ++c) out += a[c];
  } else {
    unsigned long long a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = ax::df::pk((float)seed + c, (float)seed - c);
    const unsigned long long m = ax::df::pk(1.0f - 1e-6f, 1.0f - 1e-6f);
    const unsigned long long b = ax::df::pk(1e-6f, 1e-6f);
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = ax::df::fma2(a[c], m, b);
#pragma unroll
    for (int c = 0; c < kChains; ++c) out += ax::df::lx_(a[c]) + ax::df::ly_(a[c]);
  }
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = out;
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) {
    unsigned sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    stamps[3 * blockIdx.x] = (long long)sm;
    stamps[3 * blockIdx.x + 1] = t0;
    stamps[3 * blockIdx.x + 2] = t1;
  }
}

template <int KIND>
int run_probe(int sms, int blocks_per_sm, int iters, long long *d_stamps, double *d_sink,
              double *rate, cudaStream_t st) {
  const int grid = sms * blocks_per_sm;
  probe_kernel<KIND><<<grid, kThreads, 0, st>>>(iters, 1.0, d_stamps, d_sink);  // warm-up
  probe_kernel<KIND><<<grid, kThreads, 0, st>>>(iters, 1.0, d_stamps, d_sink);
  if (ax::launch_status() != AX_OK) return AX_ELAUNCH;
  std::vector<long long> h((size_t)grid * 3);
  if (cudaMemcpyAsync(h.data(), d_stamps, sizeof(long long) * h.size(), cudaMemcpyDeviceToHost,
                      st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
  // multiply-adds per block: a packed instruction does two per thread
  const double per_block = (double)iters * kChains * (KIND == 2 ? 2 : 1) * kThreads;
  std::vector<int> count(sms, 0);
  std::vector<long long> first(sms, 0), last(sms, 0);
  for (int b = 0; b < grid; ++b) {
    const long long sm = h[3 * b];
    if (sm < 0 || sm >= sms) continue;
    if (count[sm] == 0 || h[3 * b + 1] < first[sm]) first[sm] = h[3 * b + 1];
    if (count[sm] == 0 || h[3 * b + 2] > last[sm]) last[sm] = h[3 * b + 2];
    ++count[sm];
  }
  std::vector<double> per_sm;
  for (int sm = 0; sm < sms; ++sm)
    if (count[sm] > 0 && last[sm] > first[sm])
      per_sm.push_back(per_block * count[sm] / (double)(last[sm] - first[sm]));
  if (per_sm.empty()) return AX_ELAUNCH;
  std::sort(per_sm.begin(), per_sm.end());
  *rate = per_sm[per_sm.size() / 2];
  return AX_OK;
}

}  // namespace

// rates[0] fp64, rates[1] fp32, rates[2] packed f32x2 multiply-adds per SM
// and clock on the current device (4 x 256 threads per SM, median over SMs);
// allocates a small scratch buffer, synchronises `stream`.
extern "C" int bench_probe_rates(double *rates, void *stream) {
  if (!rates) return AX_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
  constexpr int kBlocksPerSm = 4;  // 1024 threads per SM, all resident at once
  const int grid = sms * kBlocksPerSm;
  long long *d_cycles = nullptr;
  double *d_sink = nullptr;
  if (cudaMalloc((void **)&d_cycles, sizeof(long long) * 3 * grid) != cudaSuccess ||
      cudaMalloc((void **)&d_sink, sizeof(double) * grid * kThreads) != cudaSuccess) {
    (void)cudaGetLastError();
    cudaFree(d_cycles);
    return AX_ENOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int rc = run_probe<0>(sms, kBlocksPerSm, 256, d_cycles, d_sink, &rates[0], st);
  if (rc == AX_OK) rc = run_probe<1>(sms, kBlocksPerSm, 8192, d_cycles, d_sink, &rates[1], st);
  if (rc == AX_OK) rc = run_probe<2>(sms, kBlocksPerSm, 8192, d_cycles, d_sink, &rates[2], st);
  cudaStreamSynchronize(st);
  cudaFree(d_cycles);
  cudaFree(d_sink);
  return rc;
}

// ---------------------------------------------------------------------------
// Prototype for the fp64-accurate on-the-fly trilinear geometry (not a
// library path): the cost of computing G = (w_i w_j w_k / det J) adj(J)
// adj(J)^T per point from an element's 8 corners in double-float arithmetic,
// in the k-loop schedule of the fp32 trilinear kernel (the t-column of J
// fixed along a thread's k-walk, the r- and s-columns linear in k).  Timing
// this kernel alone gives the work the fp64 operator would add per point in
// exchange for the 56 bytes of stored geometry it would stop reading.  Each
// thread folds its G values into a checksum (so nothing is optimised away);
// the G of element 0 is written out in fp64 for a parity check.
namespace {

using ax::df::df2;

__device__ __forceinline__ df2 dsplit(double x) {
  df2 o;
  o.hi = (float)x;
  o.lo = (float)(x - (double)o.hi);
  return o;
}
__device__ __forceinline__ df2 dnorm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return df2{h, __fsub_rn(e, __fsub_rn(h, s))};
}
// TwoProduct of the heads, cross terms in the tail
__device__ __forceinline__ df2 dmul(df2 a, df2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dnorm(p, e);
}
// TwoSum of the heads, tails added
__device__ __forceinline__ df2 dadd(df2 a, df2 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bp = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(b.hi, bp));
  return dnorm(s, __fadd_rn(err, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df2 dneg(df2 a) { return df2{-a.hi, -a.lo}; }
__device__ __forceinline__ df2 dfms(df2 a, df2 b, df2 c, df2 d) {  // a b - c d
  return dadd(dmul(a, b), dneg(dmul(c, d)));
}
// a / b: reciprocal of the head, one correction step on the pair residual
__device__ __forceinline__ df2 ddiv(df2 a, df2 b) {
  const float r = __frcp_rn(b.hi);
  const float q1 = __fmul_rn(a.hi, r);
  const df2 res = dadd(a, dneg(dmul(b, df2{q1, 0.f})));
  const float q2 = __fmul_rn(res.hi, r);
  return dnorm(q1, q2);
}

template <int LX>
__global__ void __launch_bounds__(LX * LX) probe_tri_df_kernel(const double *__restrict__ corners,
                                                               const double *__restrict__ xi,
                                                               const double *__restrict__ wq,
                                                               int nelv, double *__restrict__ sink,
                                                               double *__restrict__ g0) {
  constexpr int N2 = LX * LX;
  __shared__ df2 cf[36], phi0[LX], phi1[LX], sw[LX];
  const int p = (int)threadIdx.x, i = p % LX, j = p / LX;
  if (p < LX) {
    phi0[p] = dsplit(0.5 * (1.0 - xi[p]));
    phi1[p] = dsplit(0.5 * (1.0 + xi[p]));
    sw[p] = dsplit(wq[p]);
  }
  float check = 0.f;
  for (long long e = blockIdx.x; e < nelv; e += gridDim.x) {
    __syncthreads();
    for (int t = p; t < 36; t += N2) {  // half edge vectors, as the fp32 kernel's
      const int dir = t / 12, d = (t / 4) % 3, q = t % 4, hi = q >> 1, lo = q & 1;
      int c0, c1;
      if (dir == 0) {
        c0 = (hi * 2 + lo) * 2;
        c1 = c0 + 1;
      } else if (dir == 1) {
        c0 = (hi * 2) * 2 + lo;
        c1 = c0 + 2;
      } else {
        c0 = hi * 2 + lo;
        c1 = c0 + 4;
      }
      const double *x = corners + (size_t)e * 24;
      cf[t] = dsplit(0.5 * (x[c1 * 3 + d] - x[c0 * 3 + d]));
    }
    __syncthreads();
    const df2 pj0 = phi0[j], pj1 = phi1[j], pi0 = phi0[i], pi1 = phi1[i];
    df2 P[3][2], Q[3][2], Jt[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        P[d][c] = dadd(dmul(cf[d * 4 + c * 2 + 1], pj1), dmul(cf[d * 4 + c * 2], pj0));
        Q[d][c] = dadd(dmul(cf[12 + d * 4 + c * 2 + 1], pi1), dmul(cf[12 + d * 4 + c * 2], pi0));
      }
      const df2 b0 = dadd(dmul(cf[24 + d * 4 + 1], pi1), dmul(cf[24 + d * 4], pi0));
      const df2 b1 = dadd(dmul(cf[24 + d * 4 + 3], pi1), dmul(cf[24 + d * 4 + 2], pi0));
      Jt[d] = dadd(dmul(b1, pj1), dmul(b0, pj0));
    }
    const df2 wij = dmul(sw[i], sw[j]);
#pragma unroll 2
    for (int k = 0; k < LX; ++k) {
      const df2 z0 = phi0[k], z1 = phi1[k];
      const df2 a = dadd(dmul(P[0][1], z1), dmul(P[0][0], z0));
      const df2 b = dadd(dmul(Q[0][1], z1), dmul(Q[0][0], z0));
      const df2 c = Jt[0];
      const df2 d = dadd(dmul(P[1][1], z1), dmul(P[1][0], z0));
      const df2 f = dadd(dmul(Q[1][1], z1), dmul(Q[1][0], z0));
      const df2 g = Jt[1];
      const df2 h = dadd(dmul(P[2][1], z1), dmul(P[2][0], z0));
      const df2 m = dadd(dmul(Q[2][1], z1), dmul(Q[2][0], z0));
      const df2 n = Jt[2];
      const df2 A00 = dfms(f, n, g, m), A01 = dfms(c, m, b, n), A02 = dfms(b, g, c, f);
      const df2 A10 = dfms(g, h, d, n), A11 = dfms(a, n, c, h), A12 = dfms(c, d, a, g);
      const df2 A20 = dfms(d, m, f, h), A21 = dfms(b, h, a, m), A22 = dfms(a, f, b, d);
      const df2 det = dadd(dmul(a, A00), dadd(dmul(b, A10), dmul(c, A20)));
      const df2 s = ddiv(dmul(wij, sw[k]), det);
      auto dot3 = [](df2 x0, df2 x1, df2 x2, df2 y0, df2 y1, df2 y2) {
        return dadd(dmul(x0, y0), dadd(dmul(x1, y1), dmul(x2, y2)));
      };
      const df2 G[6] = {dmul(s, dot3(A00, A01, A02, A00, A01, A02)),
                        dmul(s, dot3(A10, A11, A12, A10, A11, A12)),
                        dmul(s, dot3(A20, A21, A22, A20, A21, A22)),
                        dmul(s, dot3(A00, A01, A02, A10, A11, A12)),
                        dmul(s, dot3(A00, A01, A02, A20, A21, A22)),
                        dmul(s, dot3(A10, A11, A12, A20, A21, A22))};
#pragma unroll
      for (int q = 0; q < 6; ++q) check += G[q].hi;
      if (e == 0 && g0) {
#pragma unroll
        for (int q = 0; q < 6; ++q)
          g0[(size_t)q * LX * N2 + (size_t)k * N2 + p] = (double)G[q].hi + (double)G[q].lo;
      }
    }
  }
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = (double)check;
}

}  // namespace

// Times the prototype at lx = 8 over nelv elements (corners: nelv x 24
// fp64, device; xi, wq: the 8 GLL nodes and weights, device): *ms = average
// kernel time over `reps` launches after one warm-up; g0 (device, 6 x 512
// fp64, may be null) receives element 0's G (g11, g22, g33, g12, g13, g23).
// Allocates a small sink buffer; synchronises `stream`.
extern "C" int bench_probe_tri_df(const double *corners, const double *xi, const double *wq,
                                  int nelv, int reps, double *g0, float *ms, void *stream) {
  if (!corners || !xi || !wq || !ms || nelv <= 0 || reps < 1) return AX_EINVAL;
  int dev = 0, sms = 0, bps = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, probe_tri_df_kernel<8>, 64, 0) !=
          cudaSuccess ||
      bps < 1) {
    (void)cudaGetLastError();
    return AX_ELAUNCH;
  }
  const int grid = std::min<long long>((long long)sms * bps, nelv);
  double *sink = nullptr;
  if (cudaMalloc((void **)&sink, sizeof(double) * grid * 64) != cudaSuccess) {
    (void)cudaGetLastError();
    return AX_ENOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  probe_tri_df_kernel<8><<<grid, 64, 0, st>>>(corners, xi, wq, nelv, sink, g0);
  cudaEventRecord(e0, st);
  for (int r = 0; r < reps; ++r)
    probe_tri_df_kernel<8><<<grid, 64, 0, st>>>(corners, xi, wq, nelv, sink, nullptr);
  cudaEventRecord(e1, st);
  int rc = cudaEventSynchronize(e1) == cudaSuccess ? AX_OK : AX_ELAUNCH;
  float t = 0.f;
  if (rc == AX_OK) cudaEventElapsedTime(&t, e0, e1);
  *ms = t / reps;
  if (ax::launch_status() != AX_OK) rc = AX_ELAUNCH;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  return rc;
}
