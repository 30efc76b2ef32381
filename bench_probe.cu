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
