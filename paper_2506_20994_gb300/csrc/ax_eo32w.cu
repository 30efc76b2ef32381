// Host side of the warp-per-element operator (ax_eo32w.cuh): bf16 u and
// geometry, lx = 8, fp32 w.
#include <algorithm>
#include <atomic>

#include "ax_eo32w.cuh"
#include "dispatch.h"

namespace ax {
namespace e32w {

// Resident CTAs of one variant times the SMs (cached per device; the
// shared-memory limit is raised on first use).
template <class SU, class SG, bool DOT>
int grid() {
  using C = Cfg<SU, SG>;
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return 0;
  }
  int g = cache[dev].load(std::memory_order_acquire);
  if (g > 0) return g;
  auto kern = ax_eo32w_kernel<SU, SG, DOT>;
  int sms = 0, bps = 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kWarps * 32, C::SMEM) !=
          cudaSuccess ||
      bps < 1) {
    (void)cudaGetLastError();
    return 0;
  }
  g = sms * bps;
  cache[dev].store(g, std::memory_order_release);
  return g;
}

template <class SU, class SG>
int blocks(long long nelv) {
  const int g = std::min(grid<SU, SG, true>(), grid<SU, SG, false>());
  const long long need = (std::max(nelv, 1LL) + kWarps - 1) / kWarps;
  return g <= 0 ? 0 : (int)std::min<long long>(g, need);
}

template <class SU, class SG>
int launch(float *w, const SU *u, const float *dx, const float *dxt, const SG *const g[7],
           int nelv, int *err, double *dotp, cudaStream_t st) {
  const int nb = blocks<SU, SG>(nelv);
  if (nb <= 0) return AX_ELAUNCH;
  e32::Mesh<SU, SG> m;
  m.w = w;
  m.u = u;
  for (int f = 0; f < 7; ++f) m.g[f] = g[f];
  m.dx = dx;
  m.dxt = dxt;
  using C = Cfg<SU, SG>;
  if (dotp)
    ax_eo32w_kernel<SU, SG, true><<<nb, kWarps * 32, C::SMEM, st>>>(m, nelv, err, dotp);
  else
    ax_eo32w_kernel<SU, SG, false><<<nb, kWarps * 32, C::SMEM, st>>>(m, nelv, err, dotp);
  return launch_status();
}

}  // namespace e32w

int dispatch_eo32w_bf16(float *w, const __nv_bfloat16 *u, const float *dx, const float *dxt,
                        const __nv_bfloat16 *const g[7], int nelv, int *err, double *dotp,
                        cudaStream_t st) {
  return e32w::launch<__nv_bfloat16, __nv_bfloat16>(w, u, dx, dxt, g, nelv, err, dotp, st);
}

int eo32w_blocks_bf16(int nelv) { return e32w::blocks<__nv_bfloat16, __nv_bfloat16>(nelv); }

}  // namespace ax
