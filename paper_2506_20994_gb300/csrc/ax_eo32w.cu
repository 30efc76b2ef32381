// Host side of the warp-per-element operator (ax_eo32w.cuh): bf16 geometry,
// u in bf16 or fp32, lx = 8, fp32 w.
#include <algorithm>
#include <atomic>

#include "ax_eo32w.cuh"
#include "dispatch.h"

namespace ax {
namespace e32w {

// Resident CTAs of one variant times the SMs (cached per device; the
// shared-memory limit is raised on first use).
template <class SU, class SG, bool DOT, bool PUPD>
int grid() {
  using C = Cfg<SU, SG, PUPD>;
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    (void)cudaGetLastError();
    return 0;
  }
  int g = cache[dev].load(std::memory_order_acquire);
  if (g > 0) return g;
  auto kern = ax_eo32w_kernel<SU, SG, DOT, PUPD>;
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

// CTAs (and dot partials) of a launch over nelv elements: every variant of a
// storage pair launches the same grid, so that a solver sizes its partials
// once.
template <class SU, class SG>
int blocks(long long nelv) {
  int g = std::min(grid<SU, SG, true, false>(), grid<SU, SG, false, false>());
  if constexpr (std::is_same_v<SU, float>) g = std::min(g, grid<SU, SG, true, true>());
  const long long need = (std::max(nelv, 1LL) + kWarps - 1) / kWarps;
  return g <= 0 ? 0 : (int)std::min<long long>(g, need);
}

template <class SU, class SG>
int launch(float *w, const SU *u, const float *dx, const float *dxt, const SG *const g[7],
           int nelv, int *err, double *dotp, cudaStream_t st, const E32Upd *up) {
  const int nb = blocks<SU, SG>(nelv);
  if (nb <= 0) return AX_ELAUNCH;
  e32::Mesh<SU, SG> m;
  m.w = w;
  m.u = u;
  for (int f = 0; f < 7; ++f) m.g[f] = g[f];
  m.dx = dx;
  m.dxt = dxt;
  const E32Upd none{};
  constexpr int NTB = kWarps * 32;
  if (up) {
    if constexpr (std::is_same_v<SU, float>) {
      if (!dotp || !up->pw || !up->r || !up->minv || !up->beta) return AX_EINVAL;
      ax_eo32w_kernel<SU, SG, true, true>
          <<<nb, NTB, Cfg<SU, SG, true>::SMEM, st>>>(m, nelv, err, dotp, *up);
    } else {
      return AX_EINVAL;
    }
  } else if (dotp) {
    ax_eo32w_kernel<SU, SG, true><<<nb, NTB, Cfg<SU, SG>::SMEM, st>>>(m, nelv, err, dotp, none);
  } else {
    ax_eo32w_kernel<SU, SG, false><<<nb, NTB, Cfg<SU, SG>::SMEM, st>>>(m, nelv, err, dotp, none);
  }
  return launch_status();
}

}  // namespace e32w

int dispatch_eo32w_bf16(float *w, const __nv_bfloat16 *u, const float *dx, const float *dxt,
                        const __nv_bfloat16 *const g[7], int nelv, int *err, double *dotp,
                        cudaStream_t st) {
  return e32w::launch<__nv_bfloat16, __nv_bfloat16>(w, u, dx, dxt, g, nelv, err, dotp, st,
                                                    nullptr);
}

int dispatch_eo32w_f32u_bf16(float *w, const float *u, const float *dx, const float *dxt,
                             const __nv_bfloat16 *const g[7], int nelv, int *err, double *dotp,
                             cudaStream_t st, const E32Upd *up) {
  return e32w::launch<float, __nv_bfloat16>(w, u, dx, dxt, g, nelv, err, dotp, st, up);
}

int eo32w_blocks_bf16(int nelv) { return e32w::blocks<__nv_bfloat16, __nv_bfloat16>(nelv); }
int eo32w_blocks_f32u_bf16(int nelv) { return e32w::blocks<float, __nv_bfloat16>(nelv); }

}  // namespace ax
