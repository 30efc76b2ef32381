// Instantiations of the even-odd double-float element operator (even lx).
#include "ax_df64_eo.cuh"
#include "dispatch.h"

namespace ax {

int dispatch_df64eo(int lx, double *w, const double *u, const double *dx, const double *dxt,
                    const double *h1, const double *g11, const double *g22, const double *g33,
                    const double *g12, const double *g13, const double *g23, int nelv, int epb,
                    cudaStream_t st) {
  switch (lx) {
#define AX_CASE(L)                                                                             \
  case L:                                                                                      \
    return launch_df64eo<L>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, nelv, epb, st);
    AX_CASE(4) AX_CASE(6) AX_CASE(8) AX_CASE(10) AX_CASE(12)
#undef AX_CASE
    default:
      return AX_EINVAL;
  }
}

int dispatch_df64eo_prep(int lx, double *w, const double *u, const double *dx,
                         const double *dxt, const df::dd2 *gp, const guard::RawGeo &raw,
                         int nelv, int epb, cudaStream_t st, double *dotp, double *pw, const double *r_in,
                         const double *minv_in, const double *beta_p, const double *corr_in,
                         const int *use_corr_p) {
  switch (lx) {
#define AX_CASE(L)                                                                             \
  case L:                                                                                      \
    return launch_df64eo_prep<L>(w, u, dx, dxt, gp, raw, nelv, epb, st, dotp, pw, r_in,      \
                                 minv_in, beta_p, corr_in, use_corr_p);
    AX_CASE(4) AX_CASE(6) AX_CASE(8) AX_CASE(10) AX_CASE(12)
#undef AX_CASE
    default:
      return AX_EINVAL;
  }
}

__global__ void geo_keys_kernel(unsigned *__restrict__ keys, const double *__restrict__ h1,
                                const double *__restrict__ g11, const double *__restrict__ g22,
                                const double *__restrict__ g33, const double *__restrict__ g12,
                                const double *__restrict__ g13, const double *__restrict__ g23,
                                int nelv, int n3) {
  const int lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (e >= nelv) return;
  const size_t b = (size_t)e * n3;
  unsigned kg = 0u, kh = 0u;
  for (int p = lane; p < n3; p += 32) {
    const size_t q = b + p;
    kg = max(kg, max(max(guard::key(g11[q]), guard::key(g22[q])),
                     max(max(guard::key(g33[q]), guard::key(g12[q])),
                         max(guard::key(g13[q]), guard::key(g23[q])))));
    kh = max(kh, guard::key(h1[q]));
  }
  kg = __reduce_max_sync(0xffffffffu, kg);
  kh = __reduce_max_sync(0xffffffffu, kh);
  if (lane == 0) {
    keys[2 * e] = kg;
    keys[2 * e + 1] = kh;
  }
}

int df64eo_prep_blocks(int lx, int nelv) {
  switch (lx) {
    case 4: return prep_blocks<4>(nelv, 0);
    case 6: return prep_blocks<6>(nelv, 0);
    case 8: return prep_blocks<8>(nelv, 0);
    case 10: return prep_blocks<10>(nelv, 0);
    case 12: return prep_blocks<12>(nelv, 0);
    default: return 0;
  }
}

int dispatch_eo_prepare(int lx, df::dd2 *gp, const double *h1, const double *g11,
                        const double *g22, const double *g33, const double *g12,
                        const double *g13, const double *g23, int nelv, int fmask,
                        cudaStream_t st) {
  switch (lx) {
#define AX_CASE(L)                                                                             \
  case L:                                                                                      \
    return launch_eo_prepare<L>(gp, h1, g11, g22, g33, g12, g13, g23, nelv, fmask, st);
    AX_CASE(4) AX_CASE(6) AX_CASE(8) AX_CASE(10) AX_CASE(12)
#undef AX_CASE
    default:
      return AX_EINVAL;
  }
}

}  // namespace ax
