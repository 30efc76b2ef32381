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

}  // namespace ax
