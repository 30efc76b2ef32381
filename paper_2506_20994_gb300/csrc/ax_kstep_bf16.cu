// Instantiation of the k-loop element operator for storage __nv_bfloat16, arithmetic float.
#include "ax_kstep.cuh"
#include "dispatch.h"

namespace ax {

int dispatch_kstep_bf16(int lx, float *w, const __nv_bfloat16 *u, const float *dx,
                                     const float *dxt, const __nv_bfloat16 *h1, const __nv_bfloat16 *g11,
                                     const __nv_bfloat16 *g22, const __nv_bfloat16 *g33, const __nv_bfloat16 *g12,
                                     const __nv_bfloat16 *g13, const __nv_bfloat16 *g23, int nelv, int epb,
                                     cudaStream_t st) {
  switch (lx) {
#define AX_CASE(L)                                                                             \
  case L:                                                                                      \
    return launch_kstep<L, __nv_bfloat16, __nv_bfloat16, float, float>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, \
                                             nelv, epb, st);
    AX_LX_CASES(AX_CASE)
#undef AX_CASE
    default:
      return AX_EINVAL;
  }
}

}  // namespace ax
