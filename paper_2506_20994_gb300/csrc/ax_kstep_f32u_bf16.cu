// Instantiation of the k-loop element operator with fp32 u and bf16 G, h1
// (the bf16 mode of the refinement solve keeps its vectors in fp32).
#include "ax_kstep.cuh"
#include "dispatch.h"

namespace ax {

int dispatch_kstep_f32u_bf16(int lx, float *w, const float *u, const float *dx,
                                     const float *dxt, const __nv_bfloat16 *h1, const __nv_bfloat16 *g11,
                                     const __nv_bfloat16 *g22, const __nv_bfloat16 *g33, const __nv_bfloat16 *g12,
                                     const __nv_bfloat16 *g13, const __nv_bfloat16 *g23, int nelv, int epb,
                                     cudaStream_t st, double *dotp) {
  switch (lx) {
#define AX_CASE(L)                                                                             \
  case L:                                                                                      \
    return launch_kstep<L, float, __nv_bfloat16, float, float>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, \
                                             nelv, epb, st, dotp);
    AX_LX_CASES(AX_CASE)
#undef AX_CASE
    default:
      return AX_EINVAL;
  }
}

}  // namespace ax
