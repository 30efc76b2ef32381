// Instantiation of the k-loop element operator for storage float, arithmetic float.
#include "ax_kstep.cuh"
#include "dispatch.h"

namespace ax {

int dispatch_kstep_f32(int lx, float *w, const float *u, const float *dx,
                                     const float *dxt, const float *h1, const float *g11,
                                     const float *g22, const float *g33, const float *g12,
                                     const float *g13, const float *g23, int nelv, int epb,
                                     cudaStream_t st, double *dotp) {
  switch (lx) {
#define AX_CASE(L)                                                                             \
  case L:                                                                                      \
    return launch_kstep<L, float, float, float, float>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, \
                                             nelv, epb, st, dotp);
    AX_LX_CASES(AX_CASE)
#undef AX_CASE
    default:
      return AX_EINVAL;
  }
}

}  // namespace ax
