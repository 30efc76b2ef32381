// Instantiation of the k-loop element operator for storage double, arithmetic double.
#include "ax_kstep.cuh"
#include "dispatch.h"

namespace ax {

int dispatch_kstep_f64(int lx, double *w, const double *u, const double *dx,
                                     const double *dxt, const double *h1, const double *g11,
                                     const double *g22, const double *g33, const double *g12,
                                     const double *g13, const double *g23, int nelv, int epb,
                                     cudaStream_t st) {
  switch (lx) {
#define AX_CASE(L)                                                                             \
  case L:                                                                                      \
    return launch_kstep<L, double, double, double, double>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, \
                                             nelv, epb, st);
    AX_LX_CASES(AX_CASE)
#undef AX_CASE
    default:
      return AX_EINVAL;
  }
}

}  // namespace ax
