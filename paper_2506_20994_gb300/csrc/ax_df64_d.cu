// Instantiations of the double-float fp64-accurate element operator for
// lx in {13, 14} (split across files to compile in parallel).
#include "ax_df64.cuh"
#include "dispatch.h"

namespace ax {

int dispatch_df64_d(int lx, double *w, const double *u, const double *dx, const double *dxt,
                    const double *h1, const double *g11, const double *g22, const double *g33,
                    const double *g12, const double *g13, const double *g23, int nelv, int epb,
                    cudaStream_t st) {
  switch (lx) {
    case 13:
      return launch_df64<13>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, nelv, epb, st);
    case 14:
      return launch_df64<14>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, nelv, epb, st);
    default:
      return AX_EINVAL;
  }
}

}  // namespace ax
