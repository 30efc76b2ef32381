// Instantiations of the double-float fp64-accurate element operator for
// lx in {2, 3, 4, 5, 6, 7} (split across files to compile in parallel).
#include "ax_df64.cuh"
#include "dispatch.h"

namespace ax {

int dispatch_df64_a(int lx, double *w, const double *u, const double *dx, const double *dxt,
                    const double *h1, const double *g11, const double *g22, const double *g33,
                    const double *g12, const double *g13, const double *g23, int nelv, int epb,
                    cudaStream_t st) {
  switch (lx) {
    case 2:
      return launch_df64<2>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, nelv, epb, st);
    case 3:
      return launch_df64<3>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, nelv, epb, st);
    case 4:
      return launch_df64<4>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, nelv, epb, st);
    case 5:
      return launch_df64<5>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, nelv, epb, st);
    case 6:
      return launch_df64<6>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, nelv, epb, st);
    case 7:
      return launch_df64<7>(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, nelv, epb, st);
    default:
      return AX_EINVAL;
  }
}

}  // namespace ax
