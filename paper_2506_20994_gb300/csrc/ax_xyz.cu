// The element operator with one 1-D matrix per direction: the full argument
// list of the paper's interface (Listing 1) and kernel (Listing 2), where the
// forward gradient takes dx, dy, dz and the transposed one dxt, dyt, dzt.
// fp64-accurate double-float k-loop kernel for lx <= 12 (ax_xyz_a/b/c.cu),
// fp64 units above (here).  When the caller passes the same two matrices for
// every direction the entry point takes the tuned single-matrix path.
#include "ax_xyz.cuh"

namespace ax {
namespace xyz {
#define AX_XYZ_LX(M) M(13) M(14) M(15) M(16)
AX_XYZ_DISPATCH(dispatch_d, AX_XYZ_LX)
}  // namespace xyz
}  // namespace ax

extern "C" int ax_helm_xyz(double *w, const double *u, const double *dx, const double *dy,
                           const double *dz, const double *dxt, const double *dyt,
                           const double *dzt, const double *h1, const double *g11,
                           const double *g22, const double *g33, const double *g12,
                           const double *g13, const double *g23, int lx, int nelv,
                           void *stream) {
  if (!ax::lx_ok(lx) || nelv < 0) return AX_EINVAL;
  if (nelv == 0) return AX_OK;
  if (!ax::all_nonnull(w, u, dx, dy, dz, dxt, dyt, dzt, h1, g11, g22, g33, g12, g13, g23))
    return AX_EINVAL;
  if (dy == dx && dz == dx && dyt == dxt && dzt == dxt)
    return ax_helm(w, u, dx, dxt, h1, g11, g22, g33, g12, g13, g23, lx, nelv, stream);
  auto f = lx <= 7 ? ax::xyz::dispatch_a
         : lx <= 10 ? ax::xyz::dispatch_b
         : lx <= 12 ? ax::xyz::dispatch_c
                    : ax::xyz::dispatch_d;
  return f(lx, w, u, dx, dy, dz, dxt, dyt, dzt, h1, g11, g22, g33, g12, g13, g23, nelv, 0,
           (cudaStream_t)stream);
}
