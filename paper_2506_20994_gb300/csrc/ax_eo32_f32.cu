// Instantiation of the persistent even-odd fp32-arithmetic operator
// (ax_eo32.cuh) for u stored as float and the geometry as float.
#include "ax_eo32.cuh"
#include "dispatch.h"

namespace ax {

int dispatch_eo32_f32(int lx, float *w, const float *u, const float *dx, const float *dxt,
                     const float *const g[7], int nelv, int *err, double *dotp,
                     cudaStream_t st, const E32Upd *up) {
  switch (lx) {
#define AX_CASE(L) \
  case L:          \
    return e32::launch<L, float, float>(w, u, dx, dxt, g, nelv, err, dotp, st, up);
    AX_CASE(6) AX_CASE(8) AX_CASE(10) AX_CASE(12)
#undef AX_CASE
    default:
      return AX_EINVAL;
  }
}

int eo32_blocks_f32(int lx, int nelv) {
  switch (lx) {
    case 6: return e32::blocks<6, float, float>(nelv);
    case 8: return e32::blocks<8, float, float>(nelv);
    case 10: return e32::blocks<10, float, float>(nelv);
    case 12: return e32::blocks<12, float, float>(nelv);
    default: return 0;
  }
}

}  // namespace ax
