// Instantiation of the persistent even-odd fp32-arithmetic operator
// (ax_eo32.cuh) for u stored as float and the geometry as __nv_bfloat16;
// lx = 8 runs the warp-per-element form (ax_eo32w.cuh) in every variant.
#include "ax_eo32.cuh"
#include "dispatch.h"

namespace ax {

int dispatch_eo32_f32u_bf16(int lx, float *w, const float *u, const float *dx, const float *dxt,
                     const __nv_bfloat16 *const g[7], int nelv, int *err, double *dotp,
                     cudaStream_t st, const E32Upd *up) {
  switch (lx) {
#define AX_CASE(L) \
  case L:          \
    return e32::launch<L, float, __nv_bfloat16>(w, u, dx, dxt, g, nelv, err, dotp, st, up);
    AX_CASE(6) AX_CASE(10) AX_CASE(12)
    case 8:
      return dispatch_eo32w_f32u_bf16(w, u, dx, dxt, g, nelv, err, dotp, st, up);
#undef AX_CASE
    default:
      return AX_EINVAL;
  }
}

int eo32_blocks_f32u_bf16(int lx, int nelv) {
  switch (lx) {
    case 6: return e32::blocks<6, float, __nv_bfloat16>(nelv);
    case 8: return eo32w_blocks_f32u_bf16(nelv);
    case 10: return e32::blocks<10, float, __nv_bfloat16>(nelv);
    case 12: return e32::blocks<12, float, __nv_bfloat16>(nelv);
    default: return 0;
  }
}

}  // namespace ax
