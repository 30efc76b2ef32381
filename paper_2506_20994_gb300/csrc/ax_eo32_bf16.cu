// Instantiation of the persistent even-odd fp32-arithmetic operator
// (ax_eo32.cuh) for u stored as __nv_bfloat16 and the geometry as __nv_bfloat16.
#include "ax_eo32.cuh"
#include "dispatch.h"

namespace ax {

int dispatch_eo32_bf16(int lx, float *w, const __nv_bfloat16 *u, const float *dx, const float *dxt,
                     const __nv_bfloat16 *const g[7], int nelv, int *err, double *dotp,
                     cudaStream_t st, const E32Upd *up) {
  // lx = 8 without the fused update: one warp per element (ax_eo32w.cuh)
  if (lx == 8 && !up && !dotp) return dispatch_eo32w_bf16(w, u, dx, dxt, g, nelv, err, dotp, st);
  switch (lx) {
#define AX_CASE(L) \
  case L:          \
    return e32::launch<L, __nv_bfloat16, __nv_bfloat16>(w, u, dx, dxt, g, nelv, err, dotp, st, up);
    AX_CASE(6) AX_CASE(8) AX_CASE(10) AX_CASE(12)
#undef AX_CASE
    default:
      return AX_EINVAL;
  }
}

int eo32_blocks_bf16(int lx, int nelv) {
  switch (lx) {
    case 6: return e32::blocks<6, __nv_bfloat16, __nv_bfloat16>(nelv);
    case 8: return e32::blocks<8, __nv_bfloat16, __nv_bfloat16>(nelv);
    case 10: return e32::blocks<10, __nv_bfloat16, __nv_bfloat16>(nelv);
    case 12: return e32::blocks<12, __nv_bfloat16, __nv_bfloat16>(nelv);
    default: return 0;
  }
}

}  // namespace ax
