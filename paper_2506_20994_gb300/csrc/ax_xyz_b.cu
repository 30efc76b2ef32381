// Instantiations of the six-matrix element operator for lx in {8, 9, 10}
// (split across files to compile in parallel).
#include "ax_xyz.cuh"

namespace ax {
namespace xyz {
#define AX_XYZ_LX(M) M(8) M(9) M(10)
AX_XYZ_DISPATCH(dispatch_b, AX_XYZ_LX)
}  // namespace xyz
}  // namespace ax
