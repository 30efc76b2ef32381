// Instantiations of the six-matrix element operator for lx in {2, ..., 7}
// (split across files to compile in parallel).
#include "ax_xyz.cuh"

namespace ax {
namespace xyz {
#define AX_XYZ_LX(M) M(2) M(3) M(4) M(5) M(6) M(7)
AX_XYZ_DISPATCH(dispatch_a, AX_XYZ_LX)
}  // namespace xyz
}  // namespace ax
