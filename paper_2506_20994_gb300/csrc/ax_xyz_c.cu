// Instantiations of the six-matrix element operator for lx in {11, 12}
// (split across files to compile in parallel).
#include "ax_xyz.cuh"

namespace ax {
namespace xyz {
#define AX_XYZ_LX(M) M(11) M(12)
AX_XYZ_DISPATCH(dispatch_c, AX_XYZ_LX)
}  // namespace xyz
}  // namespace ax
