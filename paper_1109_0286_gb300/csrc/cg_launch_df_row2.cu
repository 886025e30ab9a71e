// Double-float (mixed mode's high precision) row-pass kernels for nx/2 = 2^11..2^12.
#include "cg_launch.cuh"
namespace cgf {
CGF_ROW_LL(, df, 11) CGF_ROW_LL(, df, 12)
}  // namespace cgf
