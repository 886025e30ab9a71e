// Double-float (mixed mode's high precision) row-pass kernels for nx/2 = 2^8..2^10.
#include "cg_launch.cuh"
namespace cgf {
CGF_ROW_LL(, df, 8) CGF_ROW_LL(, df, 9) CGF_ROW_LL(, df, 10)
}  // namespace cgf
