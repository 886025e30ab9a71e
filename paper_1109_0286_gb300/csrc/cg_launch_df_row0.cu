// Double-float (mixed mode's high precision) row-pass kernels for nx/2 = 2^4..2^7.
#include "cg_launch.cuh"
namespace cgf {
CGF_ROW_LL(, df, 4) CGF_ROW_LL(, df, 5) CGF_ROW_LL(, df, 6) CGF_ROW_LL(, df, 7)
}  // namespace cgf
