// FP64 row-pass kernels for nx/2 = 2^9..2^12.
#include "cg_launch.cuh"
namespace cgf {
CGF_ROW_LL(, double, 9) CGF_ROW_LL(, double, 10) CGF_ROW_LL(, double, 11) CGF_ROW_LL(, double, 12)
}  // namespace cgf
