// FP32 row-pass kernels for nx/2 = 2^9..2^12.
#include "cg_launch.cuh"
namespace cgf {
CGF_ROW_LL(, float, 9) CGF_ROW_LL(, float, 10) CGF_ROW_LL(, float, 11) CGF_ROW_LL(, float, 12)
}  // namespace cgf
