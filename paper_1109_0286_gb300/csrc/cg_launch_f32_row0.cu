// FP32 row-pass kernels for nx/2 = 2^4..2^8.
#include "cg_launch.cuh"
namespace cgf {
CGF_ROW_LL(, float, 4) CGF_ROW_LL(, float, 5) CGF_ROW_LL(, float, 6) CGF_ROW_LL(, float, 7) CGF_ROW_LL(, float, 8)
}  // namespace cgf
