// FP64 row-pass kernels for nx/2 = 2^4..2^8.
#include "cg_launch.cuh"
namespace cgf {
CGF_ROW_LL(, double, 4) CGF_ROW_LL(, double, 5) CGF_ROW_LL(, double, 6) CGF_ROW_LL(, double, 7) CGF_ROW_LL(, double, 8)
}  // namespace cgf
