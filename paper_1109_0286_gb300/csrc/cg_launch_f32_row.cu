// FP32 instantiations of the row-pass dispatch (the kernels are compiled in
// cg_launch_f32_row<k>.cu, one group of lengths per unit).
#include "cg_launch.cuh"
namespace cgf {
CGF_INSTANTIATE_ROWS(float)
}  // namespace cgf
