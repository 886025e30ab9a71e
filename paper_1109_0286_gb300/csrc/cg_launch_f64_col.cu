// FP64 instantiations of the column-pass and vector kernels.
#include "cg_launch.cuh"
namespace cgf {
CGF_INSTANTIATE_COLS(double)
}  // namespace cgf
