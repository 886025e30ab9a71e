// Double-float (mixed mode's high precision) instantiations of the column-pass and vector kernels.
#include "cg_launch.cuh"
namespace cgf {
CGF_INSTANTIATE_COLS(df)
}  // namespace cgf
