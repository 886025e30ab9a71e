// FP64 instantiations of the row-pass dispatch (the kernels are compiled in
// cg_launch_f64_row<k>.cu, one group of lengths per unit).
#include "cg_launch.cuh"
namespace cgf {
CGF_INSTANTIATE_ROWS(double)
}  // namespace cgf
