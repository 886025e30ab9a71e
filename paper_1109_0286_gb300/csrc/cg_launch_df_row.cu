// Double-float (mixed mode's high precision) instantiations of the row-pass dispatch (the kernels are compiled in
// cg_launch_df_row<k>.cu, one group of lengths per unit).
#include "cg_launch.cuh"
namespace cgf {
CGF_INSTANTIATE_ROWS(df)
}  // namespace cgf
