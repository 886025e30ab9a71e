// FP64 instantiations of the pass kernels.
#include "cg_launch.cuh"
template struct cgf::Launch<double>;
