// Double-float instantiations of the pass kernels (mixed mode's high precision).
#include "cg_launch.cuh"
template struct cgf::Launch<cgf::df>;
