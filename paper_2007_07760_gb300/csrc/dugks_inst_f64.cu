// FP64 instantiation of the DUGKS kernels (state and arithmetic in double).
#include "dugks_launch.cuh"
template struct dugks::Launch<double, double>;
