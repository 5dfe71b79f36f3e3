// FP32 instantiation of the DUGKS kernels (state and arithmetic in float).
#include "dugks_launch.cuh"
template struct dugks::Launch<float, float>;
