// FP32 instantiation of the DUGKS kernels (state and arithmetic in float).
#include "dugks_launch.cuh"
template struct dugks::Launch<float, float>;
template cudaError_t dugks::launch_batch_advance<float>(dugks::BatchGrid<float> *, int, const double *, double *, int *, cudaStream_t);
