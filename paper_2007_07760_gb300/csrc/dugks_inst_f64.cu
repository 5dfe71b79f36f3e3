// FP64 instantiation of the DUGKS kernels (state and arithmetic in double).
#include "dugks_launch.cuh"
template struct dugks::Launch<double, double>;
template cudaError_t dugks::launch_batch_advance<double>(dugks::BatchGrid<double> *, int, const double *, double *, int *, cudaStream_t);
