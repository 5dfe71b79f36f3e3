// many-grid step and advance kernels; state and arithmetic in double.
// (One translation unit per precision and kernel family, so they compile in parallel.)
#include "dugks_launch.cuh"

namespace dugks {
template cudaError_t Launch<double,double>::batch_step(const BatchUniform<double> &, const FaceCoefs<double> &, const BatchGrid<double> *, const int4 *, int, double *, int, int, int, int, cudaStream_t);
template int Launch<double,double>::batch_ctas_per_sm(int, int, int);
template cudaError_t launch_batch_advance<double>(BatchGrid<double> *, int, const double *, double *, int *, double, cudaStream_t);
template cudaError_t launch_batch_factors<double>(BatchGrid<double> *, int, double, cudaStream_t);
}  // namespace dugks
