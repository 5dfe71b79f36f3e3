// many-grid step and advance kernels; state and arithmetic in float.
// (One translation unit per precision and kernel family, so they compile in parallel.)
#include "dugks_launch.cuh"

namespace dugks {
template cudaError_t Launch<float,float>::batch_step(const BatchUniform<float> &, const FaceCoefs<float> &, const BatchGrid<float> *, const int4 *, int, double *, int, int, int, int, cudaStream_t);
template int Launch<float,float>::batch_ctas_per_sm(int, int, int);
template cudaError_t launch_batch_advance<float>(BatchGrid<float> *, int, const double *, double *, int *, double, cudaStream_t);
template cudaError_t launch_batch_factors<float>(BatchGrid<float> *, int, double, cudaStream_t);
}  // namespace dugks
