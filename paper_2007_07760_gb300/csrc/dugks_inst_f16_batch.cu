// many-grid step and advance kernels; FP32 arithmetic, distribution stored as half-precision deviations from w_k phi.
// (One translation unit per precision and kernel family, so they compile in parallel.)
#include "dugks_launch.cuh"

namespace dugks {
template cudaError_t Launch<float,__half>::batch_step(const BatchUniform<float> &, const FaceCoefs<float> &, const BatchGrid<float> *, const int4 *, int, double *, int, int, int, int, cudaStream_t);
template int Launch<float,__half>::batch_ctas_per_sm(int, int, int);
}  // namespace dugks
