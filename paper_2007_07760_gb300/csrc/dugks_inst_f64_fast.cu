// TMA-staged single-grid step kernels; state and arithmetic in double.
// (One translation unit per precision and kernel family, so they compile in parallel.)
#include "dugks_launch.cuh"

namespace dugks {
template FastGeom Launch<double,double>::fast_geom(int, int, int);
template cudaError_t Launch<double,double>::step_fast(const StepParams<double> &, const FaceCoefs<double> &, const FastExtra<double> &, const CUtensorMap &, const CUtensorMap &, const CUtensorMap &, int, int, int, cudaStream_t);
}  // namespace dugks
