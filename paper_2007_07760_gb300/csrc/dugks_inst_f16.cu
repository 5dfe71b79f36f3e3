// FP32 arithmetic with the distribution stored as half-precision scaled
// deviations from w_k phi (phi kept in FP32).
#include "dugks_launch.cuh"
template struct dugks::Launch<float, __half>;
