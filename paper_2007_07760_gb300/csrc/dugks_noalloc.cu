// dugks_noalloc.cu -- FP64 sum of a device field that allocates no device memory.
//
// The context API keeps its per-tile mass partials in memory it allocates
// with cudaMalloc. Some callers cannot allocate at the point where they need a
// mass: hosts whose device memory is entirely reserved by another allocator (a
// framework's caching pool, which hands out no raw cudaMalloc memory), and
// latency-critical loops that must not take the implicit device
// synchronisation of cudaMalloc / cudaFree. For them this file provides the
// same two-kernel reduction (one FP64 partial per 32 x 8 tile, then one CTA
// summing the partials in a fixed order) with the partials in a file-scope
// device array instead.
//
// The array is static device memory of this library: every GPU on which the
// library's kernels are loaded holds it (512 KiB) until the process exits.
#include <mutex>

#include "../../include/dugks.h"
#include "dugks_internal.h"

namespace {

constexpr int NOALLOC_MAX_TILES = DUGKS_NOALLOC_MAX_TILES;
constexpr int NOALLOC_TILE_X = 32, NOALLOC_TILE_Y = 8;

// One FP64 partial per tile, shared by every call on a device. Each call
// overwrites entries [0, tiles) before reading them, so nothing has to start
// at zero; calls whose kernels overlap on the GPU race on these entries.
static __device__ __align__(256) double g_noalloc_partial[NOALLOC_MAX_TILES];

template <typename T>
__global__ void __launch_bounds__(256)
field_partial_kernel(const T *field, int nx, int ny, int pitch, int tiles_x, double *partial) {
    __shared__ double sred[32];
    // one-dimensional grid of tiles (tile = by * tiles_x + bx): a field one tile
    // wide may have up to NOALLOC_MAX_TILES tile rows, beyond the y-grid limit
    const int tile = blockIdx.x, by = tile / tiles_x, bx = tile - by * tiles_x;
    const int x0 = bx * NOALLOC_TILE_X, y0 = by * NOALLOC_TILE_Y;
    double msum = 0.0;
    for (int idx = threadIdx.x; idx < NOALLOC_TILE_X * NOALLOC_TILE_Y; idx += blockDim.x) {
        const int ly = idx / NOALLOC_TILE_X, lx = idx - ly * NOALLOC_TILE_X;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= nx || gy >= ny) continue;
        msum += (double)field[(size_t)gy * pitch + gx];
    }
    const double s = dugks::block_sum(msum, sred);
    if (threadIdx.x == 0) partial[tile] = s;
}

__global__ void __launch_bounds__(256) field_final_kernel(const double *partial, int n, double *out) {
    __shared__ double sred[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    s = dugks::block_sum(s, sred);
    if (threadIdx.x == 0) *out = s;
}

// Host side: the device address of g_noalloc_partial, looked up once per device
// (in host code the symbol name is only a host-side stand-in for it).
constexpr int MAX_DEVICES = 64;
double *g_scratch[MAX_DEVICES] = {};
std::mutex g_scratch_mu;

int scratch_for_current_device(double **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return DUGKS_ECUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_partial) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return DUGKS_ECUDA;
        }
        g_scratch[dev] = static_cast<double *>(ptr);
    }
    *out = g_scratch[dev];
    return DUGKS_OK;
}

}  // namespace

extern "C" int dugks_field_mass_noalloc(const void *field, int dtype, int32_t nx, int32_t ny, int32_t pitch,
                                        double *out_dev, void *cuda_stream) {
    if (!field || !out_dev || nx < 1 || ny < 1 || pitch < nx || (dtype != 0 && dtype != 1)) return DUGKS_EINVAL;
    const int tiles_x = (nx + NOALLOC_TILE_X - 1) / NOALLOC_TILE_X;
    const int64_t tiles = (int64_t)tiles_x * ((ny + NOALLOC_TILE_Y - 1) / NOALLOC_TILE_Y);
    if (tiles > NOALLOC_MAX_TILES) return DUGKS_EINVAL;   // beyond the static scratch
    double *scratch = nullptr;
    int r = scratch_for_current_device(&scratch);
    if (r != DUGKS_OK) return r;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // launched through cudaLaunchKernel so that each launch's own status is
    // returned (an earlier, unrelated error pending on this thread is neither
    // reported as this call's failure nor cleared)
    const void *field_arg = field;
    int ntiles = (int)tiles, nx_ = nx, ny_ = ny, pitch_ = pitch, tx_ = tiles_x;
    void *pargs[] = {&field_arg, &nx_, &ny_, &pitch_, &tx_, &scratch};
    const void *pk = dtype == 0 ? reinterpret_cast<const void *>(&field_partial_kernel<double>)
                                : reinterpret_cast<const void *>(&field_partial_kernel<float>);
    if (cudaLaunchKernel(pk, dim3(ntiles), dim3(256), pargs, 0, s) != cudaSuccess) return DUGKS_ECUDA;
    void *fargs[] = {&scratch, &ntiles, &out_dev};
    if (cudaLaunchKernel(reinterpret_cast<const void *>(&field_final_kernel), dim3(1), dim3(256), fargs, 0, s) !=
        cudaSuccess)
        return DUGKS_ECUDA;
    return DUGKS_OK;
}
