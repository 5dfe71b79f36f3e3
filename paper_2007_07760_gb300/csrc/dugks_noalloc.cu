// dugks_noalloc.cu -- FP64 sum of a device field that allocates no device memory.
//
// The context API keeps its per-tile mass partials in memory it allocates
// with cudaMalloc. Some callers cannot allocate at the point where they need a
// mass: code that runs while a stream is being captured into a CUDA graph
// (cudaMalloc is not a stream operation and may be refused there), hosts whose
// device memory is entirely reserved by another allocator (a framework's
// caching pool), and latency-critical loops that must not take the implicit
// device synchronisation of cudaMalloc / cudaFree. For them this file provides
// the same two-kernel reduction (one FP64 partial per 32 x 8 tile, then one
// CTA summing the partials in a fixed order) with the partials in a
// file-scope device array instead.
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
    const int x0 = blockIdx.x * NOALLOC_TILE_X, y0 = blockIdx.y * NOALLOC_TILE_Y;
    double msum = 0.0;
    for (int idx = threadIdx.x; idx < NOALLOC_TILE_X * NOALLOC_TILE_Y; idx += blockDim.x) {
        const int ly = idx / NOALLOC_TILE_X, lx = idx - ly * NOALLOC_TILE_X;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= nx || gy >= ny) continue;
        msum += (double)field[(size_t)gy * pitch + gx];
    }
    const double s = dugks::block_sum(msum, sred);
    if (threadIdx.x == 0) partial[blockIdx.y * tiles_x + blockIdx.x] = s;
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
    dim3 grid(tiles_x, (ny + NOALLOC_TILE_Y - 1) / NOALLOC_TILE_Y);
    if (dtype == 0)
        field_partial_kernel<double><<<grid, 256, 0, s>>>(static_cast<const double *>(field), nx, ny, pitch, tiles_x,
                                                          scratch);
    else
        field_partial_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float *>(field), nx, ny, pitch, tiles_x,
                                                         scratch);
    field_final_kernel<<<1, 256, 0, s>>>(scratch, (int)tiles, out_dev);
    return cudaGetLastError() == cudaSuccess ? DUGKS_OK : DUGKS_ECUDA;
}
