// lee_noalloc.cu -- acoustic-energy reduction that allocates no device memory.
//
// lee_energy() reduces into scratch inside the context's arena.  Some callers
// cannot provide or allocate such scratch: their device memory belongs to
// another runtime or memory pool that only hands out the field arrays, so any
// cudaMalloc (or a temporary from an allocating library) is not allowed on
// their side.  lee_energy_noalloc() takes only the caller's input and output
// pointers and keeps its scratch in a fixed-size static device array.
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "lee_internal.h"
#include "../../include/lee.h"

namespace lee {

namespace {

// Scratch: one partial sum per grid row.  Every GPU that loads the library
// holds this array (128 KiB) until the process exits; every call on a device
// shares it, so calls that overlap on the GPU race.
static __device__ __align__(256) double g_row_partials[LEE_NOALLOC_MAX_ROWS];

// one warp per row; lane-strided sum, then a fixed shuffle tree
template <typename T>
__global__ void row_energy_kernel(const T *__restrict__ p, const T *__restrict__ u, const T *__restrict__ v,
                                  const unsigned char *__restrict__ mask, int nx, int ny, long long pitch,
                                  double *__restrict__ partials) {
    const int row = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= ny) return;
    const long long o0 = (long long)row * pitch;
    double acc = 0.0;
    for (int i = lane; i < nx; i += 32) {
        const long long o = o0 + i;
        if (mask[o] != 1) continue;
        const double a = (double)p[o], b = (double)u[o], c = (double)v[o];
        acc += a * a + b * b + c * c;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) partials[row] = acc;            // every row < ny is written: nothing to clear
}

// one block: fixed-order sum of the row partials, times 1/2 h^2
__global__ void sum_rows_kernel(const double *__restrict__ partials, int ny, double scale, double *out) {
    __shared__ double s[1024];
    double acc = 0.0;
    for (int j = threadIdx.x; j < ny; j += blockDim.x) acc += partials[j];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = scale * s[0];
}

// Device address of the scratch on the current device.  Host code may not
// pass g_row_partials itself (in host code the name is a host-side stand-in),
// so the address is looked up once per device, with that device current.
double *scratch_on_current_device(std::string &err) {
    static std::mutex mu;
    static double *ptrs[128] = {nullptr};
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 128) {
        err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!ptrs[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_row_partials);
        if (e != cudaSuccess || !p) {
            err = std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e);
            return nullptr;
        }
        ptrs[dev] = (double *)p;
    }
    return ptrs[dev];
}

}  // namespace
}  // namespace lee

extern "C" int lee_energy_noalloc(const void *p, const void *u, const void *v, const unsigned char *mask, int nx,
                                  int ny, long long pitch, int precision, double h, double *out, void *stream) {
    using namespace lee;
    if (ny > LEE_NOALLOC_MAX_ROWS) {
        set_global_error("lee_energy_noalloc: ny = " + std::to_string(ny) + " exceeds the static scratch of " +
                         std::to_string(LEE_NOALLOC_MAX_ROWS) + " rows");
        return LEE_ERR_ARG;
    }
    if (!p || !u || !v || !mask || !out || nx < 1 || ny < 1 || pitch < nx || !(h > 0) ||
        (precision != LEE_FP64 && precision != LEE_FP32)) {
        set_global_error("lee_energy_noalloc: bad argument");
        return LEE_ERR_ARG;
    }
    std::string err;
    double *partials = scratch_on_current_device(err);
    if (!partials) {
        set_global_error(err);
        return LEE_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = 256, blocks = (ny * 32 + threads - 1) / threads;
    if (precision == LEE_FP32)
        row_energy_kernel<float><<<blocks, threads, 0, s>>>((const float *)p, (const float *)u, (const float *)v, mask,
                                                             nx, ny, pitch, partials);
    else
        row_energy_kernel<double><<<blocks, threads, 0, s>>>((const double *)p, (const double *)u, (const double *)v,
                                                              mask, nx, ny, pitch, partials);
    sum_rows_kernel<<<1, 1024, 0, s>>>(partials, ny, 0.5 * h * h, out);
    count_launch(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_global_error(std::string("lee_energy_noalloc: ") + cudaGetErrorString(e));
        return LEE_ERR_CUDA;
    }
    return LEE_OK;
}
