// lee_measure.cu -- measurement utility for the FP64 roofline: a kernel that
// issues FP64 fused multiply-adds only.  The paper has no counterpart; the
// benchmark times it with CUDA events to obtain this GPU's FP64 FMA rate, the
// bound of the FP64 stencil path (about 32 FP64 instructions per point-stage
// against 66 bytes of HBM traffic).
#include <string>

#include <cuda_runtime.h>

#include "lee_internal.h"
#include "../../include/lee.h"

namespace lee {
namespace {

constexpr int FMA_THREADS = 256;
constexpr int FMA_CHAINS = 8;           // independent chains per thread (covers the pipe latency)

// x <- x * a + b on FMA_CHAINS chains; |a| < 1 keeps every value bounded, so
// the store of the sum happens only if the arithmetic were to misbehave
__global__ void __launch_bounds__(FMA_THREADS) fma_probe_kernel(long long iters, double *sink) {
    double x[FMA_CHAINS];
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    const double a = 0.999999, b = 1e-7 * (1 + (blockIdx.x & 7));
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < FMA_CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; ++c) s += x[c];
    if (!(s < 1e30)) *sink = s;
}

}  // namespace
}  // namespace lee

extern "C" int lee_fp64_fma_probe(int blocks, long long iters, double *sink, void *stream) {
    using namespace lee;
    if (blocks < 1 || iters < 1 || !sink) {
        set_global_error("lee_fp64_fma_probe: bad argument");
        return LEE_ERR_ARG;
    }
    fma_probe_kernel<<<blocks, FMA_THREADS, 0, (cudaStream_t)stream>>>(iters, sink);
    count_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_global_error(std::string("lee_fp64_fma_probe: ") + cudaGetErrorString(e));
        return LEE_ERR_CUDA;
    }
    return LEE_OK;
}
