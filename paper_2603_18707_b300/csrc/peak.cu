// Arithmetic peak microbenchmark: the denominators of the blend's roofline.
//
// The blend is bound by the FP32 FMA pipe (FP16x2 for the packed variant), not
// by HBM or tensor cores, so its roofline fraction needs the rate at which
// this GPU retires FFMA (HFMA2) lanes. Each thread runs kChains independent
// FMA chains for `iters` rounds; the chains are long enough that the pipe,
// not latency, sets the rate when at least 4 warps per scheduler are resident.
// The values stay finite (x <- x * m + c with |m| < 1) and one sum per
// thread is written so that nothing is optimised away.
#include <cuda_fp16.h>

#include "gs_common.cuh"

namespace gs {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) ffma_peak_kernel(int iters, float *sink)
{
    const float m = 0.999f, c = 1e-3f * (float)(threadIdx.x & 7);
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = (float)(threadIdx.x + i);
    for (int r = 0; r < iters; ++r) {
#pragma unroll 16
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], m, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) hfma2_peak_kernel(int iters, float *sink)
{
    const __half2 m = __float2half2_rn(0.999f), c = __float2half2_rn(1e-3f * (float)(threadIdx.x & 7));
    __half2 x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = __float2half2_rn((float)((threadIdx.x + i) & 63) * 0.01f);
    for (int r = 0; r < iters; ++r) {
#pragma unroll 16
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = __hfma2(x[i], m, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += __low2float(x[i]) + __high2float(x[i]);
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

} // namespace
} // namespace gs

using namespace gs;

extern "C" gs_status gs_fma_peak(void *stream, int32_t half2, int32_t blocks, int32_t iters, float *d_sink,
                                 double *flop)
{
    if (blocks <= 0 || iters <= 0 || !d_sink || !flop || (half2 != 0 && half2 != 1)) return GS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (half2)
        hfma2_peak_kernel<<<blocks, 256, 0, s>>>(iters, d_sink);
    else
        ffma_peak_kernel<<<blocks, 256, 0, s>>>(iters, d_sink);
    if (cudaPeekAtLastError() != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    count_launch();
    // an FMA is 2 FLOP per lane; a half2 FMA carries two lanes
    *flop = (double)blocks * 256.0 * (double)iters * 16.0 * kChains * 2.0 * (half2 ? 2.0 : 1.0);
    return GS_OK;
}
