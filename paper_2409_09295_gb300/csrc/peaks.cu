// Throughput probes of the FP32 FMA pipe and the MUFU ex2 unit (the units the
// blend and its reverse walk are bound by), timed by the caller.
#include "../../include/gevo_bench.h"
#include "gevo_internal.cuh"

namespace gevo {

__global__ void __launch_bounds__(256) k_bench_fma(int iters, float* __restrict__ sink)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = 1.0f + 1e-3f * (float)(i + k);
    const float b = 0.999999f, c = 1e-7f;
    for (int t = 0; t < iters; t++) {
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = __fmaf_rn(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; k++) s += a[k];
    sink[i] = s;
}

__global__ void __launch_bounds__(256) k_bench_ex2(int iters, float* __restrict__ sink)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = 0.5f + 1e-4f * (float)((i + k) & 1023);
    for (int t = 0; t < iters; t++) {
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = ex2_approx(-x[k]);   // stays in [0.5, 1)
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; k++) s += x[k];
    sink[i] = s;
}

// The FMA probe with the paired instruction: 8 independent fma.rn.f32x2
// chains, 16 FMAs (32 FLOP) per thread and step.
__global__ void __launch_bounds__(256) k_bench_fma2(int iters, float* __restrict__ sink)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    f2 a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = f2_make(1.0f + 1e-3f * (float)(i + k), 1.0f - 1e-3f * (float)k);
    const f2 b = f2_splat(0.999999f), c = f2_splat(1e-7f);
    for (int t = 0; t < iters; t++) {
#pragma unroll
        for (int k = 0; k < 8; k++) a[k] = f2_fma(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; k++) s += f2_lo(a[k]) + f2_hi(a[k]);
    sink[i] = s;
}

// MUFU reciprocal (rcp.approx, the reverse walk's transmittance recovery):
// 8 independent chains.
__global__ void __launch_bounds__(256) k_bench_rcp(int iters, float* __restrict__ sink)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = 1.5f + 1e-4f * (float)((i + k) & 1023);
    for (int t = 0; t < iters; t++) {
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = rcp_approx(x[k]) + 0.5f;   // settles near 1.37
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; k++) s += x[k];
    sink[i] = s;
}

}  // namespace gevo

using namespace gevo;

extern "C" gevo_status gevo_bench_fma2(int32_t blocks, int32_t iters, float* sink, void* stream)
{
    if (blocks < 1 || iters < 1 || !sink) return GEVO_ERR_INVALID;
    k_bench_fma2<<<blocks, 256, 0, (cudaStream_t)stream>>>(iters, sink);
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}

extern "C" gevo_status gevo_bench_rcp(int32_t blocks, int32_t iters, float* sink, void* stream)
{
    if (blocks < 1 || iters < 1 || !sink) return GEVO_ERR_INVALID;
    k_bench_rcp<<<blocks, 256, 0, (cudaStream_t)stream>>>(iters, sink);
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}

extern "C" gevo_status gevo_bench_fma(int32_t blocks, int32_t iters, float* sink, void* stream)
{
    if (blocks < 1 || iters < 1 || !sink) return GEVO_ERR_INVALID;
    k_bench_fma<<<blocks, 256, 0, (cudaStream_t)stream>>>(iters, sink);
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}

extern "C" gevo_status gevo_bench_ex2(int32_t blocks, int32_t iters, float* sink, void* stream)
{
    if (blocks < 1 || iters < 1 || !sink) return GEVO_ERR_INVALID;
    k_bench_ex2<<<blocks, 256, 0, (cudaStream_t)stream>>>(iters, sink);
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}
