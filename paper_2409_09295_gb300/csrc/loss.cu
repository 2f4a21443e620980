// Stage a8: the L1 photometric (+ rendered-depth) loss of GEVO's objectives --
// E_pho of the local stage (Section III-B1, Eq. 2) and the photometric
// consistency E_pc over rendered past keyframes with stop-gradient targets
// (Section III-B2, Eq. 6) -- fused with its gradient in one HBM pass.
#include "gevo_internal.cuh"

namespace gevo {

// grid = (blocks over the largest view, n_views); one view per block row.
__global__ void __launch_bounds__(256)
k_loss_l1(gevo_layout L, const float4* __restrict__ rgb, const float4* __restrict__ trgb,
          const float4* __restrict__ d, const float4* __restrict__ td, float lambda,
          float4* __restrict__ g_rgb, float4* __restrict__ g_d, float* __restrict__ loss,
          int vec_ok)
{
    const int v = blockIdx.y;
    const size_t P = (size_t)L.width[v] * L.height[v];
    const size_t base = (size_t)L.pix_base[v];
    const float sc = 1.f / (3.f * (float)P);
    const float sd = lambda / (float)P;
    float acc = 0.f;
    const float* rgbf = reinterpret_cast<const float*>(rgb) + 3 * base;
    const float* trgbf = reinterpret_cast<const float*>(trgb) + 3 * base;
    float* grgbf = reinterpret_cast<float*>(g_rgb) + 3 * base;
    const float* df = d ? reinterpret_cast<const float*>(d) + base : nullptr;
    const float* tdf = td ? reinterpret_cast<const float*>(td) + base : nullptr;
    float* gdf = g_d ? reinterpret_cast<float*>(g_d) + base : nullptr;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (vec_ok) {
        // 3P and P are multiples of 4 and every plane is 16-byte aligned
        const size_t n3 = 3 * P / 4;
        for (size_t i = i0; i < n3; i += stride) {
            const float4 a = reinterpret_cast<const float4*>(rgbf)[i];
            const float4 b = reinterpret_cast<const float4*>(trgbf)[i];
            const float e0 = a.x - b.x, e1 = a.y - b.y, e2 = a.z - b.z, e3 = a.w - b.w;
            acc += sc * (fabsf(e0) + fabsf(e1) + fabsf(e2) + fabsf(e3));
            reinterpret_cast<float4*>(grgbf)[i] =
                make_float4(sc * (float)((e0 > 0.f) - (e0 < 0.f)), sc * (float)((e1 > 0.f) - (e1 < 0.f)),
                            sc * (float)((e2 > 0.f) - (e2 < 0.f)), sc * (float)((e3 > 0.f) - (e3 < 0.f)));
        }
        if (lambda != 0.f) {
            const size_t n1 = P / 4;
            for (size_t i = i0; i < n1; i += stride) {
                const float4 a = reinterpret_cast<const float4*>(df)[i];
                const float4 b = reinterpret_cast<const float4*>(tdf)[i];
                const float e0 = a.x - b.x, e1 = a.y - b.y, e2 = a.z - b.z, e3 = a.w - b.w;
                acc += sd * (fabsf(e0) + fabsf(e1) + fabsf(e2) + fabsf(e3));
                reinterpret_cast<float4*>(gdf)[i] =
                    make_float4(sd * (float)((e0 > 0.f) - (e0 < 0.f)), sd * (float)((e1 > 0.f) - (e1 < 0.f)),
                                sd * (float)((e2 > 0.f) - (e2 < 0.f)), sd * (float)((e3 > 0.f) - (e3 < 0.f)));
            }
        }
    } else {
        for (size_t i = i0; i < 3 * P; i += stride) {
            const float e = rgbf[i] - trgbf[i];
            acc += sc * fabsf(e);
            grgbf[i] = sc * (float)((e > 0.f) - (e < 0.f));
        }
        if (lambda != 0.f) {
            for (size_t i = i0; i < P; i += stride) {
                const float e = df[i] - tdf[i];
                acc += sd * fabsf(e);
                gdf[i] = sd * (float)((e > 0.f) - (e < 0.f));
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float s_acc[8];
    if ((threadIdx.x & 31) == 0) s_acc[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_acc[w];
        atomicAdd(loss + v, t);
    }
}

// The same loss with the per-pixel error e(u) = (|dr| + |dg| + |db|) / 3 of the
// rendering-error criterion (Section III-B2, Eq. 5): one thread per pixel reads
// its three channels, so e(u) needs no second pass.
__global__ void __launch_bounds__(256)
k_loss_l1_err(gevo_layout L, const float* __restrict__ rgb, const float* __restrict__ trgb,
              const float* __restrict__ d, const float* __restrict__ td, float lambda,
              float* __restrict__ g_rgb, float* __restrict__ g_d, float* __restrict__ loss,
              float* __restrict__ pix_err)
{
    const int v = blockIdx.y;
    const size_t P = (size_t)L.width[v] * L.height[v];
    const size_t base = (size_t)L.pix_base[v];
    const float sc = 1.f / (3.f * (float)P);
    const float sd = lambda / (float)P;
    const float* a = rgb + 3 * base;
    const float* b = trgb + 3 * base;
    float* g = g_rgb + 3 * base;
    float acc = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < P;
         i += (size_t)gridDim.x * blockDim.x) {
        const float e0 = a[i] - b[i], e1 = a[P + i] - b[P + i], e2 = a[2 * P + i] - b[2 * P + i];
        const float s = fabsf(e0) + fabsf(e1) + fabsf(e2);
        acc += sc * s;
        g[i] = sc * (float)((e0 > 0.f) - (e0 < 0.f));
        g[P + i] = sc * (float)((e1 > 0.f) - (e1 < 0.f));
        g[2 * P + i] = sc * (float)((e2 > 0.f) - (e2 < 0.f));
        pix_err[base + i] = s * (1.f / 3.f);
        if (lambda != 0.f) {
            const float e = d[base + i] - td[base + i];
            acc += sd * fabsf(e);
            g_d[base + i] = sd * (float)((e > 0.f) - (e < 0.f));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float s_acc[8];
    if ((threadIdx.x & 31) == 0) s_acc[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s_acc[w];
        atomicAdd(loss + v, t);
    }
}

}  // namespace gevo

using namespace gevo;

extern "C" gevo_status gevo_loss_l1(const gevo_layout* layout, const float* rgb,
                                    const float* target_rgb, const float* depth,
                                    const float* target_depth, float lambda_depth, float* dL_drgb,
                                    float* dL_ddepth, float* loss, void* workspace, void* stream)
{
    (void)workspace;
    if (!layout || !gevo::layout_valid(*layout) || !rgb || !target_rgb || !dL_drgb || !loss)
        return GEVO_ERR_INVALID;
    if (lambda_depth != 0.f && (!depth || !target_depth || !dL_ddepth)) return GEVO_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(loss, 0, sizeof(float) * layout->n_views, st) != cudaSuccess)
        return GEVO_ERR_CUDA;
    int vec_ok = gevo_aligned(rgb, 16) && gevo_aligned(target_rgb, 16) && gevo_aligned(dL_drgb, 16);
    if (lambda_depth != 0.f)
        vec_ok = vec_ok && gevo_aligned(depth, 16) && gevo_aligned(target_depth, 16) &&
                 gevo_aligned(dL_ddepth, 16);
    int64_t maxP = 0;
    for (int v = 0; v < layout->n_views; v++) {
        const int64_t P = (int64_t)layout->width[v] * layout->height[v];
        if (P % 4 != 0 || layout->pix_base[v] % 4 != 0) vec_ok = 0;
        maxP = std::max(maxP, P);
    }
    const int bx = (int)std::min<int64_t>((3 * maxP / 4 + 255) / 256 + 1, (int64_t)sm_count() * 4);
    dim3 grid(bx, layout->n_views);
    k_loss_l1<<<grid, 256, 0, st>>>(
        *layout, reinterpret_cast<const float4*>(rgb), reinterpret_cast<const float4*>(target_rgb),
        reinterpret_cast<const float4*>(depth), reinterpret_cast<const float4*>(target_depth),
        lambda_depth, reinterpret_cast<float4*>(dL_drgb), reinterpret_cast<float4*>(dL_ddepth), loss,
        vec_ok);
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}

extern "C" gevo_status gevo_loss_l1_err(const gevo_layout* layout, const float* rgb,
                                        const float* target_rgb, const float* depth,
                                        const float* target_depth, float lambda_depth,
                                        float* dL_drgb, float* dL_ddepth, float* loss,
                                        float* pix_err, void* workspace, void* stream)
{
    (void)workspace;
    if (!layout || !gevo::layout_valid(*layout) || !rgb || !target_rgb || !dL_drgb || !loss || !pix_err)
        return GEVO_ERR_INVALID;
    if (lambda_depth != 0.f && (!depth || !target_depth || !dL_ddepth)) return GEVO_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(loss, 0, sizeof(float) * layout->n_views, st) != cudaSuccess)
        return GEVO_ERR_CUDA;
    int64_t maxP = 0;
    for (int v = 0; v < layout->n_views; v++)
        maxP = std::max(maxP, (int64_t)layout->width[v] * layout->height[v]);
    const int bx = (int)std::min<int64_t>((maxP + 255) / 256, (int64_t)sm_count() * 4);
    dim3 grid(bx, layout->n_views);
    k_loss_l1_err<<<grid, 256, 0, st>>>(*layout, rgb, target_rgb, depth, target_depth, lambda_depth,
                                        dL_drgb, dL_ddepth, loss, pix_err);
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}
