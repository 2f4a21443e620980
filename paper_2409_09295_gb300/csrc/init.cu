// Initialisation of new Gaussians from depth (Section III-A).
//
// The paper builds a photometric cost volume over N keyframes (Eq. 1): for each
// pixel u of the newest keyframe I_{N-1}, downsampled 4x, and each of 64 depth
// hypotheses spaced linearly over 0.25-25 m, V(u, d) = mean over the other
// keyframes of |I_{N-1}(u) - I_i(pi(u, d, T^i_{N-1}))|, then extracts depth with
// belief propagation and upsamples it edge-aware before SPGF* makes Gaussians.
// Here: the cost volume as Eq. 1 defines it (grey = mean of RGB, bilinear
// sampling, out-of-image samples left out of the mean), winner-take-all over
// hypotheses in place of belief propagation, nearest x4 upsampling in place of
// the edge-aware filter, and one Gaussian per selected pixel in place of SPGF*
// (the parts the paper only cites).  The learned depth prior feeds the same
// unprojection.
#include "../../include/gevo_prior.h"
#include "gevo_internal.cuh"

namespace gevo {

// 4x4 box average of the mean of RGB: planar [nk][3][H][W] -> [nk][H/4][W/4]
__global__ void k_grey4(int nk, int H, int W, const float* __restrict__ rgb, float* __restrict__ g)
{
    const int h = H / 4, w = W / 4;
    const size_t n = (size_t)nk * h * w;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % w);
        const size_t t = i / w;
        const int y = (int)(t % h);
        const size_t k = t / h;
        float acc = 0.f;
        for (int ch = 0; ch < 3; ch++) {
            const float* p = rgb + (k * 3 + ch) * (size_t)H * W;
            for (int dy = 0; dy < 4; dy++)
                for (int dx = 0; dx < 4; dx++) acc += p[(size_t)(4 * y + dy) * W + 4 * x + dx];
        }
        g[i] = acc * (1.f / 48.f);
    }
}

__device__ __forceinline__ float bilinear(const float* img, int w, int h, float u, float v, bool& ok)
{
    // pixel i is sampled at coordinate i
    ok = u >= 0.f && v >= 0.f && u <= (float)(w - 1) && v <= (float)(h - 1);
    if (!ok) return 0.f;
    const int x0 = min((int)u, w - 2 < 0 ? 0 : w - 2), y0 = min((int)v, h - 2 < 0 ? 0 : h - 2);
    const float fx = u - (float)x0, fy = v - (float)y0;
    const float a = img[y0 * w + x0], b = img[y0 * w + x0 + 1];
    const float c = img[(y0 + 1) * w + x0], d = img[(y0 + 1) * w + x0 + 1];
    return (1.f - fy) * ((1.f - fx) * a + fx * b) + fy * ((1.f - fx) * c + fx * d);
}

// cams: [nk][16] (R, t, fx, fy, cx, cy) of the full-resolution keyframes;
// the reference is keyframe `ref`, the sources all the others.
__global__ void k_cost_volume(int nk, int ref, int h, int w, const float* __restrict__ grey,
                              const float* __restrict__ cams, int nd, float d0, float d1,
                              float* __restrict__ V)
{
    const size_t n = (size_t)h * w * nd;
    const float* cr = cams + 16 * ref;
    const float fx = cr[12] * 0.25f, fy = cr[13] * 0.25f, cx = cr[14] * 0.25f, cy = cr[15] * 0.25f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % nd);
        const size_t q = i / nd;
        const int x = (int)(q % w), y = (int)(q / w);
        const float d = d0 + (d1 - d0) * (float)k / (float)(nd - 1);
        // camera-frame point of pixel (x, y) at depth d (pixel i sits at i + 0.5 - c)
        const float pc[3] = {((float)x + 0.5f - cx) / fx * d, ((float)y + 0.5f - cy) / fy * d, d};
        float pw[3];
        for (int j = 0; j < 3; j++)
            pw[j] = cr[j] * (pc[0] - cr[9]) + cr[3 + j] * (pc[1] - cr[10]) + cr[6 + j] * (pc[2] - cr[11]);
        const float I0 = grey[((size_t)ref * h + y) * w + x];
        float acc = 0.f;
        int cnt = 0;
        for (int s = 0; s < nk; s++) {
            if (s == ref) continue;
            const float* cs = cams + 16 * s;
            float p[3];
            for (int j = 0; j < 3; j++)
                p[j] = cs[3 * j] * pw[0] + cs[3 * j + 1] * pw[1] + cs[3 * j + 2] * pw[2] + cs[9 + j];
            if (!(p[2] > 1e-3f)) continue;
            const float u = cs[12] * 0.25f * p[0] / p[2] + cs[14] * 0.25f - 0.5f;
            const float v = cs[13] * 0.25f * p[1] / p[2] + cs[15] * 0.25f - 0.5f;
            bool ok;
            const float I = bilinear(grey + (size_t)s * h * w, w, h, u, v, ok);
            if (!ok) continue;
            acc += fabsf(I0 - I);
            cnt++;
        }
        V[i] = cnt > 0 ? acc / (float)cnt : 1.f;
    }
}

// winner-take-all over hypotheses (lowest cost, then lowest index), nearest x4
// upsampling to full resolution
__global__ void k_wta_up4(int h, int w, int nd, float d0, float d1, const float* __restrict__ V,
                          float* __restrict__ depth)
{
    const size_t n = (size_t)h * w * 16;
    const int W = 4 * w;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int X = (int)(i % W), Y = (int)(i / W);
        const float* v = V + ((size_t)(Y / 4) * w + X / 4) * nd;
        int best = 0;
        for (int k = 1; k < nd; k++)
            if (v[k] < v[best]) best = k;
        depth[i] = d0 + (d1 - d0) * (float)best / (float)(nd - 1);
    }
}

__device__ __forceinline__ uint32_t hash32(uint32_t x)
{
    x ^= x >> 16; x *= 0x7feb352du; x ^= x >> 15; x *= 0x846ca68bu; x ^= x >> 16;
    return x;
}

// New Gaussians from a depth map: every masked pixel whose hash falls under
// `keep` becomes one Gaussian at its back-projected point, coloured by the
// pixel (SH DC (c - 0.5) / Y00, higher bands 0), isotropic scale
// scale_px * depth / f, identity rotation, opacity `opac`.
__global__ void k_unproject(int H, int W, const float* __restrict__ rgb, const float* __restrict__ depth,
                            const float* __restrict__ mask, const float* __restrict__ cam,
                            uint32_t keep, uint32_t seed, float scale_px, float opac, int K,
                            uint32_t* __restrict__ counter, int cap, float* __restrict__ means,
                            float* __restrict__ scales, float* __restrict__ quats,
                            float* __restrict__ opacities, float* __restrict__ sh)
{
    const size_t P = (size_t)H * W;
    const float fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    const float kY00 = 0.28209479177387814f;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        if (!(mask[p] > 0.5f)) continue;
        if (hash32((uint32_t)p * 2654435761u + seed) > keep) continue;
        const uint32_t slot = atomicAdd(counter, 1u);
        if ((int)slot >= cap) continue;
        const int x = (int)(p % W), y = (int)(p / W);
        const float d = depth[p];
        const float pc[3] = {((float)x + 0.5f - cx) / fx * d, ((float)y + 0.5f - cy) / fy * d, d};
        for (int j = 0; j < 3; j++)
            means[3 * slot + j] = cam[j] * (pc[0] - cam[9]) + cam[3 + j] * (pc[1] - cam[10]) +
                                  cam[6 + j] * (pc[2] - cam[11]);
        const float s = scale_px * d / fx;
        scales[3 * slot] = s; scales[3 * slot + 1] = s; scales[3 * slot + 2] = s;
        quats[4 * slot] = 1.f; quats[4 * slot + 1] = 0.f; quats[4 * slot + 2] = 0.f; quats[4 * slot + 3] = 0.f;
        opacities[slot] = opac;
        for (int ch = 0; ch < 3; ch++) {
            sh[(size_t)slot * K * 3 + ch] = (rgb[ch * P + p] - 0.5f) / kY00;
            for (int k = 1; k < K; k++) sh[((size_t)slot * K + k) * 3 + ch] = 0.f;
        }
    }
}

// ---------------------------------------------------------------------------
// Belief propagation over the cost volume (Section III-A2; the min-sum
// algorithm of Felzenszwalb and Huttenlocher, 2006): 4-connected grid, data
// cost V(p, d_f), discontinuity cost min(s |f_p - f_q|, tau), synchronous
// iterations from zero messages, each message shifted to minimum 0.
// One warp per pixel; lane l holds labels l and l + 32.  The minimisation over
// f_p of h(f_p) + min(s |f_p - f|, tau) splits into
//   min( s f + min_{f_p <= f} (h(f_p) - s f_p),  -s f + min_{f_p >= f} (h(f_p) + s f_p),
//        min h + tau ),
// two warp scans (prefix and suffix minimum) in place of the linear-time
// forward / backward passes.
// msgs: [4][h * w][nd], direction d = message sent to the left, right, upper,
// lower neighbour.
// ---------------------------------------------------------------------------
__device__ __constant__ int c_bp_dy[4] = {0, 0, -1, 1};
__device__ __constant__ int c_bp_dx[4] = {-1, 1, 0, 0};
__device__ __constant__ int c_bp_opp[4] = {1, 0, 3, 2};

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// inclusive prefix (up = true) or suffix minimum over the lanes
__device__ __forceinline__ float warp_scan_min(float v, bool up)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float u = up ? __shfl_up_sync(0xffffffffu, v, o) : __shfl_down_sync(0xffffffffu, v, o);
        if (up ? lane >= o : lane + o < 32) v = fminf(v, u);
    }
    return v;
}

// Loads the data cost and the four incoming messages of pixel (x, y) for
// labels f0 = lane, f1 = lane + 32 (INF past nd for the data cost, 0 for
// messages).
__device__ __forceinline__ void bp_load(int h, int w, int nd, const float* __restrict__ V,
                                        const float* __restrict__ msg, int x, int y, float D[2],
                                        float inc[4][2])
{
    const int lane = threadIdx.x & 31;
    const size_t hw = (size_t)h * w;
    const size_t p = (size_t)y * w + x;
    for (int j = 0; j < 2; j++) {
        const int f = lane + 32 * j;
        D[j] = f < nd ? V[p * nd + f] : INFINITY;
    }
    for (int d = 0; d < 4; d++) {
        const int ny = y + c_bp_dy[d], nx = x + c_bp_dx[d];
        const bool in = ny >= 0 && ny < h && nx >= 0 && nx < w;
        const float* src = msg + (size_t)c_bp_opp[d] * hw * nd + ((size_t)ny * w + nx) * nd;
        for (int j = 0; j < 2; j++) {
            const int f = lane + 32 * j;
            inc[d][j] = (in && f < nd) ? src[f] : 0.f;
        }
    }
}

__global__ void __launch_bounds__(256)
k_bp_iter(int h, int w, int nd, const float* __restrict__ V, const float* __restrict__ msg_in,
          float* __restrict__ msg_out, float s, float tau)
{
    const int lane = threadIdx.x & 31;
    const size_t hw = (size_t)h * w;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (size_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < hw; p += warps) {
        const int x = (int)(p % w), y = (int)(p / w);
        float D[2], inc[4][2];
        bp_load(h, w, nd, V, msg_in, x, y, D, inc);
        float tot[2];
        for (int j = 0; j < 2; j++) tot[j] = D[j] + inc[0][j] + inc[1][j] + inc[2][j] + inc[3][j];
        for (int d = 0; d < 4; d++) {
            float hv[2], a[2], b[2];
            for (int j = 0; j < 2; j++) hv[j] = tot[j] - inc[d][j];   // INF past nd
            const float f0 = (float)lane, f1 = (float)(lane + 32);
            // prefix over f = 0..63: first half, then second half with the first's total
            a[0] = warp_scan_min(hv[0] - s * f0, true);
            const float a0_all = __shfl_sync(0xffffffffu, a[0], 31);
            a[1] = fminf(a0_all, warp_scan_min(hv[1] - s * f1, true));
            // suffix: second half, then first half with the second's total
            b[1] = warp_scan_min(hv[1] + s * f1, false);
            const float b1_all = __shfl_sync(0xffffffffu, b[1], 0);
            b[0] = fminf(b1_all, warp_scan_min(hv[0] + s * f0, false));
            const float hmin = warp_min(fminf(hv[0], hv[1]));
            float m[2];
            m[0] = fminf(fminf(a[0] + s * f0, b[0] - s * f0), hmin + tau);
            m[1] = fminf(fminf(a[1] + s * f1, b[1] - s * f1), hmin + tau);
            if (lane + 32 >= nd) m[1] = INFINITY;
            if (lane >= nd) m[0] = INFINITY;
            const float mmin = warp_min(fminf(m[0], m[1]));
            float* dst = msg_out + (size_t)d * hw * nd + p * nd;
            if (lane < nd) dst[lane] = m[0] - mmin;
            if (lane + 32 < nd) dst[lane + 32] = m[1] - mmin;
        }
    }
}

// Beliefs D + all incoming messages; label = argmin (lowest on ties); depth
// of the label written to the 4 x 4 full-resolution pixels it covers.
__global__ void __launch_bounds__(256)
k_bp_labels(int h, int w, int nd, const float* __restrict__ V, const float* __restrict__ msg,
            float d0, float d1, float* __restrict__ depth, int* __restrict__ labels,
            float* __restrict__ beliefs)
{
    const int lane = threadIdx.x & 31;
    const size_t hw = (size_t)h * w;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (size_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < hw; p += warps) {
        const int x = (int)(p % w), y = (int)(p / w);
        float D[2], inc[4][2];
        bp_load(h, w, nd, V, msg, x, y, D, inc);
        float bv = INFINITY;
        int bi = 0x7fffffff;
        for (int j = 0; j < 2; j++) {
            const int f = lane + 32 * j;
            if (f >= nd) continue;
            const float b = D[j] + inc[0][j] + inc[1][j] + inc[2][j] + inc[3][j];
            if (beliefs) beliefs[p * nd + f] = b;
            if (b < bv) { bv = b; bi = f; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov < bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if (labels && lane == 0) labels[p] = bi;
        if (lane < 16) {
            const int W = 4 * w;
            depth[(size_t)(4 * y + (lane >> 2)) * W + 4 * x + (lane & 3)] =
                d0 + (d1 - d0) * (float)bi / (float)(nd - 1);
        }
    }
}

static int gridn(size_t n) { return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, (size_t)sm_count() * 16)); }

}  // namespace gevo

using namespace gevo;

extern "C" {

gevo_status gevo_cost_volume(int32_t nk, int32_t ref, int32_t H, int32_t W, const float* rgb,
                             const float* cams, int32_t nd, float d0, float d1, float* grey,
                             float* volume, float* depth, void* stream)
{
    if (nk < 2 || ref < 0 || ref >= nk || H % 4 || W % 4 || H < 8 || W < 8 || !rgb || !cams ||
        nd < 2 || !(d1 > d0) || !grey || !volume || !depth)
        return GEVO_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    const int h = H / 4, w = W / 4;
    k_grey4<<<gridn((size_t)nk * h * w), 256, 0, st>>>(nk, H, W, rgb, grey);
    GEVO_CHECK_LAUNCH();
    k_cost_volume<<<gridn((size_t)h * w * nd), 256, 0, st>>>(nk, ref, h, w, grey, cams, nd, d0, d1, volume);
    GEVO_CHECK_LAUNCH();
    k_wta_up4<<<gridn((size_t)H * W), 256, 0, st>>>(h, w, nd, d0, d1, volume, depth);
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}

gevo_status gevo_unproject(int32_t H, int32_t W, const float* rgb, const float* depth,
                           const float* mask, const float* cam, uint32_t keep, uint32_t seed,
                           float scale_px, float opacity, int32_t sh_degree, uint32_t* counter,
                           int32_t cap, float* means, float* scales, float* quats,
                           float* opacities, float* sh, void* stream)
{
    if (H <= 0 || W <= 0 || !rgb || !depth || !mask || !cam || !counter || cap < 0 || !means ||
        !scales || !quats || !opacities || !sh || sh_degree < 0 || sh_degree > 3)
        return GEVO_ERR_INVALID;
    const int K = (sh_degree + 1) * (sh_degree + 1);
    k_unproject<<<gridn((size_t)H * W), 256, 0, (cudaStream_t)stream>>>(
        H, W, rgb, depth, mask, cam, keep, seed, scale_px, opacity, K, counter, cap, means, scales,
        quats, opacities, sh);
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}

gevo_status gevo_depth_bp(int32_t h, int32_t w, int32_t nd, const float* volume, float s,
                          float tau, int32_t iters, float d0, float d1, float* msgs, float* depth,
                          int32_t* labels, float* beliefs, void* stream)
{
    if (h < 1 || w < 1 || nd < 2 || nd > 64 || !volume || !(s >= 0.f) || !(tau >= 0.f) ||
        iters < 0 || !(d1 > d0) || !msgs || !depth)
        return GEVO_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t per = (size_t)4 * h * w * nd;
    float* a = msgs;
    float* b = msgs + per;
    if (cudaMemsetAsync(a, 0, sizeof(float) * per, st) != cudaSuccess) return GEVO_ERR_CUDA;
    const int grid = gridn((size_t)h * w * 32);
    for (int it = 0; it < iters; it++) {
        k_bp_iter<<<grid, 256, 0, st>>>(h, w, nd, volume, a, b, s, tau);
        GEVO_CHECK_LAUNCH();
        float* t = a; a = b; b = t;
    }
    k_bp_labels<<<grid, 256, 0, st>>>(h, w, nd, volume, a, d0, d1, depth, labels, beliefs);
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}

}  // extern "C"
