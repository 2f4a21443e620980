// Kernels of the learned depth prior (a small BF16 U-Net) around its tensor-core
// convolutions (gemm_tc.cu).  The paper initialises the Gaussians of a newly
// observed region from a photometric cost volume + belief propagation (Section
// III-A); the prior proposes those depths from one rendered RGB image instead,
// trained on (RGB, depth) pairs rendered from the map itself.
//
// Activations are NHWC BF16 with channels a multiple of 8; activation
// gradients are NHWC FP32; parameters are FP32 masters with BF16 copies.
// Every kernel here is HBM-bound elementwise / reduction work.
#include <cuda_bf16.h>

#include "../../include/gevo_prior.h"
#include "gevo_internal.cuh"

namespace gevo {
gevo_status gemm_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb, void* C,
                      int ldc, int out_bf16, const float* bias, int relu, float beta, int ksplit,
                      uint32_t* err, cudaStream_t st, int trans_c);
gevo_status conv3x3_bf16(int nb, int H, int W, int Cin, const void* X, int Cout, const void* Wt,
                         void* Y, int ldy, int out_bf16, const float* bias, int relu, float beta,
                         uint32_t* err, cudaStream_t st);
gevo_status conv3x3_wgrad_bf16(int nb, int H, int W, int Cin, const void* X, int Cout,
                               const void* dZt, float* dWt, int ksplit, uint32_t* err,
                               cudaStream_t st);

using bf16 = __nv_bfloat16;

static int grid_for(size_t n, int threads = 256)
{
    return (int)std::max<size_t>(1, std::min<size_t>((n + threads - 1) / threads, (size_t)sm_count() * 16));
}

// planar FP32 RGB [nb][3][H][W] -> NHWC BF16 with 8 channels (3 used, 5 zero),
// centred: rgb - 0.5.  With all-positive inputs the He-initialised first
// layer's channels start either on or off for every pixel, and training sat
// near a constant-depth predictor for many epochs (two of four seeds never
// left it in 30 epochs); centred, all four left it within 8 epochs.
__global__ void k_rgb_pack(size_t P, int HW, const float* __restrict__ rgb, bf16* __restrict__ X)
{
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        const size_t b = p / HW, q = p - b * HW;
        const float* src = rgb + b * 3 * (size_t)HW + q;
        __align__(16) bf16 v[8];
        v[0] = __float2bfloat16_rn(src[0] - 0.5f);
        v[1] = __float2bfloat16_rn(src[HW] - 0.5f);
        v[2] = __float2bfloat16_rn(src[2 * (size_t)HW] - 0.5f);
#pragma unroll
        for (int i = 3; i < 8; i++) v[i] = __float2bfloat16_rn(0.f);
        *reinterpret_cast<uint4*>(X + p * 8) = *reinterpret_cast<uint4*>(v);
    }
}

// dZ = dY * [Y > 0] for a ReLU layer: writes dZ (BF16, [P][C]) and dZ^T (BF16,
// [C][P], the K-major operand of the weight gradient) and adds the bias
// gradient sum_p dZ into db.  Block = 64 pixels x C channels through shared memory.
// vec: C, ldy a multiple of 8, lddy of 4, all three arrays 16-byte aligned --
// 8 channels of a pixel move as one 16-byte piece of Y and dZ and two of dY.
__global__ void __launch_bounds__(256)
k_relu_bwd(size_t P, int C, const float* __restrict__ dY, int lddy, const bf16* __restrict__ Y,
           int ldy, bf16* __restrict__ dZ, bf16* __restrict__ dZt, float* __restrict__ db, int vec)
{
    __shared__ float s_t[64][129];
    const size_t p0 = (size_t)blockIdx.x * 64;
    if (vec) {
        const int C8 = C / 8;
        for (int i = threadIdx.x; i < 64 * C8; i += blockDim.x) {
            const int r = i / C8, c = 8 * (i - r * C8);
            const size_t p = p0 + r;
            float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (p < P) {
                const uint4 y = *reinterpret_cast<const uint4*>(Y + p * ldy + c);
                const float4 g0 = *reinterpret_cast<const float4*>(dY + p * lddy + c);
                const float4 g1 = *reinterpret_cast<const float4*>(dY + p * lddy + c + 4);
                const uint32_t yw[4] = {y.x, y.y, y.z, y.w};
                const float g[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
                uint32_t o[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    // bf16 > 0 as a float: the low half shifted up, the high half masked
                    z[2 * q] = __uint_as_float(yw[q] << 16) > 0.f ? g[2 * q] : 0.f;
                    z[2 * q + 1] = __uint_as_float(yw[q] & 0xffff0000u) > 0.f ? g[2 * q + 1] : 0.f;
                    const __nv_bfloat162 pr = __floats2bfloat162_rn(z[2 * q], z[2 * q + 1]);
                    o[q] = *reinterpret_cast<const uint32_t*>(&pr);
                }
                *reinterpret_cast<uint4*>(dZ + p * C + c) = make_uint4(o[0], o[1], o[2], o[3]);
            }
#pragma unroll
            for (int q = 0; q < 8; q++) s_t[r][c + q] = z[q];
        }
    } else {
        for (int i = threadIdx.x; i < 64 * C; i += blockDim.x) {
            const int r = i / C, c = i - r * C;
            const size_t p = p0 + r;
            float z = 0.f;
            if (p < P) {
                const float y = __bfloat162float(Y[p * ldy + c]);
                z = y > 0.f ? dY[p * lddy + c] : 0.f;
                dZ[p * C + c] = __float2bfloat16_rn(z);
            }
            s_t[r][c] = z;
        }
    }
    __syncthreads();
    // bias gradient: one partial per channel per block
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float acc = 0.f;
        for (int r = 0; r < 64; r++) acc += s_t[r][c];
        if (acc != 0.f) atomicAdd(db + c, acc);
    }
    if (dZt) {
        for (int i = threadIdx.x; i < 64 * C; i += blockDim.x) {
            const int c = i / 64, r = i - c * 64;
            const size_t p = p0 + r;
            if (p < P) dZt[(size_t)c * P + p] = __float2bfloat16_rn(s_t[r][c]);
        }
    }
}

// 2x2 max pool, NHWC; X rows have stride ldx (a channel slice of a wider buffer)
// I: the index type, 32-bit whenever the element count allows (the index
// arithmetic's divisions dominate these element-wise kernels)
template <typename I>
__global__ void k_maxpool2(int nb, int H, int W, int C, const bf16* __restrict__ X, int ldx,
                           bf16* __restrict__ Y)
{
    const int h = H / 2, w = W / 2;
    const I n = (I)nb * h * w * C;
    for (I i = blockIdx.x * (I)blockDim.x + threadIdx.x; i < n; i += (I)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const I q = i / C;
        const int x = (int)(q % w);
        const I t = q / w;
        const int y = (int)(t % h);
        const I b = t / h;
        const size_t base = (((size_t)b * H + 2 * y) * W + 2 * x) * ldx + c;
        float m = __bfloat162float(X[base]);
        m = fmaxf(m, __bfloat162float(X[base + ldx]));
        m = fmaxf(m, __bfloat162float(X[base + (size_t)W * ldx]));
        m = fmaxf(m, __bfloat162float(X[base + (size_t)W * ldx + ldx]));
        Y[i] = __float2bfloat16_rn(m);
    }
}

// gradient of the 2x2 max pool: the first maximum (row-major scan) of each
// window receives dY; dX = beta dX + that (FP32, stride lddx)
template <typename I>
__global__ void k_maxpool2_bwd(int nb, int H, int W, int C, const bf16* __restrict__ X, int ldx,
                               const float* __restrict__ dY, float* __restrict__ dX, int lddx,
                               float beta)
{
    const int h = H / 2, w = W / 2;
    const I n = (I)nb * h * w * C;
    for (I i = blockIdx.x * (I)blockDim.x + threadIdx.x; i < n; i += (I)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const I q = i / C;
        const int x = (int)(q % w);
        const I t = q / w;
        const int y = (int)(t % h);
        const size_t b = (size_t)(t / h);
        const size_t pix[4] = {(b * H + 2 * y) * W + 2 * x, (b * H + 2 * y) * W + 2 * x + 1,
                               (b * H + 2 * y + 1) * W + 2 * x, (b * H + 2 * y + 1) * W + 2 * x + 1};
        float v[4];
        int arg = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            v[k] = __bfloat162float(X[pix[k] * ldx + c]);
            if (v[k] > v[arg]) arg = k;
        }
        const float g = dY[i];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            float* o = dX + pix[k] * lddx + c;
            const float add = k == arg ? g : 0.f;
            *o = beta != 0.f ? beta * *o + add : add;
        }
    }
}

// nearest x2 upsample: Y (stride ldy, a channel slice) from X [nb][h][w][C]
// vec: 8 channels (16 bytes) per step, 32-bit indices (C, ldy multiples of 8,
// 16-byte aligned, fewer than 2^31 pieces)
__global__ void k_upsample2_vec(int nb, int h, int w, int C, const bf16* __restrict__ X,
                                bf16* __restrict__ Y, int ldy)
{
    const int H = 2 * h, W = 2 * w, C8 = C / 8;
    const unsigned n = (unsigned)nb * H * W * C8;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned c8 = i % C8, q = i / C8;
        const unsigned x = q % W, t = q / W;
        const unsigned y = t % H, b = t / H;
        *reinterpret_cast<uint4*>(Y + (size_t)q * ldy + 8 * c8) =
            *reinterpret_cast<const uint4*>(X + ((size_t)(b * h + y / 2) * w + x / 2) * C + 8 * c8);
    }
}

__global__ void k_upsample2(int nb, int h, int w, int C, const bf16* __restrict__ X,
                            bf16* __restrict__ Y, int ldy)
{
    const int H = 2 * h, W = 2 * w;
    const size_t n = (size_t)nb * H * W * C;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t q = i / C;
        const int x = (int)(q % W);
        const size_t t = q / W;
        const int y = (int)(t % H);
        const size_t b = t / H;
        Y[q * ldy + c] = X[((b * h + y / 2) * w + x / 2) * C + c];
    }
}

// gradient of the x2 upsample: dX[y][x] = sum of the four dY it was copied to;
// vec: 4 channels (16 bytes) per step, 32-bit indices
__global__ void k_upsample2_bwd_vec(int nb, int h, int w, int C, const float* __restrict__ dY,
                                    int lddy, float* __restrict__ dX)
{
    const int W = 2 * w, C4 = C / 4;
    const unsigned n = (unsigned)nb * h * w * C4;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned c4 = i % C4, q = i / C4;
        const unsigned x = q % w, t = q / w;
        const unsigned y = t % h, b = t / h;
        const size_t r0 = ((size_t)b * 2 * h + 2 * y) * W + 2 * x;
        const float4 a = *reinterpret_cast<const float4*>(dY + r0 * lddy + 4 * c4);
        const float4 e = *reinterpret_cast<const float4*>(dY + (r0 + 1) * lddy + 4 * c4);
        const float4 f = *reinterpret_cast<const float4*>(dY + (r0 + W) * lddy + 4 * c4);
        const float4 g = *reinterpret_cast<const float4*>(dY + (r0 + W + 1) * lddy + 4 * c4);
        *reinterpret_cast<float4*>(dX + (size_t)q * C + 4 * c4) =
            make_float4(a.x + e.x + f.x + g.x, a.y + e.y + f.y + g.y, a.z + e.z + f.z + g.z,
                        a.w + e.w + f.w + g.w);
    }
}

__global__ void k_upsample2_bwd(int nb, int h, int w, int C, const float* __restrict__ dY,
                                int lddy, float* __restrict__ dX)
{
    const int W = 2 * w;
    const size_t n = (size_t)nb * h * w * C;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t q = i / C;
        const int x = (int)(q % w);
        const size_t t = q / w;
        const int y = (int)(t % h);
        const size_t b = t / h;
        const size_t r0 = (b * 2 * h + 2 * y) * W + 2 * x;
        dX[i] = dY[r0 * lddy + c] + dY[(r0 + 1) * lddy + c] + dY[(r0 + W) * lddy + c] +
                dY[(r0 + W + 1) * lddy + c];
    }
}

// Wf[ci][tap][co] = W[co][8 - tap][ci]: the data gradient of a 3x3 convolution
// is the convolution of dZ with these weights
__global__ void k_flip3x3(int Cout, int Cin, const bf16* __restrict__ Wt, bf16* __restrict__ Wf)
{
    const int n = Cout * 9 * Cin;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ci = i % Cin, tap = (i / Cin) % 9, co = i / (9 * Cin);
        Wf[((size_t)ci * 9 + (8 - tap)) * Cout + co] = Wt[i];
    }
}

// 1x1 head: pred[p] = sum_c w[c] X[p][c] + b  (C = 16, FP32 out)
__global__ void k_head_fwd(size_t P, int C, const bf16* __restrict__ X, const float* __restrict__ w,
                           const float* __restrict__ b, float* __restrict__ pred)
{
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        float acc = b[0];
        for (int c = 0; c < C; c++) acc += w[c] * __bfloat162float(X[p * C + c]);
        pred[p] = acc;
    }
}

__global__ void __launch_bounds__(256)
k_head_bwd(size_t P, int C, const bf16* __restrict__ X, const float* __restrict__ w,
           const float* __restrict__ dpred, float* __restrict__ dX, float* __restrict__ dw,
           float* __restrict__ db)
{
    __shared__ float s_w[16 + 1][8];
    float aw[16];
#pragma unroll
    for (int c = 0; c < 16; c++) aw[c] = 0.f;
    float ab = 0.f;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        const float g = dpred[p];
        ab += g;
#pragma unroll
        for (int c = 0; c < 16; c++) {
            if (c < C) {
                dX[p * C + c] = g * w[c];
                aw[c] += g * __bfloat162float(X[p * C + c]);
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 17; c++) {
        float v = c < 16 ? aw[c] : ab;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_w[c][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 17) {
        float t = 0.f;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += s_w[threadIdx.x][k];
        if (threadIdx.x < 16) {
            if (threadIdx.x < C) atomicAdd(dw + threadIdx.x, t);
        } else {
            atomicAdd(db, t);
        }
    }
}

// target log-depth and weight from a render: depth D = sum w z and final T;
// the mean depth D / (1 - T) is the target where 1 - T >= 0.5
__global__ void k_depth_target(size_t P, const float* __restrict__ D, const float* __restrict__ T,
                               float* __restrict__ target, float* __restrict__ weight)
{
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        const float a = 1.f - T[p];
        const bool ok = a >= 0.5f && D[p] > 0.f;
        target[p] = ok ? logf(D[p] / a) : 0.f;
        weight[p] = ok ? 1.f : 0.f;
    }
}

// L = (1/P) sum_p w_p |pred_p - target_p|; grad = w sign(.) / P
__global__ void __launch_bounds__(256)
k_depth_l1(size_t P, const float* __restrict__ pred, const float* __restrict__ target,
           const float* __restrict__ weight, float* __restrict__ loss, float* __restrict__ grad)
{
    const float inv = 1.f / (float)P;
    float acc = 0.f;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        const float e = pred[p] - target[p];
        const float wt = weight[p];
        acc += wt * fabsf(e);
        grad[p] = wt * inv * (float)((e > 0.f) - (e < 0.f));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float s[8];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += s[k];
        atomicAdd(loss, t * inv);
    }
}

// Adam on FP32 masters, optional BF16 copy of the updated parameters
__global__ void k_adam(size_t n, float* __restrict__ p, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, bf16* __restrict__ p16,
                       float lr, float b1, float b2, float eps, float bc1, float bc2)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        p[i] = pi;
        if (p16) p16[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void k_to_bf16(size_t n, const float* __restrict__ x, bf16* __restrict__ y)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

}  // namespace gevo

using namespace gevo;

#define GEVO_LAUNCHED() \
    do { GEVO_CHECK_LAUNCH(); return GEVO_OK; } while (0)

// The convolution kernels keep a pixel's (y, x) as y << 16 | x and pixel
// indices in 32 bits.
static bool conv_sizes_ok(int32_t nb, int32_t H, int32_t W)
{
    return H < 32768 && W < 65536 && (int64_t)nb * H * W < ((int64_t)1 << 31);
}

extern "C" {

gevo_status gevo_conv3x3(int32_t nb, int32_t H, int32_t W, int32_t Cin, const void* X, int32_t Cout,
                         const void* Wt, const float* bias, void* Y, int32_t ldy, int32_t out_bf16,
                         int32_t relu, float beta, void* workspace, void* stream)
{
    if (nb <= 0 || H <= 0 || W <= 0 || Cin <= 0 || Cin % 8 || Cout <= 0 || !X || !Wt || !Y ||
        !workspace || ldy < Cout || !gevo_aligned(X, 16) || !gevo_aligned(Wt, 16) ||
        !conv_sizes_ok(nb, H, W))
        return GEVO_ERR_INVALID;
    return conv3x3_bf16(nb, H, W, Cin, X, Cout, Wt, Y, ldy, out_bf16, bias, relu, beta,
                        reinterpret_cast<uint32_t*>(workspace), (cudaStream_t)stream);
}

gevo_status gevo_conv3x3_wgrad(int32_t nb, int32_t H, int32_t W, int32_t Cin, const void* X,
                               int32_t Cout, const void* dZt, float* dWt, void* workspace,
                               void* stream)
{
    if (nb <= 0 || H <= 0 || W <= 0 || Cin <= 0 || Cin % 8 || Cout <= 0 || Cout % 8 || !X ||
        !dZt || !dWt || !workspace || ((int64_t)nb * H * W) % 8 || !conv_sizes_ok(nb, H, W) ||
        !gevo_aligned(X, 16) || !gevo_aligned(dZt, 16))
        return GEVO_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* err = reinterpret_cast<uint32_t*>(workspace);
    const size_t P = (size_t)nb * H * W;
    const int K9 = 9 * Cin;
    if (cudaMemsetAsync(dWt, 0, sizeof(float) * (size_t)K9 * Cout, st) != cudaSuccess)
        return GEVO_ERR_CUDA;
    // rows of the product are the 9 Cin taps x channels (many: full 128-row MMA
    // tiles), columns the Cout output channels, stored transposed into dW's
    // [Cout][9 Cin] layout; the pixels are split into enough K ranges for about
    // eight CTAs per SM, each at least 512 pixels long
    const size_t mtiles = ((size_t)K9 + 127) / 128;
    const size_t want = ((size_t)sm_count() * 8 + mtiles - 1) / mtiles;
    const int ksplit = (int)std::max<size_t>(2, std::min<size_t>(P / 512, want));
    return conv3x3_wgrad_bf16(nb, H, W, Cin, X, Cout, dZt, dWt, ksplit, err, st);
}

gevo_status gevo_relu_bwd(int64_t P, int32_t C, const float* dY, int32_t lddy, const void* Y,
                          int32_t ldy, void* dZ, void* dZt, float* db, void* stream)
{
    if (P <= 0 || C <= 0 || C > 128 || !dY || !Y || !dZ || !db) return GEVO_ERR_INVALID;
    const int vec = C % 8 == 0 && ldy % 8 == 0 && lddy % 4 == 0 && gevo_aligned(Y, 16) &&
                    gevo_aligned(dY, 16) && gevo_aligned(dZ, 16);
    k_relu_bwd<<<(unsigned)((P + 63) / 64), 256, 0, (cudaStream_t)stream>>>(
        (size_t)P, C, dY, lddy, reinterpret_cast<const bf16*>(Y), ldy, reinterpret_cast<bf16*>(dZ),
        reinterpret_cast<bf16*>(dZt), db, vec);
    GEVO_LAUNCHED();
}

gevo_status gevo_maxpool2(int32_t nb, int32_t H, int32_t W, int32_t C, const void* X, int32_t ldx,
                          void* Y, void* stream)
{
    if (nb <= 0 || H % 2 || W % 2 || C <= 0 || !X || !Y) return GEVO_ERR_INVALID;
    const size_t n = (size_t)nb * (H / 2) * (W / 2) * C;
    auto kern = n < ((size_t)1 << 31) ? k_maxpool2<uint32_t> : k_maxpool2<size_t>;
    kern<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(
        nb, H, W, C, reinterpret_cast<const bf16*>(X), ldx, reinterpret_cast<bf16*>(Y));
    GEVO_LAUNCHED();
}

gevo_status gevo_maxpool2_bwd(int32_t nb, int32_t H, int32_t W, int32_t C, const void* X,
                              int32_t ldx, const float* dY, float* dX, int32_t lddx, float beta,
                              void* stream)
{
    if (nb <= 0 || H % 2 || W % 2 || C <= 0 || !X || !dY || !dX) return GEVO_ERR_INVALID;
    const size_t n = (size_t)nb * (H / 2) * (W / 2) * C;
    auto kern = n < ((size_t)1 << 31) ? k_maxpool2_bwd<uint32_t> : k_maxpool2_bwd<size_t>;
    kern<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(
        nb, H, W, C, reinterpret_cast<const bf16*>(X), ldx, dY, dX, lddx, beta);
    GEVO_LAUNCHED();
}

gevo_status gevo_upsample2(int32_t nb, int32_t h, int32_t w, int32_t C, const void* X, void* Y,
                           int32_t ldy, void* stream)
{
    if (nb <= 0 || h <= 0 || w <= 0 || C <= 0 || !X || !Y) return GEVO_ERR_INVALID;
    const size_t n = (size_t)nb * 4 * h * w * C;
    if (C % 8 == 0 && ldy % 8 == 0 && gevo_aligned(X, 16) && gevo_aligned(Y, 16) &&
        n / 8 < ((size_t)1 << 31))
        k_upsample2_vec<<<grid_for(n / 8), 256, 0, (cudaStream_t)stream>>>(
            nb, h, w, C, reinterpret_cast<const bf16*>(X), reinterpret_cast<bf16*>(Y), ldy);
    else
        k_upsample2<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(
            nb, h, w, C, reinterpret_cast<const bf16*>(X), reinterpret_cast<bf16*>(Y), ldy);
    GEVO_LAUNCHED();
}

gevo_status gevo_upsample2_bwd(int32_t nb, int32_t h, int32_t w, int32_t C, const float* dY,
                               int32_t lddy, float* dX, void* stream)
{
    if (nb <= 0 || h <= 0 || w <= 0 || C <= 0 || !dY || !dX) return GEVO_ERR_INVALID;
    const size_t n = (size_t)nb * h * w * C;
    if (C % 4 == 0 && lddy % 4 == 0 && gevo_aligned(dY, 16) && gevo_aligned(dX, 16) &&
        n / 4 < ((size_t)1 << 31))
        k_upsample2_bwd_vec<<<grid_for(n / 4), 256, 0, (cudaStream_t)stream>>>(nb, h, w, C, dY,
                                                                              lddy, dX);
    else
        k_upsample2_bwd<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(nb, h, w, C, dY, lddy, dX);
    GEVO_LAUNCHED();
}

gevo_status gevo_flip3x3(int32_t Cout, int32_t Cin, const void* Wt, void* Wf, void* stream)
{
    if (Cout <= 0 || Cin <= 0 || !Wt || !Wf) return GEVO_ERR_INVALID;
    k_flip3x3<<<grid_for((size_t)Cout * 9 * Cin), 256, 0, (cudaStream_t)stream>>>(
        Cout, Cin, reinterpret_cast<const bf16*>(Wt), reinterpret_cast<bf16*>(Wf));
    GEVO_LAUNCHED();
}

gevo_status gevo_rgb_pack(int32_t nb, int32_t H, int32_t W, const float* rgb, void* X, void* stream)
{
    if (nb <= 0 || H <= 0 || W <= 0 || !rgb || !X || !gevo_aligned(X, 16)) return GEVO_ERR_INVALID;
    const size_t P = (size_t)nb * H * W;
    k_rgb_pack<<<grid_for(P), 256, 0, (cudaStream_t)stream>>>(P, H * W, rgb, reinterpret_cast<bf16*>(X));
    GEVO_LAUNCHED();
}

gevo_status gevo_head_fwd(int64_t P, int32_t C, const void* X, const float* w, const float* b,
                          float* pred, void* stream)
{
    if (P <= 0 || C <= 0 || C > 16 || !X || !w || !b || !pred) return GEVO_ERR_INVALID;
    k_head_fwd<<<grid_for((size_t)P), 256, 0, (cudaStream_t)stream>>>((size_t)P, C,
                                                                      reinterpret_cast<const bf16*>(X), w, b, pred);
    GEVO_LAUNCHED();
}

gevo_status gevo_head_bwd(int64_t P, int32_t C, const void* X, const float* w, const float* dpred,
                          float* dX, float* dw, float* db, void* stream)
{
    if (P <= 0 || C <= 0 || C > 16 || !X || !w || !dpred || !dX || !dw || !db) return GEVO_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(dw, 0, sizeof(float) * C, st) != cudaSuccess ||
        cudaMemsetAsync(db, 0, sizeof(float), st) != cudaSuccess)
        return GEVO_ERR_CUDA;
    k_head_bwd<<<grid_for((size_t)P), 256, 0, st>>>((size_t)P, C, reinterpret_cast<const bf16*>(X),
                                                    w, dpred, dX, dw, db);
    GEVO_LAUNCHED();
}

gevo_status gevo_depth_target(int64_t P, const float* depth, const float* T_final, float* target,
                              float* weight, void* stream)
{
    if (P <= 0 || !depth || !T_final || !target || !weight) return GEVO_ERR_INVALID;
    k_depth_target<<<grid_for((size_t)P), 256, 0, (cudaStream_t)stream>>>((size_t)P, depth, T_final,
                                                                          target, weight);
    GEVO_LAUNCHED();
}

gevo_status gevo_depth_l1(int64_t P, const float* pred, const float* target, const float* weight,
                          float* loss, float* grad, void* stream)
{
    if (P <= 0 || !pred || !target || !weight || !loss || !grad) return GEVO_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess) return GEVO_ERR_CUDA;
    k_depth_l1<<<grid_for((size_t)P), 256, 0, st>>>((size_t)P, pred, target, weight, loss, grad);
    GEVO_LAUNCHED();
}

gevo_status gevo_adam(int64_t n, float* param, const float* grad, float* m, float* v,
                      void* param_bf16, float lr, float beta1, float beta2, float eps, int32_t step,
                      void* stream)
{
    if (n <= 0 || !param || !grad || !m || !v || step < 1) return GEVO_ERR_INVALID;
    const float bc1 = 1.f - powf(beta1, (float)step), bc2 = 1.f - powf(beta2, (float)step);
    k_adam<<<grid_for((size_t)n), 256, 0, (cudaStream_t)stream>>>(
        (size_t)n, param, grad, m, v, reinterpret_cast<bf16*>(param_bf16), lr, beta1, beta2, eps,
        bc1, bc2);
    GEVO_LAUNCHED();
}

gevo_status gevo_to_bf16(int64_t n, const float* x, void* y, void* stream)
{
    if (n <= 0 || !x || !y) return GEVO_ERR_INVALID;
    k_to_bf16<<<grid_for((size_t)n), 256, 0, (cudaStream_t)stream>>>((size_t)n, x,
                                                                      reinterpret_cast<bf16*>(y));
    GEVO_LAUNCHED();
}

}  // extern "C"
