// BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores (tcgen05 + TMEM),
// the contraction under the learned depth prior's convolutions (implicit GEMM:
// rows = pixels, columns = output channels, depth = 9 x input channels).
//
//   C[M x N] = A[M x K] * B[N x K]^T  (+ bias[N]) (ReLU optional)
//
// A and B are row-major with K contiguous ("K-major").  One CTA of 128 threads
// computes a 128 x BN tile (BN in {16, 32, 64, 128, 256}) over K in slices of
// 64, through a ring of kGemmStages shared-memory stages:
//   1. every thread copies 16-byte pieces of a slice's 128 x 64 block of A and
//      BN x 64 block of B into a stage with asynchronous copies (cp.async,
//      zero-filled outside the matrix), arranged as the canonical no-swizzle
//      K-major layout of 8-row x 16-byte core matrices (core matrices 128 B
//      apart along K, 1 KB apart along M / N); the copies run kGemmStages - 1
//      slices ahead of the tensor core;
//   2. once a slice has landed, one elected thread issues four tcgen05.mma
//      (K = 16 each) that accumulate into a 128-lane x BN-column FP32 tile in
//      tensor memory, and tcgen05.commit arrives on the stage's mbarrier when
//      they have completed;
//   3. a stage is refilled only after its mbarrier shows that the MMAs reading
//      it are done (bounded waits: after ~1 s a CTA records GEVO_ERR_TIMEOUT
//      in the error word and stops issuing);
//   4. the epilogue reads the accumulator with tcgen05.ld (warp w owns lanes
//      32w..32w+31 = rows) and writes FP32 or BF16 with bias and ReLU.
#include <cuda_bf16.h>

#include "gevo_internal.cuh"

namespace gevo {

constexpr int kGemmBM = 128;
constexpr int kGemmBK = 64;
// two stages: the layers' K is short (3-18 slices) and more resident CTAs hide
// the gathers' latency better than a deeper ring (measured: 2 > 3 > 4 stages)
constexpr int kGemmStages = 2;
constexpr long long kWaitLimit = 1ll << 22;    // try_wait rounds before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start >> 4 (bits 0-13), leading-dimension
// byte offset >> 4 (16-29), stride byte offset >> 4 (32-45), descriptor version
// 1 (bit 46), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B
// BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: true if the phase completed.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (long long it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(mbar, parity)) return true;
    return false;
}

template <int NCOL>
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// 16-byte asynchronous global -> shared copy; a piece outside the matrix is
// zero-filled (source size 0: nothing is read, the address given is the
// matrix base).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Copies rows [row0, row0 + ROWS) x columns [k0, k0 + 64) of a K-major bf16
// matrix into the core-matrix layout at shared address `dst`, zero-filling
// outside the matrix.
template <int ROWS>
__device__ __forceinline__ void stage_tile(const __nv_bfloat16* __restrict__ src, int ld, int nrows,
                                           int K, int row0, int k0, uint32_t dst)
{
    constexpr int CHUNKS = ROWS * (kGemmBK / 8);      // 16-byte pieces
    for (int c = threadIdx.x; c < CHUNKS; c += blockDim.x) {
        const int r = c / (kGemmBK / 8);
        const int kg = c % (kGemmBK / 8);
        const int gr = row0 + r, gk = k0 + kg * 8;
        // K is a multiple of 8, so a piece is all in or all out
        const bool in = gr < nrows && gk < K;
        const int off = (r >> 3) * 1024 + kg * 128 + (r & 7) * 16;
        cp_async16(dst + off, in ? src + (size_t)gr * ld + gk : src, in);
    }
}

// Implicit im2col of a 3x3, stride-1, zero-padded convolution over an NHWC
// activation X[nb][H][W][C] (C a multiple of 8): row r = pixel (b, y, x),
// column k = (tap, c) with tap = 3 ky + kx.  One 16-byte piece is 8 consecutive
// channels of one neighbour, contiguous in NHWC.
struct ConvA {
    const __nv_bfloat16* X;
    int H, W, C;
};

// Thread t stages the 16-byte pieces (row t / 8 + 16 j, column group t % 8),
// j < 8, of every slice: the rows' (y, x) are decomposed once per CTA (yx[j] =
// y << 16 | x, or -1 past the last row), and the slice's tap and channel once
// per slice, so no integer division runs per piece.
constexpr int kConvRowsPerThread = kGemmBM * (kGemmBK / 8) / 128;   // 8

__device__ __forceinline__ void conv_rows(const ConvA& cv, int M, int row0, int yx[kConvRowsPerThread])
{
#pragma unroll
    for (int j = 0; j < kConvRowsPerThread; j++) {
        const int gr = row0 + (int)(threadIdx.x >> 3) + 16 * j;
        yx[j] = -1;
        if (gr < M) {
            const int x = gr % cv.W, y = (gr / cv.W) % cv.H;
            yx[j] = (y << 16) | x;
        }
    }
}

__device__ __forceinline__ void stage_conv_tile(const ConvA& cv, int K, int row0, int k0,
                                                const int yx[kConvRowsPerThread], uint32_t dst)
{
    const int kg = threadIdx.x & 7;
    const int gk = k0 + kg * 8;
    const bool kin = gk < K;
    const int tap = kin ? gk / cv.C : 0;
    const int ch = gk - tap * cv.C;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const ptrdiff_t shift = ((ptrdiff_t)dy * cv.W + dx) * cv.C + ch;
#pragma unroll
    for (int j = 0; j < kConvRowsPerThread; j++) {
        const int r = (int)(threadIdx.x >> 3) + 16 * j;
        const int y = yx[j] >> 16, x = yx[j] & 0xffff;
        const bool in = kin && yx[j] >= 0 && (unsigned)(y + dy) < (unsigned)cv.H &&
                        (unsigned)(x + dx) < (unsigned)cv.W;
        const __nv_bfloat16* p = in ? cv.X + (ptrdiff_t)(row0 + r) * cv.C + shift : cv.X;
        const int off = (r >> 3) * 1024 + kg * 128 + (r & 7) * 16;
        cp_async16(dst + off, p, in);
    }
}

// Weight-gradient operand without a materialised im2col: rows m = (tap, ci)
// (m = tap Cin + ci, tap = 3 ky + kx), depth k = pixel p, element
// X[p + (ky - 1) W + (kx - 1)][ci] (zero outside the image).  A 16-byte piece
// of X (8 channels of one pixel) is a column of 8 rows of one core matrix, so it
// is scattered as 8 two-byte stores.  Thread t takes pixel column t % 64 and
// row groups t / 64 + 2 j, j < 8; the rows' (tap, ci) are decomposed once per
// CTA (wr[j] = tap << 16 | ci, or -1 past the last row), the pixel once per
// slice.
__device__ __forceinline__ void wgrad_rows(const ConvA& cv, int M, int row0, int wr[8])
{
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const int m = row0 + 8 * ((int)(threadIdx.x >> 6) + 2 * j);
        wr[j] = -1;
        if (m < M) {
            const int tap = m / cv.C;
            wr[j] = (tap << 16) | (m - tap * cv.C);
        }
    }
}

// Loads the pieces of one slice into registers (issued a slice ahead, so their
// latency overlaps the wait for the previous slice) ...
__device__ __forceinline__ void wgrad_fetch(const ConvA& cv, int P, int k0, const int wr[8],
                                            uint4 pa[8])
{
    const int p = k0 + (int)(threadIdx.x & 63);
    int y = -1, x = 0;
    if (p < P) {
        x = p % cv.W;
        y = (p / cv.W) % cv.H;
    }
#pragma unroll
    for (int j = 0; j < 8; j++) {
        pa[j] = make_uint4(0u, 0u, 0u, 0u);
        if (wr[j] >= 0 && y >= 0) {
            const int tap = wr[j] >> 16, ci = wr[j] & 0xffff;
            const int dy = tap / 3 - 1, dx = tap % 3 - 1;
            if ((unsigned)(y + dy) < (unsigned)cv.H && (unsigned)(x + dx) < (unsigned)cv.W)
                pa[j] = *reinterpret_cast<const uint4*>(cv.X + ((size_t)p + dy * cv.W + dx) * cv.C + ci);
        }
    }
}

// ... and scatters them into a stage: piece j is rows 8 g .. 8 g + 7 (g = t / 64
// + 2 j) of pixel column t % 64.  This operand's core matrices sit kWgradLBO =
// 144 bytes apart along K (8-row groups kWgradSBO = 8 x 144 apart) instead of
// 128: the 32 lanes of a store then hit 16 distinct banks, two lanes per word,
// where 128 put four columns on one bank.
constexpr int kWgradLBO = 144;
constexpr int kWgradSBO = 8 * kWgradLBO;

__device__ __forceinline__ void wgrad_store(const uint4 pa[8], unsigned char* dst)
{
    const int kk = threadIdx.x & 63;
    unsigned char* col = dst + (kk >> 3) * kWgradLBO + (kk & 7) * 2;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        unsigned char* d = col + ((int)(threadIdx.x >> 6) + 2 * j) * kWgradSBO;
        const uint32_t w[4] = {pa[j].x, pa[j].y, pa[j].z, pa[j].w};
#pragma unroll
        for (int i = 0; i < 4; i++) {
            *reinterpret_cast<uint16_t*>(d + (2 * i) * 16) = (uint16_t)(w[i] & 0xffffu);
            *reinterpret_cast<uint16_t*>(d + (2 * i + 1) * 16) = (uint16_t)(w[i] >> 16);
        }
    }
}

// Operand modes of k_gemm_bf16.
constexpr int kModePlain = 0;   // A a K-major matrix
constexpr int kModeConv = 1;    // A the implicit im2col of a 3x3 convolution
constexpr int kModeWgrad = 2;   // A the implicit transposed im2col (weight gradient)

template <int BN, int MODE>
__global__ void __launch_bounds__(128)
k_gemm_bf16(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int lda, ConvA cv,
            const __nv_bfloat16* __restrict__ B, int ldb, void* __restrict__ C, int ldc,
            int out_bf16, const float* __restrict__ bias, int relu, float beta, int ksplit,
            uint32_t* __restrict__ err, int trans_c)
{
    constexpr int TMEM_COLS = BN < 32 ? 32 : BN;
    constexpr int S = kGemmStages;
    // A block (16 KB; 18 KB padded for the weight gradient), then B block
    constexpr uint32_t A_BYTES = MODE == kModeWgrad ? (kGemmBM / 8) * kWgradSBO : kGemmBM * kGemmBK * 2;
    constexpr uint32_t STAGE = A_BYTES + BN * kGemmBK * 2;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long s_mbar[S];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.x * kGemmBM, col0 = blockIdx.y * BN;
    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int i = 0; i < S; i++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar[i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    constexpr uint32_t idesc = idesc_bf16(kGemmBM, BN);
    const uint32_t base = smem_u32(smem);

    // split-K: CTA z of ksplit handles K slices [kc0, kc1)
    const int nk_all = (K + kGemmBK - 1) / kGemmBK;
    const int per = (nk_all + ksplit - 1) / ksplit;
    const int kc0 = min(nk_all, (int)blockIdx.z * per), kc1 = min(nk_all, kc0 + per);
    const int nk = kc1 - kc0;
    int yx[kConvRowsPerThread];
    if (MODE == kModeConv) conv_rows(cv, M, row0, yx);
    if (MODE == kModeWgrad) wgrad_rows(cv, M, row0, yx);
    uint4 pa[MODE == kModeWgrad ? 8 : 1];   // the weight gradient's next A slice
    auto load = [&](int i) {   // slice kc0 + i into stage i % S
        const uint32_t st = base + (uint32_t)(i % S) * STAGE;
        const int k0 = (kc0 + i) * kGemmBK;
        if (MODE == kModeConv) {
            stage_conv_tile(cv, K, row0, k0, yx, st);
        } else if (MODE == kModeWgrad) {
            // A of this slice is in registers: store it, then fetch the next one
            wgrad_store(pa, smem + (size_t)(i % S) * STAGE);
            if (i + 1 < nk) wgrad_fetch(cv, K, k0 + kGemmBK, yx, pa);
        } else {
            stage_tile<kGemmBM>(A, lda, M, K, row0, k0, st);
        }
        stage_tile<BN>(B, ldb, N, K, col0, k0, st + A_BYTES);
    };
    if (MODE == kModeWgrad && nk > 0) wgrad_fetch(cv, K, kc0 * kGemmBK, yx, pa);
    // the copies run S - 1 slices ahead; every iteration commits one group
    // (possibly empty) so that group i always holds slice i
#pragma unroll
    for (int i = 0; i < S - 1; i++) {
        if (i < nk) load(i);
        cp_async_commit();
    }
    int issued = 0;
    for (int i = 0; i < nk; i++) {
        cp_async_wait<S - 2>();                       // slice i has landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (s_fail) break;
        const int s = i % S;
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t aBase = base + (uint32_t)s * STAGE, bBase = aBase + A_BYTES;
#pragma unroll
            for (int k16 = 0; k16 < kGemmBK / 16; k16++) {
                const uint64_t da = MODE == kModeWgrad
                                        ? smem_desc(aBase + k16 * 2 * kWgradLBO, kWgradLBO, kWgradSBO)
                                        : smem_desc(aBase + k16 * 256, 128, 1024);
                const uint64_t db = smem_desc(bBase + k16 * 256, 128, 1024);
                mma_bf16(tmem, da, db, idesc, (i > 0 || k16 > 0) ? 1u : 0u);
            }
            mma_commit(smem_u32(&s_mbar[s]));
        }
        issued = i + 1;
        const int j = i + S - 1;
        if (j < nk) {
            const int sj = j % S;
            // stage sj was last read by the MMAs of slice j - S (its use (j - S) / S)
            bool ok = true;
            if (j >= S) ok = mbar_wait(smem_u32(&s_mbar[sj]), (uint32_t)((j - S) / S) & 1u);
            if (ok) {
                load(j);
            } else {
                s_fail = 1;
                atomicOr(err, kErrTimeout);
            }
        }
        cp_async_commit();
    }
    cp_async_wait<0>();
    // the last commit arrives once every MMA issued before it has completed
    if (issued > 0) {
        const int last = issued - 1;
        if (!mbar_wait(smem_u32(&s_mbar[last % S]), (uint32_t)(last / S) & 1u)) {
            s_fail = 1;
            atomicOr(err, kErrTimeout);
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (!s_fail && nk > 0) {
        // epilogue: warp w reads accumulator lanes (rows) 32w .. 32w + 31
        const int r = row0 + warp * 32 + lane;
        // whole 16-column groups of a row are stored as 16-byte vectors when the
        // rows keep 16-byte alignment
        const bool vec_ok = ((uintptr_t)C % 16 == 0) && (ldc % (out_bf16 ? 8 : 4) == 0);
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16<16>(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (r < M && ksplit <= 1 && col0 + c0 + 16 <= N && vec_ok) {
                // 16 whole columns of this row: bias, beta, ReLU, then 16-byte
                // stores (one row's 16 values are contiguous)
                const int cb = col0 + c0;
#pragma unroll
                for (int i = 0; i < 16; i++)
                    if (bias) v[i] += bias[cb + i];
                if (out_bf16) {
                    uint4* o = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(C) +
                                                        (size_t)r * ldc + cb);
                    uint32_t w[8];
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const uint4 old = beta != 0.f ? o[h] : make_uint4(0u, 0u, 0u, 0u);
                        const uint32_t ow[4] = {old.x, old.y, old.z, old.w};
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            float x0 = v[8 * h + 2 * q], x1 = v[8 * h + 2 * q + 1];
                            if (beta != 0.f) {
                                x0 += beta * __uint_as_float(ow[q] << 16);
                                x1 += beta * __uint_as_float(ow[q] & 0xffff0000u);
                            }
                            if (relu) { x0 = fmaxf(x0, 0.f); x1 = fmaxf(x1, 0.f); }
                            const __nv_bfloat162 pr = __floats2bfloat162_rn(x0, x1);
                            w[4 * h + q] = *reinterpret_cast<const uint32_t*>(&pr);
                        }
                    }
                    o[0] = make_uint4(w[0], w[1], w[2], w[3]);
                    o[1] = make_uint4(w[4], w[5], w[6], w[7]);
                } else {
                    float4* o = reinterpret_cast<float4*>(reinterpret_cast<float*>(C) + (size_t)r * ldc + cb);
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        float4 x = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                        if (beta != 0.f) {
                            const float4 old = o[q];
                            x.x += beta * old.x; x.y += beta * old.y;
                            x.z += beta * old.z; x.w += beta * old.w;
                        }
                        if (relu) {
                            x.x = fmaxf(x.x, 0.f); x.y = fmaxf(x.y, 0.f);
                            x.z = fmaxf(x.z, 0.f); x.w = fmaxf(x.w, 0.f);
                        }
                        o[q] = x;
                    }
                }
            } else if (r < M) {
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    const int c = col0 + c0 + i;
                    if (c < N) {
                        float x = v[i];
                        if (ksplit > 1) {   // split-K partial: FP32 atomic accumulation
                            // (trans_c: C^T is stored, element (r, c) at c * ldc + r, so
                            // the lanes' consecutive rows are consecutive addresses)
                            atomicAdd(reinterpret_cast<float*>(C) +
                                          (trans_c ? (size_t)c * ldc + r : (size_t)r * ldc + c), x);
                            continue;
                        }
                        if (bias) x += bias[c];
                        if (out_bf16) {
                            __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(C) + (size_t)r * ldc + c;
                            if (beta != 0.f) x += beta * __bfloat162float(*o);
                            if (relu) x = fmaxf(x, 0.f);
                            *o = __float2bfloat16_rn(x);
                        } else {
                            float* o = reinterpret_cast<float*>(C) + (size_t)r * ldc + c;
                            if (beta != 0.f) x += beta * *o;
                            if (relu) x = fmaxf(x, 0.f);
                            *o = x;
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
}

template <int BN, int MODE>
static gevo_status launch_gemm(int M, int N, int K, const __nv_bfloat16* A, int lda, ConvA cv,
                               const __nv_bfloat16* B, int ldb, void* C, int ldc, int out_bf16,
                               const float* bias, int relu, float beta, int ksplit, uint32_t* err,
                               cudaStream_t st, int trans_c)
{
    const size_t a_bytes = MODE == kModeWgrad ? (kGemmBM / 8) * kWgradSBO : kGemmBM * kGemmBK * 2;
    const size_t smem = (size_t)kGemmStages * (a_bytes + BN * kGemmBK * 2);
    // set on every launch: a host-only call of about a microsecond, correct for
    // whichever device is current and free of shared state between host threads
    cudaFuncSetAttribute(k_gemm_bf16<BN, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    dim3 grid((M + kGemmBM - 1) / kGemmBM, (N + BN - 1) / BN, ksplit);
    k_gemm_bf16<BN, MODE><<<grid, 128, smem, st>>>(M, N, K, A, lda, cv, B, ldb, C, ldc, out_bf16,
                                                   bias, relu, beta, ksplit, err, trans_c);
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}

template <int MODE>
static gevo_status gemm_dispatch(int M, int N, int K, const __nv_bfloat16* a, int lda, ConvA cv,
                                 const __nv_bfloat16* b, int ldb, void* C, int ldc, int out_bf16,
                                 const float* bias, int relu, float beta, int ksplit,
                                 uint32_t* err, cudaStream_t st, int trans_c = 0)
{
    if (N <= 16) return launch_gemm<16, MODE>(M, N, K, a, lda, cv, b, ldb, C, ldc, out_bf16, bias, relu, beta, ksplit, err, st, trans_c);
    if (N <= 32) return launch_gemm<32, MODE>(M, N, K, a, lda, cv, b, ldb, C, ldc, out_bf16, bias, relu, beta, ksplit, err, st, trans_c);
    if (N <= 64) return launch_gemm<64, MODE>(M, N, K, a, lda, cv, b, ldb, C, ldc, out_bf16, bias, relu, beta, ksplit, err, st, trans_c);
    if (N <= 128) return launch_gemm<128, MODE>(M, N, K, a, lda, cv, b, ldb, C, ldc, out_bf16, bias, relu, beta, ksplit, err, st, trans_c);
    return launch_gemm<256, MODE>(M, N, K, a, lda, cv, b, ldb, C, ldc, out_bf16, bias, relu, beta, ksplit, err, st, trans_c);
}

gevo_status gemm_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb, void* C,
                      int ldc, int out_bf16, const float* bias, int relu, float beta, int ksplit,
                      uint32_t* err, cudaStream_t st, int trans_c)
{
    if (trans_c && ksplit <= 1) return GEVO_ERR_INVALID;   // transposed store: split-K path only
    ConvA cv{nullptr, 0, 0, 0};
    return gemm_dispatch<kModePlain>(M, N, K, reinterpret_cast<const __nv_bfloat16*>(A), lda, cv,
                                reinterpret_cast<const __nv_bfloat16*>(B), ldb, C, ldc, out_bf16,
                                bias, relu, beta, ksplit, err, st, trans_c);
}

gevo_status conv3x3_bf16(int nb, int H, int W, int Cin, const void* X, int Cout, const void* Wt,
                         void* Y, int ldy, int out_bf16, const float* bias, int relu, float beta,
                         uint32_t* err, cudaStream_t st)
{
    ConvA cv{reinterpret_cast<const __nv_bfloat16*>(X), H, W, Cin};
    return gemm_dispatch<kModeConv>(nb * H * W, Cout, 9 * Cin, nullptr, 0, cv,
                               reinterpret_cast<const __nv_bfloat16*>(Wt), 9 * Cin, Y, ldy,
                               out_bf16, bias, relu, beta, 1, err, st);
}

// dWt[co][(tap, ci)] = sum_p dZt[co][p] X[p + shift(tap)][ci]: rows 9 Cin, columns
// Cout, depth P pixels, split over ksplit CTAs and summed with FP32 atomics into
// the transposed (Wt-layout) result, which the caller zeroes.
gevo_status conv3x3_wgrad_bf16(int nb, int H, int W, int Cin, const void* X, int Cout,
                               const void* dZt, float* dWt, int ksplit, uint32_t* err,
                               cudaStream_t st)
{
    ConvA cv{reinterpret_cast<const __nv_bfloat16*>(X), H, W, Cin};
    return gemm_dispatch<kModeWgrad>(9 * Cin, Cout, nb * H * W, nullptr, 0, cv,
                                     reinterpret_cast<const __nv_bfloat16*>(dZt), nb * H * W, dWt,
                                     9 * Cin, 0, nullptr, 0, 1.f, ksplit, err, st, 1);
}

}  // namespace gevo

extern "C" gevo_status gevo_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, int32_t lda,
                                      const void* B, int32_t ldb, void* C, int32_t ldc,
                                      int32_t out_bf16, const float* bias, int32_t relu, float beta,
                                      void* workspace, void* stream)
{
    if (M < 0 || N < 0 || K <= 0 || !A || !B || !C || !workspace || K % 8 != 0 || lda % 8 != 0 ||
        ldb % 8 != 0 || lda < K || ldb < K || ldc < N || !gevo_aligned(A, 16) ||
        !gevo_aligned(B, 16))
        return GEVO_ERR_INVALID;
    if (M == 0 || N == 0) return GEVO_OK;
    return gevo::gemm_bf16(M, N, K, A, lda, B, ldb, C, ldc, out_bf16, bias, relu, beta, 1,
                           reinterpret_cast<uint32_t*>(workspace), (cudaStream_t)stream, 0);
}
