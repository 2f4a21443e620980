// Active set of the global stage (Section III-B2): A_t = M~_t u E_t with
// E_t = {g : max_k E_k(g) > eps} over the window's keyframes, E_k(g) the
// per-Gaussian rendering error of Eq. 5 (accumulated by the reverse walk).
// Output: a bit mask (consumed by the masked reverse walk) and the ascending
// list of active indices with its length on the device (consumed by the
// masked projection backward), in three launches and no host round trip:
//   1. k_active_bits: one warp per 32 Gaussians (a ballot is one mask word);
//      each 1024-thread block also writes its population count;
//   2. k_active_scan: one block turns the block counts into exclusive offsets
//      and the total;
//   3. k_active_list: each block writes its active indices at its offset.
#include "../../include/gevo_map.h"
#include "gevo_internal.cuh"

namespace gevo {

constexpr int kActBlock = 1024;   // Gaussians per block = 32 mask words

__global__ void __launch_bounds__(kActBlock)
k_active_bits(int V, int n, const float* __restrict__ E, float eps, const uint32_t* __restrict__ force,
              uint32_t* __restrict__ bits, uint32_t* __restrict__ block_count)
{
    __shared__ uint32_t s_cnt[kActBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = blockIdx.x * kActBlock + threadIdx.x;
    const int w = g >> 5;
    bool a = false;
    if (g < n) {
        for (int v = 0; v < V && !a; v++) a = E[(size_t)v * n + g] > eps;
        if (force && ((__ldg(force + w) >> lane) & 1u)) a = true;
    }
    const uint32_t word = __ballot_sync(0xffffffffu, a);
    if (lane == 0) {
        if (w < (n + 31) / 32) bits[w] = word;
        s_cnt[warp] = __popc(word);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < kActBlock / 32; i++) t += s_cnt[i];
        block_count[blockIdx.x] = t;
    }
}

// counts[1 + b] <- sum of block counts before b; counts[0] <- total.
__global__ void __launch_bounds__(1024) k_active_scan(int nb, uint32_t* __restrict__ counts)
{
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t x = i < nb ? counts[1 + i] : 0u;
        uint32_t inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            uint32_t t = s_w[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            s_w[lane] = t;   // inclusive over warps
        }
        __syncthreads();
        const uint32_t carry = s_carry;
        const uint32_t excl = carry + (warp > 0 ? s_w[warp - 1] : 0u) + inc - x;
        if (i < nb) counts[1 + i] = excl;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + s_w[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) counts[0] = s_carry;
}

__global__ void __launch_bounds__(kActBlock)
k_active_list(int n, const uint32_t* __restrict__ bits, const uint32_t* __restrict__ counts,
              uint32_t* __restrict__ list)
{
    __shared__ uint32_t s_cnt[kActBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = blockIdx.x * kActBlock + threadIdx.x;
    const int w = g >> 5;
    const uint32_t word = w < (n + 31) / 32 ? bits[w] : 0u;
    if (lane == 0) s_cnt[warp] = __popc(word);
    __syncthreads();
    uint32_t off = counts[1 + blockIdx.x];
    for (int i = 0; i < warp; i++) off += s_cnt[i];
    if ((word >> lane) & 1u) list[off + __popc(word & ((1u << lane) - 1u))] = (uint32_t)g;
}

// Pruning after the global stage: keep unless a candidate with opacity below
// the threshold.
__global__ void __launch_bounds__(kActBlock)
k_keep_bits(int n, const float* __restrict__ opac, const uint32_t* __restrict__ cand, float thresh,
            uint32_t* __restrict__ bits, uint32_t* __restrict__ block_count)
{
    __shared__ uint32_t s_cnt[kActBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = blockIdx.x * kActBlock + threadIdx.x;
    const int w = g >> 5;
    bool keep = false;
    if (g < n) {
        const bool c = !cand || ((__ldg(cand + w) >> lane) & 1u);
        keep = !(c && opac[g] < thresh);
    }
    const uint32_t word = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) {
        if (w < (n + 31) / 32) bits[w] = word;
        s_cnt[warp] = __popc(word);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < kActBlock / 32; i++) t += s_cnt[i];
        block_count[blockIdx.x] = t;
    }
}

}  // namespace gevo

using namespace gevo;

extern "C" gevo_status gevo_active_set(int32_t n_views, int32_t n, const float* gauss_err, float eps,
                                       const uint32_t* force, uint32_t* active,
                                       uint32_t* active_list, uint32_t* counts, void* stream)
{
    if (n_views < 1 || n < 0 || n > INT32_MAX - kActBlock || !gauss_err || !active ||
        !active_list || !counts)
        return GEVO_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) return cudaMemsetAsync(counts, 0, 4, st) == cudaSuccess ? GEVO_OK : GEVO_ERR_CUDA;
    const int nb = (n + kActBlock - 1) / kActBlock;
    k_active_bits<<<nb, kActBlock, 0, st>>>(n_views, n, gauss_err, eps, force, active, counts + 1);
    GEVO_CHECK_LAUNCH();
    k_active_scan<<<1, 1024, 0, st>>>(nb, counts);
    GEVO_CHECK_LAUNCH();
    k_active_list<<<nb, kActBlock, 0, st>>>(n, active, counts, active_list);
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}

extern "C" gevo_status gevo_prune_keep(int32_t n, const float* opacities, const uint32_t* candidates,
                                       float threshold, uint32_t* keep, uint32_t* keep_list,
                                       uint32_t* counts, void* stream)
{
    if (n < 0 || n > INT32_MAX - kActBlock || !opacities || !keep || !keep_list || !counts)
        return GEVO_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) return cudaMemsetAsync(counts, 0, 4, st) == cudaSuccess ? GEVO_OK : GEVO_ERR_CUDA;
    const int nb = (n + kActBlock - 1) / kActBlock;
    k_keep_bits<<<nb, kActBlock, 0, st>>>(n, opacities, candidates, threshold, keep, counts + 1);
    GEVO_CHECK_LAUNCH();
    k_active_scan<<<1, 1024, 0, st>>>(nb, counts);
    GEVO_CHECK_LAUNCH();
    k_active_list<<<nb, kActBlock, 0, st>>>(n, keep, counts, keep_list);
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}
