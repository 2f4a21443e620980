// Stage a5 (front-to-back alpha blending) and stage a6 (its reverse walk) of the
// splatting renderer R(M, T) GEVO optimises through (Section I "GS"; Section
// III-B Eq. 2, Eq. 3 and the rendered past keyframes of Eq. 6).
//
// Work item = one 16x16 tile of one view.  A block of 256 / PPT threads owns the
// tile; thread t owns pixels (t % 16, (t / 16) * PPT + k), k < PPT, so a warp
// covers a compact 16 x (2 PPT) strip.  The tile's list is staged into shared
// memory in short batches (one record per thread in the blend, half that in the
// reverse walk) gathered by Gaussian id (40-byte records that mostly hit L2);
// each warp then walks, from shared memory, the batch entries that its strip
// can see.  Per-pixel state stays in registers.
//
// Early termination: a pixel stops at the first entry that would push T below
// 1e-4; a thread leaves the batch loop when all its pixels stopped, and the
// block leaves the tile when every thread has (__syncthreads_and per batch).
//
// Exponentials: the conic is pre-scaled by -log2(e)/2 (and -log2(e) for the
// cross term) when staged, so alpha = o * ex2(power2) costs one MUFU.EX2.  The
// backward evaluates the very same expression, so both passes take identical
// skip / clamp / stop decisions.
#include "gevo_internal.cuh"

namespace gevo {



struct Rec {
    float2 xy;
    float4 co;   // pre-scaled conic (a', b', c') and opacity
    float4 rz;   // colour, depth
};

__device__ __forceinline__ float4 prescale(float4 co)
{
    return make_float4(-0.5f * kLog2e * co.x, -kLog2e * co.y, -0.5f * kLog2e * co.z, co.w);
}

// Pixel box outside which alpha = o exp(-d^T Q d / 2) < 1/255 for certain:
// the ellipse d^T Q d <= 2 ln(255 o) has half-extents sqrt(k2 Sigma_xx) and
// sqrt(k2 Sigma_yy), Sigma = Q^-1.  det(Q) uses Kahan's fused 2x2 determinant
// so elongated splats keep full precision; the box is widened by 0.1% + 1 px,
// far more than the binary32 error of the per-pixel test near its threshold
// and the few-ulp error of the approximate reciprocal and square root.
// Returns (xmin, xmax, ymin, ymax); an empty box if o < 1/255.
__device__ __forceinline__ float4 alpha_box(float2 m, float4 co)
{
    // alpha <= o everywhere: o < 1/255 (with a margin for __logf) can never blend
    const float lg = __logf(255.f * co.w);
    if (!(lg > -1e-4f)) return make_float4(1e30f, -1e30f, 1e30f, -1e30f);
    const float k2 = 2.f * fmaxf(lg, 0.f) + 2e-4f;
    const float w = co.y * co.y;
    const float e = __fmaf_rn(-co.y, co.y, w);
    const float det = __fmaf_rn(co.x, co.z, -w) + e;
    const float rdet = rcp_approx(det);
    const float sxx = co.z * rdet, syy = co.x * rdet;
    const float hx = sqrt_approx(k2 * sxx) * 1.001f + 1.f;
    const float hy = sqrt_approx(k2 * syy) * 1.001f + 1.f;
    if (!(det > 0.f) || !(hx < 1e30f) || !(hy < 1e30f))
        return make_float4(-1e30f, 1e30f, -1e30f, 1e30f);   // degenerate: never cull
    return make_float4(m.x - hx, m.x + hx, m.y - hy, m.y + hy);
}

// Which warps of the block may blend this entry at some pixel: warp w covers
// tile columns 0..15 and rows w*rows .. w*rows + rows - 1.  For each such
// strip the minimum of q(d) = a dx^2 + 2 b dx dy + c dy^2, d = mean - pixel, over
// the continuous rectangle spanned by its pixel centres (a lower bound of the
// minimum over the pixels) is compared with 2 ln(255 o), the level below which
// alpha < 1/255: zero if the mean lies inside, else the least of the four
// edge minima (a 1-D quadratic per edge, its vertex clamped to the edge).  The
// threshold is widened by 0.2% + 2e-4 against rounding.  The edge vertex is
// placed with approximate reciprocals: a vertex off by a few ulp raises q by
// c * delta^2 only (second order), far inside that margin; conics with an
// entry at or below 1e-30 take the box test alone.  A strip the bounding
// box of the ellipse overlaps but the ellipse itself misses -- a thin or
// tilted splat crossing a corner -- is culled, which the box alone cannot.
__device__ __forceinline__ uint32_t strip_mask(float2 m, float4 co, float x0, float y0, int nw,
                                               int rows)
{
    const float4 box = alpha_box(m, co);
    if (!(box.x <= box.y)) return 0u;               // o < 1/255: blends nowhere
    const float a = co.x, b = co.y, c = co.z;
    const float lg = __logf(255.f * co.w);
    const float k2 = (2.f * fmaxf(lg, 0.f) + 2e-4f) * 1.002f;
    const bool exact = a > 1e-30f && c > 1e-30f && box.x > -1e29f;   // else box only
    const float ra = rcp_approx(a), rc = rcp_approx(c);
    const float dxl = m.x - (x0 + (float)(kTile - 1)), dxh = m.x - x0;
    const bool in_x = dxl <= 0.f && dxh >= 0.f;
    uint32_t mask = 0u;
    for (int w = 0; w < nw; w++) {
        const float ys0 = y0 + (float)(w * rows), ys1 = ys0 + (float)(rows - 1);
        if (box.w < ys0 || box.z > ys1 || box.y < x0 || box.x > x0 + (float)(kTile - 1)) continue;
        if (!exact) { mask |= 1u << w; continue; }
        const float dyl = m.y - ys1, dyh = m.y - ys0;
        float q = 0.f;
        if (!(in_x && dyl <= 0.f && dyh >= 0.f)) {
            q = 3.0e38f;
            const float ex[2] = {dxl, dxh}, ey[2] = {dyl, dyh};
#pragma unroll
            for (int e = 0; e < 2; e++) {
                const float dx = ex[e];
                const float dy = fminf(fmaxf(-b * dx * rc, dyl), dyh);
                q = fminf(q, a * dx * dx + 2.f * b * dx * dy + c * dy * dy);
                const float dy2 = ey[e];
                const float dx2 = fminf(fmaxf(-b * dy2 * ra, dxl), dxh);
                q = fminf(q, a * dx2 * dx2 + 2.f * b * dx2 * dy2 + c * dy2 * dy2);
            }
        }
        if (q <= k2) mask |= 1u << w;
    }
    return mask;
}


// log2 of the Gaussian falloff at offset (dx, dy) with the pre-scaled conic,
// a' dx^2 + (b' dx + c' dy) dy: a thread's pixels share their column, so
// a' dx^2 and b' dx (power2_col) are formed once per entry and each pixel costs
// two FMAs.  Both passes evaluate exactly this expression.
__device__ __forceinline__ float2 power2_col(const float4& co, float dx)
{
    return make_float2(__fmul_rn(__fmul_rn(co.x, dx), dx), __fmul_rn(co.y, dx));
}

__device__ __forceinline__ float power2_at(const float4& co, float2 col, float dy)
{
    return __fmaf_rn(__fmaf_rn(co.z, dy, col.y), dy, col.x);
}

__device__ __forceinline__ void tile_of(const gevo_layout& L, int tile, int& v, int& x0, int& y0)
{
    v = view_of_tile(L, tile);
    const int local = tile - L.tile_base[v];
    const int tx = L.tiles_x[v];
    x0 = (local % tx) * kTile;
    y0 = (local / tx) * kTile;
}

// ACT: also record, per pixel, where the reverse walk of an active-set
// backward has to start: 1 + the list position of the last blended entry of an
// active Gaussian (0 if none), the transmittance right after it, and the colour
// (with T_final bg) and depth blended behind it.  The colour is summed in two
// parts, up to the last active entry and since it, so that the part behind
// needs no difference of two sums; the bookkeeping runs only at active
// entries (a warp-uniform branch), and the pixel colour is the sum of the two
// parts.
template <int PPT, bool COUNT, bool ACT>
__global__ void __launch_bounds__(256 / PPT)
k_render_fwd(gevo_layout L, int n, const float2* __restrict__ xy, const float4* __restrict__ co,
             const float4* __restrict__ rz, const uint32_t* __restrict__ vals,
             const uint2* __restrict__ ranges, float bg0, float bg1, float bg2,
             float* __restrict__ out_rgb, float* __restrict__ out_d, float* __restrict__ out_T,
             uint32_t* __restrict__ out_nc, uint32_t* __restrict__ out_ne,
             const uint32_t* __restrict__ order, uint32_t* queue, int n_items,
             const uint32_t* __restrict__ active, uint32_t* __restrict__ act_last,
             float* __restrict__ act_T, float4* __restrict__ act_rest,
             uint32_t* __restrict__ out_nb)
{
    constexpr int NT = 256 / PPT;
    // staging batch: one record per thread (measured on the benchmark: 64
    // entries at 64 threads beat 32, 96, 128 and 256 -- a block leaves its tile
    // as soon as all its pixels stopped, which happens early in most lists)
    constexpr int kBatch = NT;
    __shared__ float2 s_xy[kBatch];
    __shared__ float4 s_co[kBatch];
    __shared__ float4 s_rz[kBatch];
    __shared__ uint32_t s_mask[kBatch];
    __shared__ uint32_t s_act[ACT ? kBatch : 1];
    __shared__ uint16_t s_list[NT / 32][kBatch];
    __shared__ uint32_t s_item;
    const int tid = threadIdx.x;
    constexpr int WROWS = 2 * PPT;

    for (int it = 0;; it++) {
        int item;
        if (queue) {
            if (tid == 0) s_item = atomicAdd(queue, 1u);
            __syncthreads();
            item = (int)s_item;
            __syncthreads();
        } else {
            if (it > 0) break;
            item = blockIdx.x;
        }
        if (item >= n_items) break;
        const int tile = order ? (int)order[item] : item;
        int v, x0, y0;
        tile_of(L, tile, v, x0, y0);
        const int W = L.width[v], H = L.height[v];
        const size_t P = (size_t)W * H;
        const int px = x0 + (tid & 15);
        const int py0 = y0 + (tid >> 4) * PPT;
        const uint2 rg = ranges[tile];
        const size_t vbase = (size_t)v * n;

        float T[PPT], C0[PPT], C1[PPT], C2[PPT], Dp[PPT];
        float B0[PPT], B1[PPT], B2[PPT], BD[PPT], Ta[PPT];   // colour, depth through the last active entry
        uint32_t last[PPT], cnt[PPT], la[PPT], nbl[PPT];
        bool done[PPT];
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            T[k] = 1.f; C0[k] = C1[k] = C2[k] = Dp[k] = 0.f;
            last[k] = 0u; cnt[k] = 0u; nbl[k] = 0u;
            done[k] = !(px < W && py0 + k < H);
            if (ACT) { B0[k] = B1[k] = B2[k] = BD[k] = 0.f; Ta[k] = 1.f; la[k] = 0u; }
        }
        const float fpx = (float)px;

        for (uint32_t b = rg.x; b < rg.y; b += kBatch) {
            bool mine = true;
#pragma unroll
            for (int k = 0; k < PPT; k++) mine = mine && done[k];
            if (__syncthreads_and(mine)) break;
            const int nb = (int)min((uint32_t)kBatch, rg.y - b);
            for (int j = tid; j < nb; j += NT) {
                const uint32_t gid = vals[b + j];
                const size_t id = vbase + gid;
                const float2 m = xy[id];
                const float4 c = co[id];
                s_xy[j] = m;
                s_co[j] = prescale(c);
                s_rz[j] = rz[id];
                s_mask[j] = strip_mask(m, c, (float)x0, (float)y0, NT / 32, WROWS);
                if (ACT) s_act[j] = (__ldg(active + (gid >> 5)) >> (gid & 31)) & 1u;
            }
            __syncthreads();
            // the batch entries whose strip mask has this warp's bit, in order: the
            // walk below runs over them without a per-entry mask branch
            const int warp = tid >> 5;
            int nl = 0;
            {
                const uint32_t my_bit = 1u << warp, lt = (1u << (tid & 31)) - 1u;
                for (int r = 0; r < nb; r += 32) {
                    const int jj = r + (tid & 31);
                    const bool in = jj < nb && (s_mask[jj] & my_bit);
                    const uint32_t bal = __ballot_sync(0xffffffffu, in);
                    if (in) s_list[warp][nl + __popc(bal & lt)] = (uint16_t)jj;
                    nl += __popc(bal);
                }
                __syncwarp();
            }
            for (int q = 0; q < nl; q++) {
                bool all = true;
#pragma unroll
                for (int k = 0; k < PPT; k++) all = all && done[k];
                if (all) break;
                const int j = s_list[warp][q];
                const float2 m = s_xy[j];
                const float4 c = s_co[j];
                const float4 r = s_rz[j];
                const float dx = __fsub_rn(m.x, fpx);
                const uint32_t pos1 = b + j - rg.x + 1;
                // the PPT pixels are independent: evaluate them branch-free so
                // their dependency chains interleave
                float p2[PPT], G[PPT];
                const float2 col = power2_col(c, dx);
#pragma unroll
                for (int k = 0; k < PPT; k++) {
                    const float dy = __fsub_rn(m.y, (float)(py0 + k));
                    p2[k] = power2_at(c, col, dy);
                }
#pragma unroll
                for (int k = 0; k < PPT; k++) G[k] = ex2_approx(p2[k]);
#pragma unroll
                for (int k = 0; k < PPT; k++) {
                    const float alpha = fminf(kAlphaMax, __fmul_rn(c.w, G[k]));
                    const bool ok = !done[k] && !(p2[k] > 0.f) && !(alpha < kAlphaMin);
                    const float Tn = __fmaf_rn(-alpha, T[k], T[k]);   // T (1 - alpha), one rounding
                    const bool stop = ok && Tn < kTStop;
                    const bool bl = ok && !stop;
                    done[k] = done[k] || stop;
                    // entries examined = the stopping entry's position (entries
                    // past the stop, masked or not, are not examined)
                    if (COUNT && stop) cnt[k] = pos1;
                    const float w = bl ? __fmul_rn(alpha, T[k]) : 0.f;
                    C0[k] = __fmaf_rn(w, r.x, C0[k]);
                    C1[k] = __fmaf_rn(w, r.y, C1[k]);
                    C2[k] = __fmaf_rn(w, r.z, C2[k]);
                    Dp[k] = __fmaf_rn(w, r.w, Dp[k]);
                    T[k] = bl ? Tn : T[k];
                    last[k] = bl ? pos1 : last[k];
                    if (COUNT) nbl[k] += bl ? 1u : 0u;
                }
                if (ACT && s_act[j]) {
                    // an active entry: move the part since the previous one
                    // into the part up to here (C holds the part since)
#pragma unroll
                    for (int k = 0; k < PPT; k++) {
                        const bool at = last[k] == pos1;   // blended right here
                        B0[k] = at ? __fadd_rn(B0[k], C0[k]) : B0[k];
                        B1[k] = at ? __fadd_rn(B1[k], C1[k]) : B1[k];
                        B2[k] = at ? __fadd_rn(B2[k], C2[k]) : B2[k];
                        BD[k] = at ? __fadd_rn(BD[k], Dp[k]) : BD[k];
                        C0[k] = at ? 0.f : C0[k];
                        C1[k] = at ? 0.f : C1[k];
                        C2[k] = at ? 0.f : C2[k];
                        Dp[k] = at ? 0.f : Dp[k];
                        Ta[k] = at ? T[k] : Ta[k];
                        la[k] = at ? pos1 : la[k];
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int py = py0 + k;
            if (px < W && py < H) {
                const size_t pix = (size_t)py * W + px;
                const size_t gp = (size_t)L.pix_base[v] + pix;
                if (ACT) {
                    // C, Dp hold the part behind the last active entry
                    act_last[gp] = la[k];
                    act_T[gp] = Ta[k];
                    act_rest[gp] = la[k] ? make_float4(__fmaf_rn(T[k], bg0, C0[k]), __fmaf_rn(T[k], bg1, C1[k]),
                                                       __fmaf_rn(T[k], bg2, C2[k]), Dp[k])
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
                    C0[k] = __fadd_rn(B0[k], C0[k]);
                    C1[k] = __fadd_rn(B1[k], C1[k]);
                    C2[k] = __fadd_rn(B2[k], C2[k]);
                    Dp[k] = __fadd_rn(BD[k], Dp[k]);
                }
                float* rgb = out_rgb + 3 * (size_t)L.pix_base[v];
                rgb[pix] = __fmaf_rn(T[k], bg0, C0[k]);
                rgb[P + pix] = __fmaf_rn(T[k], bg1, C1[k]);
                rgb[2 * P + pix] = __fmaf_rn(T[k], bg2, C2[k]);
                out_d[gp] = Dp[k];
                out_T[gp] = T[k];
                out_nc[gp] = last[k];
                if (COUNT) {
                    out_ne[gp] = cnt[k] ? cnt[k] : rg.y - rg.x;   // never stopped: the whole list
                    if (out_nb) out_nb[gp] = nbl[k];
                }
            }
        }
    }
}

// Rows of visible records get zeroed before the reverse walk accumulates.
__global__ void k_zero_grad2d(size_t total, const int* __restrict__ radius, float2* gxy,
                              float4* gco, float4* grz)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        if (radius[i] > 0) {
            gxy[i] = make_float2(0.f, 0.f);
            gco[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            grz[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

// Sums ten per-lane values over the warp by recursive halving: at each of the
// five butterfly levels a lane keeps half of its partial sums and sends the
// other half, so 12 shuffles replace 50.  Afterwards the even lanes with
// `slot` in 0..9 hold the total of value `slot`; other lanes get slot = -1.
__device__ __forceinline__ float warp_reduce10(const float v[10], int& slot)
{
    const int lane = threadIdx.x & 31;
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4, h2 = lane & 2;
    float r[6];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const float keep = h16 ? v[5 + i] : v[i];
        const float send = h16 ? v[i] : v[5 + i];
        r[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    r[5] = 0.f;
    float q[4];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const float keep = h8 ? r[3 + i] : r[i];
        const float send = h8 ? r[i] : r[3 + i];
        q[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    q[3] = 0.f;
    float u[2];
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const float keep = h4 ? q[2 + i] : q[i];
        const float send = h4 ? q[i] : q[2 + i];
        u[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    const float keep = h2 ? u[1] : u[0];
    const float send = h2 ? u[0] : u[1];
    float x = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    const int local = (h4 ? 2 : 0) + (h2 ? 1 : 0);
    const bool valid = !(lane & 1) && (h8 ? local < 2 : local < 3);
    slot = valid ? (h16 ? 5 : 0) + (h8 ? 3 : 0) + local : -1;
    return x;
}

// The same transpose-reduction for 11 values (the 10 gradient sums and the
// error weight of Eq. 5) padded to 12: 13 shuffles.  Slot (h16 ? 6 : 0) +
// (h8 ? 3 : 0) + local on the even lanes with local < 3.
__device__ __forceinline__ float warp_reduce12(const float v[12], int& slot)
{
    const int lane = threadIdx.x & 31;
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4, h2 = lane & 2;
    float r[6];
#pragma unroll
    for (int i = 0; i < 6; i++) {
        const float keep = h16 ? v[6 + i] : v[i];
        const float send = h16 ? v[i] : v[6 + i];
        r[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    float q[4];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const float keep = h8 ? r[3 + i] : r[i];
        const float send = h8 ? r[i] : r[3 + i];
        q[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    q[3] = 0.f;
    float u[2];
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const float keep = h4 ? q[2 + i] : q[i];
        const float send = h4 ? q[i] : q[2 + i];
        u[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    const float keep = h2 ? u[1] : u[0];
    const float send = h2 ? u[0] : u[1];
    float x = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    const int local = (h4 ? 2 : 0) + (h2 ? 1 : 0);
    const bool valid = !(lane & 1) && local < 3;
    slot = valid ? (h16 ? 6 : 0) + (h8 ? 3 : 0) + local : -1;
    return x;
}

// EXT adds the per-Gaussian error of Eq. 5 (pix_err -> gauss_err) and the
// active-set mask: inactive entries (a warp-uniform property, the entry is the
// same for the whole warp) only recover T and the suffix colour.
template <int PPT, bool DD, bool DT, bool EXT>
__global__ void __launch_bounds__(256 / PPT)
k_render_bwd(gevo_layout L, int n, const float2* __restrict__ xy, const float4* __restrict__ co,
             const float4* __restrict__ rz, const uint32_t* __restrict__ vals,
             const uint2* __restrict__ ranges, float bg0, float bg1, float bg2,
             const float* __restrict__ T_final, const uint32_t* __restrict__ n_contrib,
             const float* __restrict__ dL_drgb, const float* __restrict__ dL_dd,
             const float* __restrict__ dL_dT, float2* __restrict__ g_xy, float4* __restrict__ g_co,
             float4* __restrict__ g_rz, const uint32_t* __restrict__ order, uint32_t* queue,
             int n_items, const float* __restrict__ pix_err, float* __restrict__ gauss_err,
             const uint32_t* __restrict__ active, const uint32_t* __restrict__ act_last,
             const float* __restrict__ act_T, const float4* __restrict__ act_rest)
{
    constexpr int NT = 256 / PPT;
    constexpr int NW = NT / 32;
    // staging batch: half a record per thread (measured on the benchmark: 32
    // entries at 64 threads beat 64, 96, 128 and 256; the walk starts near each
    // warp's last blended position, so short batches waste less)
    constexpr int kBatch = NT >= 64 ? NT / 2 : NT;
    __shared__ float2 s_xy[kBatch];
    __shared__ float4 s_co[kBatch];
    __shared__ float4 s_rz[kBatch];
    __shared__ uint32_t s_mask[kBatch];
    __shared__ uint32_t s_id[kBatch];
    constexpr int NG = EXT ? 11 : 10;   // per-entry sums: 10 gradients (+ the error weight)
    __shared__ float s_g[kBatch][NG];
    __shared__ uint16_t s_list[NW][kBatch];
    __shared__ uint32_t s_item;
    __shared__ uint32_t s_max[NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int WROWS = 2 * PPT;

    for (int it = 0;; it++) {
        int item;
        if (queue) {
            if (tid == 0) s_item = atomicAdd(queue, 1u);
            __syncthreads();
            item = (int)s_item;
            __syncthreads();
        } else {
            if (it > 0) break;
            item = blockIdx.x;
        }
        if (item >= n_items) break;
        const int tile = order ? (int)order[item] : item;
        int v, x0, y0;
        tile_of(L, tile, v, x0, y0);
        const int W = L.width[v], H = L.height[v];
        const size_t P = (size_t)W * H;
        const int px = x0 + (tid & 15);
        const int py0 = y0 + (tid >> 4) * PPT;
        const uint2 rg = ranges[tile];
        const size_t vbase = (size_t)v * n;
        const float fpx = (float)px;

        // Only the projection of the suffix colour and depth S onto the
        // pixel's upstream gradient, Pg = dL/dC . S (+ dL/dD S_D), enters
        // dL/dalpha = T_i (dL/dC . c + dL/dD z - Pg), and it follows
        // S <- S + alpha (c - S) as Pg <- Pg + alpha (q - Pg), q = dL/dC . c +
        // dL/dD z: one scalar per pixel instead of four.
        float T[PPT], Pg[PPT];
        float gC0[PPT], gC1[PPT], gC2[PPT], gD[PPT], gTT[PPT], pe[PPT];
        uint32_t last[PPT];
        uint32_t mymax = 0;
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int py = py0 + k;
            Pg[k] = 0.f;
            if (px < W && py < H) {
                const size_t pix = (size_t)py * W + px;
                const size_t gp = (size_t)L.pix_base[v] + pix;
                const float* g3 = dL_drgb + 3 * (size_t)L.pix_base[v];
                T[k] = T_final[gp];
                last[k] = n_contrib[gp];
                gC0[k] = g3[pix]; gC1[k] = g3[P + pix]; gC2[k] = g3[2 * P + pix];
                gD[k] = DD ? dL_dd[gp] : 0.f;
                gTT[k] = DT ? dL_dT[gp] * T[k] : 0.f;
                pe[k] = (EXT && pix_err) ? pix_err[gp] : 0.f;
                Pg[k] = gC0[k] * bg0 + gC1[k] * bg1 + gC2[k] * bg2;
                if (EXT && act_last) {
                    // start at the last active entry: what lies behind it is
                    // summarised by the transmittance after it and the colour
                    // and depth blended behind it
                    last[k] = act_last[gp];
                    if (last[k]) {
                        const float Ta = act_T[gp];
                        const float4 q = act_rest[gp];
                        T[k] = Ta;
                        Pg[k] = __fdiv_rn(gC0[k] * q.x + gC1[k] * q.y + gC2[k] * q.z + gD[k] * q.w, Ta);
                    }
                }
            } else {
                T[k] = 1.f; last[k] = 0u;
                gC0[k] = gC1[k] = gC2[k] = gD[k] = gTT[k] = pe[k] = 0.f;
            }
            mymax = max(mymax, last[k]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mymax = max(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
        if (lane == 0) s_max[warp] = mymax;
        __syncthreads();
        uint32_t bmax = 0;
#pragma unroll
        for (int w = 0; w < NW; w++) bmax = max(bmax, s_max[w]);

        const uint32_t end = rg.x + bmax;
        for (uint32_t bend = end; bend > rg.x; bend -= min((uint32_t)kBatch, bend - rg.x)) {
            const uint32_t bstart = bend - min((uint32_t)kBatch, bend - rg.x);
            const int nb = (int)(bend - bstart);
            __syncthreads();
            for (int j = tid; j < nb; j += NT) {
                const uint32_t id = vals[bstart + j];
                const size_t gid = vbase + id;
                const float2 m = xy[gid];
                const float4 c = co[gid];
                // ids are < 2^31 (n is an int32): the top bit marks inactive entries
                const bool inactive = EXT && active && !((__ldg(active + (id >> 5)) >> (id & 31)) & 1u);
                s_id[j] = id | (inactive ? 0x80000000u : 0u);
                s_xy[j] = m;
                s_co[j] = prescale(c);
                s_rz[j] = rz[gid];
                s_mask[j] = strip_mask(m, c, (float)x0, (float)y0, NT / 32, WROWS);
#pragma unroll
                for (int q = 0; q < NG; q++) s_g[j][q] = 0.f;
            }
            __syncthreads();
            // entries at or past this warp's last blended position concern no lane
            const uint32_t boff = bstart - rg.x;
            const int jend = mymax > boff ? (int)min((uint32_t)nb, mymax - boff) : 0;
            // the entries below jend whose strip mask has this warp's bit, in order
            // (walked backwards below, without a per-entry mask branch)
            int nl = 0;
            {
                const uint32_t my_bit = 1u << warp, lt = (1u << lane) - 1u;
                for (int r = 0; r < jend; r += 32) {
                    const int jj = r + lane;
                    const bool in = jj < jend && (s_mask[jj] & my_bit);
                    const uint32_t bal = __ballot_sync(0xffffffffu, in);
                    if (in) s_list[warp][nl + __popc(bal & lt)] = (uint16_t)jj;
                    nl += __popc(bal);
                }
                __syncwarp();
            }
            for (int q = nl - 1; q >= 0; q--) {
                const int j = s_list[warp][q];
                const uint32_t pos = boff + j;   // list position
                const float2 m = s_xy[j];
                const float4 c = s_co[j];
                const float dx = __fsub_rn(m.x, fpx);
                float p2[PPT], G[PPT], dyk[PPT];
                const float2 col = power2_col(c, dx);
#pragma unroll
                for (int k = 0; k < PPT; k++) {
                    dyk[k] = __fsub_rn(m.y, (float)(py0 + k));
                    p2[k] = power2_at(c, col, dyk[k]);
                }
#pragma unroll
                for (int k = 0; k < PPT; k++) G[k] = ex2_approx(p2[k]);
                // no warp-wide skip when no pixel uses the entry: the vote
                // separates the test from the update, and measured slower
                float al[PPT];
                bool use[PPT];
#pragma unroll
                for (int k = 0; k < PPT; k++) {
                    al[k] = fminf(kAlphaMax, __fmul_rn(c.w, G[k]));
                    use[k] = pos < last[k] && !(p2[k] > 0.f) && !(al[k] < kAlphaMin);
                }
                const float4 r = s_rz[j];
                const bool act = !EXT || !(s_id[j] >> 31);
                if (EXT && !act) {
                    // inactive: transmittance and suffix colour only (+ the error weight)
                    float a_e = 0.f;
#pragma unroll
                    for (int k = 0; k < PPT; k++) {
                        const float alpha = use[k] ? al[k] : 0.f;
                        const float om = 1.f - alpha;
                        const float Ti = use[k] ? T[k] * rcp_approx(om) : T[k];
                        T[k] = Ti;
                        a_e += alpha * Ti * pe[k];
                        float qc = gC0[k] * r.x + gC1[k] * r.y + gC2[k] * r.z;
                        if (DD) qc += gD[k] * r.w;
                        Pg[k] += alpha * (qc - Pg[k]);
                    }
                    if (pix_err) {
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) a_e += __shfl_xor_sync(0xffffffffu, a_e, o);
                        if ((threadIdx.x & 31) == 0 && a_e != 0.f) atomicAdd(&s_g[j][NG - 1], a_e);
                    }
                    continue;
                }
                // A thread's pixels share the column, so dx is the same for all
                // of them: the conic and mean gradients are linear in the
                // per-pixel dp = dL/dalpha * alpha with coefficients in 1, dy,
                // dy^2, so the pixel loop keeps three moments and the
                // coefficients are applied once per entry.
                float m0 = 0.f, m1 = 0.f, m2 = 0.f, a_o = 0.f;
                float a_r = 0.f, a_g = 0.f, a_b = 0.f, a_z = 0.f, a_e = 0.f;
                // branch-free over the pixels: an unused pixel takes alpha = 0,
                // which leaves T and the suffix unchanged and adds zeros
#pragma unroll
                for (int k = 0; k < PPT; k++) {
                    const float alpha = use[k] ? al[k] : 0.f;
                    const float dy = dyk[k];
                    const float om = 1.f - alpha;
                    const float inv = rcp_approx(om);
                    const float Ti = use[k] ? T[k] * inv : T[k];
                    T[k] = Ti;
                    const float w = alpha * Ti;
                    if (EXT) a_e += w * pe[k];
                    // (c - S) . dL/dC, shared by dL/dalpha = T_i gd
                    // (- dL/dT_final T_final / (1 - alpha)) and the suffix update
                    float qc = gC0[k] * r.x + gC1[k] * r.y + gC2[k] * r.z;
                    if (DD) qc += gD[k] * r.w;
                    const float gd = qc - Pg[k];
                    Pg[k] += alpha * gd;
                    a_r += gC0[k] * w; a_g += gC1[k] * w; a_b += gC2[k] * w;
                    if (DD) a_z += gD[k] * w;
                    // dp = dL/dalpha * alpha on unclamped pixels
                    const bool unclamped = use[k] && __fmul_rn(c.w, G[k]) <= kAlphaMax;
                    float dp;
                    if (DT) {
                        const float dLda = gd * Ti - gTT[k] * inv;
                        a_o += unclamped ? dLda * G[k] : 0.f;
                        dp = unclamped ? dLda * alpha : 0.f;
                    } else {
                        dp = unclamped ? gd * w : 0.f;
                    }
                    const float t = dp * dy;
                    m0 += dp;
                    m1 += t;
                    m2 += t * dy;
                }
                // without dL/dT_final, dL/do = sum dL/dalpha G = m0 / o (alpha = o G
                // on every unclamped pixel), one product per entry
                if (!DT) a_o = m0 * rcp_approx(c.w);
                // d alpha / d(a, b, c) = alpha (-dx^2 / 2, -dx dy, -dy^2 / 2);
                // d alpha / d(mean) = alpha ln2 (2 a' dx + b' dy, 2 c' dy + b' dx)
                // with the pre-scaled conic (a', b', c')
                const float a_ca = -0.5f * dx * dx * m0;
                const float a_cb = -dx * m1;
                const float a_cc = -0.5f * m2;
                const float a_xy0 = kLn2 * (2.f * c.x * dx * m0 + c.y * m1);
                const float a_xy1 = kLn2 * (2.f * c.z * m1 + c.y * dx * m0);
                if (EXT) {
                    const float vals12[12] = {a_xy0, a_xy1, a_ca, a_cb, a_cc, a_o,
                                              a_r,   a_g,   a_b,  a_z,  a_e,  0.f};
                    int slot;
                    const float tot = warp_reduce12(vals12, slot);
                    if (slot >= 0 && slot < NG && tot != 0.f) atomicAdd(&s_g[j][slot], tot);
                } else {
                    const float vals10[10] = {a_xy0, a_xy1, a_ca, a_cb, a_cc, a_o, a_r, a_g, a_b, a_z};
                    int slot;
                    const float tot = warp_reduce10(vals10, slot);
                    if (slot >= 0 && tot != 0.f) atomicAdd(&s_g[j][slot], tot);
                }
            }
            __syncthreads();
            for (int j = tid; j < nb; j += NT) {
                const float* gg = s_g[j];
                if (EXT && pix_err && gg[NG - 1] != 0.f)
                    atomicAdd(gauss_err + vbase + (s_id[j] & 0x7FFFFFFFu), gg[NG - 1]);
                bool nz = false;
#pragma unroll
                for (int q = 0; q < 10; q++) nz = nz || gg[q] != 0.f;
                if (!nz) continue;
                const size_t gid = vbase + (EXT ? (s_id[j] & 0x7FFFFFFFu) : s_id[j]);
                atomicAdd(g_xy + gid, make_float2(gg[0], gg[1]));
                atomicAdd(g_co + gid, make_float4(gg[2], gg[3], gg[4], gg[5]));
                atomicAdd(g_rz + gid, make_float4(gg[6], gg[7], gg[8], gg[9]));
            }
        }
    }
}

static int pick_ppt(const gevo_tuning* t)
{
    const int th = t ? t->threads_per_tile : 256;
    return th == 32 ? 8 : (th == 64 ? 4 : (th == 128 ? 2 : 1));
}

template <int PPT, typename K>
static int persistent_grid(K kernel, const gevo_tuning* t)
{
    int per_sm = t ? t->blocks_per_sm : 0;
    if (per_sm <= 0) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 256 / PPT, 0);
        per_sm = occ > 0 ? occ : 1;
    }
    return per_sm * sm_count();
}

template <int PPT>
static gevo_status launch_fwd(const gevo_layout& L, int n, const gevo_proj& p, const uint32_t* vals,
                              const uint32_t* ranges, const float* bg, float* rgb, float* depth,
                              float* Tf, uint32_t* nc, uint32_t* ne, const gevo_tuning* t,
                              char* ws, cudaStream_t st, const uint32_t* active = nullptr,
                              const gevo_active_state* as = nullptr, uint32_t* nb = nullptr)
{
    const WsLayout w = ws_layout(L, n, 0);
    const uint32_t* order = reinterpret_cast<const uint32_t*>(ws + w.tile_order);
    uint32_t* queue = nullptr;
    int grid = L.total_tiles;
    if (t && t->persistent) {
        queue = reinterpret_cast<uint32_t*>(ws + w.err) + kQueueFwd;
        if (cudaMemsetAsync(queue, 0, 4, st) != cudaSuccess) return GEVO_ERR_CUDA;
    }
    auto kern = as ? k_render_fwd<PPT, false, true>
                   : (ne ? k_render_fwd<PPT, true, false> : k_render_fwd<PPT, false, false>);
    if (queue) grid = std::min(grid, persistent_grid<PPT>(kern, t));
    kern<<<grid, 256 / PPT, 0, st>>>(
        L, n, reinterpret_cast<const float2*>(p.xy), reinterpret_cast<const float4*>(p.conic_opacity),
        reinterpret_cast<const float4*>(p.rgb_depth), vals, reinterpret_cast<const uint2*>(ranges),
        bg[0], bg[1], bg[2], rgb, depth, Tf, nc, ne, order, queue, L.total_tiles, active,
        as ? as->last : nullptr, as ? as->T : nullptr,
        as ? reinterpret_cast<float4*>(as->rest) : nullptr, nb);
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}

template <int PPT, bool EXT>
static auto pick_bwd(bool dd, bool dt)
{
    return dd ? (dt ? k_render_bwd<PPT, true, true, EXT> : k_render_bwd<PPT, true, false, EXT>)
              : (dt ? k_render_bwd<PPT, false, true, EXT> : k_render_bwd<PPT, false, false, EXT>);
}

template <int PPT>
static gevo_status launch_bwd(const gevo_layout& L, int n, const gevo_proj& p, const uint32_t* vals,
                              const uint32_t* ranges, const float* bg, const float* Tf,
                              const uint32_t* nc, const float* gC, const float* gD, const float* gT,
                              const gevo_grad2d& out, const gevo_tuning* t, char* ws,
                              cudaStream_t st, const float* pix_err = nullptr,
                              float* gauss_err = nullptr, const uint32_t* active = nullptr,
                              const uint32_t* act_last = nullptr, const float* act_T = nullptr,
                              const float* act_rest = nullptr)
{
    const WsLayout w = ws_layout(L, n, 0);
    const uint32_t* order = reinterpret_cast<const uint32_t*>(ws + w.tile_order);
    uint32_t* queue = nullptr;
    int grid = L.total_tiles;
    if (t && t->persistent) {
        queue = reinterpret_cast<uint32_t*>(ws + w.err) + kQueueBwd;
        if (cudaMemsetAsync(queue, 0, 4, st) != cudaSuccess) return GEVO_ERR_CUDA;
    }
    const bool ext = pix_err || active;
    auto kern = ext ? pick_bwd<PPT, true>(gD, gT) : pick_bwd<PPT, false>(gD, gT);
    if (queue) grid = std::min(grid, persistent_grid<PPT>(kern, t));
    kern<<<grid, 256 / PPT, 0, st>>>(
        L, n, reinterpret_cast<const float2*>(p.xy), reinterpret_cast<const float4*>(p.conic_opacity),
        reinterpret_cast<const float4*>(p.rgb_depth), vals, reinterpret_cast<const uint2*>(ranges),
        bg[0], bg[1], bg[2], Tf, nc, gC, gD, gT, reinterpret_cast<float2*>(out.xy),
        reinterpret_cast<float4*>(out.conic_opacity), reinterpret_cast<float4*>(out.rgb_depth),
        order, queue, L.total_tiles, pix_err, gauss_err, active, act_last, act_T,
        reinterpret_cast<const float4*>(act_rest));
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}

static bool valid_tuning(const gevo_tuning* t)
{
    if (!t) return true;
    return (t->threads_per_tile == 32 || t->threads_per_tile == 64 || t->threads_per_tile == 128 ||
            t->threads_per_tile == 256) &&
           t->blocks_per_sm >= 0;
}

}  // namespace gevo

using namespace gevo;

extern "C" gevo_status gevo_render_fwd(const gevo_layout* layout, int32_t n, const gevo_proj* proj,
                                       const uint32_t* vals, const uint32_t* ranges,
                                       const float* bg, float* rgb, float* depth, float* T_final,
                                       uint32_t* n_contrib, uint32_t* n_eval,
                                       const gevo_tuning* tuning, void* workspace, void* stream)
{
    if (!layout || layout->n_views < 1 || n < 0 || !proj || !proj->xy || !proj->conic_opacity ||
        !proj->rgb_depth || !ranges || !bg || !rgb || !depth || !T_final || !n_contrib ||
        !workspace || !gevo_aligned(workspace, 256) || !valid_tuning(tuning) ||
        !gevo_aligned(ranges, 8) || !gevo_aligned(proj->conic_opacity, 16) ||
        !gevo_aligned(proj->rgb_depth, 16) || !gevo_aligned(proj->xy, 8))
        return GEVO_ERR_INVALID;
    if (!vals) return GEVO_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = reinterpret_cast<char*>(workspace);
    switch (pick_ppt(tuning)) {
    case 8: return launch_fwd<8>(*layout, n, *proj, vals, ranges, bg, rgb, depth, T_final, n_contrib, n_eval, tuning, ws, st);
    case 4: return launch_fwd<4>(*layout, n, *proj, vals, ranges, bg, rgb, depth, T_final, n_contrib, n_eval, tuning, ws, st);
    case 2: return launch_fwd<2>(*layout, n, *proj, vals, ranges, bg, rgb, depth, T_final, n_contrib, n_eval, tuning, ws, st);
    default: return launch_fwd<1>(*layout, n, *proj, vals, ranges, bg, rgb, depth, T_final, n_contrib, n_eval, tuning, ws, st);
    }
}

extern "C" gevo_status gevo_render_fwd_counts(const gevo_layout* layout, int32_t n,
                                              const gevo_proj* proj, const uint32_t* vals,
                                              const uint32_t* ranges, const float* bg, float* rgb,
                                              float* depth, float* T_final, uint32_t* n_contrib,
                                              uint32_t* n_eval, uint32_t* n_blend,
                                              const gevo_tuning* tuning, void* workspace,
                                              void* stream)
{
    if (!layout || layout->n_views < 1 || n < 0 || !proj || !proj->xy || !proj->conic_opacity ||
        !proj->rgb_depth || !vals || !ranges || !bg || !rgb || !depth || !T_final || !n_contrib ||
        !n_eval || !n_blend || !workspace || !gevo_aligned(workspace, 256) ||
        !valid_tuning(tuning) || !gevo_aligned(ranges, 8) ||
        !gevo_aligned(proj->conic_opacity, 16) || !gevo_aligned(proj->rgb_depth, 16) ||
        !gevo_aligned(proj->xy, 8))
        return GEVO_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = reinterpret_cast<char*>(workspace);
    switch (pick_ppt(tuning)) {
    case 8: return launch_fwd<8>(*layout, n, *proj, vals, ranges, bg, rgb, depth, T_final, n_contrib, n_eval, tuning, ws, st, nullptr, nullptr, n_blend);
    case 4: return launch_fwd<4>(*layout, n, *proj, vals, ranges, bg, rgb, depth, T_final, n_contrib, n_eval, tuning, ws, st, nullptr, nullptr, n_blend);
    case 2: return launch_fwd<2>(*layout, n, *proj, vals, ranges, bg, rgb, depth, T_final, n_contrib, n_eval, tuning, ws, st, nullptr, nullptr, n_blend);
    default: return launch_fwd<1>(*layout, n, *proj, vals, ranges, bg, rgb, depth, T_final, n_contrib, n_eval, tuning, ws, st, nullptr, nullptr, n_blend);
    }
}

extern "C" gevo_status gevo_render_fwd_active(const gevo_layout* layout, int32_t n,
                                              const gevo_proj* proj, const uint32_t* vals,
                                              const uint32_t* ranges, const float* bg, float* rgb,
                                              float* depth, float* T_final, uint32_t* n_contrib,
                                              const uint32_t* active, gevo_active_state* state,
                                              const gevo_tuning* tuning, void* workspace,
                                              void* stream)
{
    if (!layout || layout->n_views < 1 || n < 0 || !proj || !proj->xy || !proj->conic_opacity ||
        !proj->rgb_depth || !vals || !ranges || !bg || !rgb || !depth || !T_final || !n_contrib ||
        !active || !state || !state->last || !state->T || !state->rest || !workspace ||
        !gevo_aligned(workspace, 256) || !valid_tuning(tuning) || !gevo_aligned(ranges, 8) ||
        !gevo_aligned(proj->conic_opacity, 16) || !gevo_aligned(proj->rgb_depth, 16) ||
        !gevo_aligned(proj->xy, 8) || !gevo_aligned(state->rest, 16))
        return GEVO_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = reinterpret_cast<char*>(workspace);
    switch (pick_ppt(tuning)) {
    case 8: return launch_fwd<8>(*layout, n, *proj, vals, ranges, bg, rgb, depth, T_final, n_contrib, nullptr, tuning, ws, st, active, state);
    case 4: return launch_fwd<4>(*layout, n, *proj, vals, ranges, bg, rgb, depth, T_final, n_contrib, nullptr, tuning, ws, st, active, state);
    case 2: return launch_fwd<2>(*layout, n, *proj, vals, ranges, bg, rgb, depth, T_final, n_contrib, nullptr, tuning, ws, st, active, state);
    default: return launch_fwd<1>(*layout, n, *proj, vals, ranges, bg, rgb, depth, T_final, n_contrib, nullptr, tuning, ws, st, active, state);
    }
}

extern "C" gevo_status gevo_render_bwd(const gevo_layout* layout, int32_t n, const gevo_proj* proj,
                                       const uint32_t* vals, const uint32_t* ranges,
                                       const float* bg, const float* T_final,
                                       const uint32_t* n_contrib, const float* dL_drgb,
                                       const float* dL_ddepth, const float* dL_dT,
                                       gevo_grad2d* out, const gevo_tuning* tuning,
                                       void* workspace, void* stream)
{
    if (!layout || layout->n_views < 1 || n < 0 || !proj || !proj->xy || !proj->conic_opacity ||
        !proj->rgb_depth || !proj->radius || !vals || !ranges || !bg || !T_final || !n_contrib ||
        !dL_drgb || !out || !out->xy || !out->conic_opacity || !out->rgb_depth || !workspace ||
        !gevo_aligned(workspace, 256) || !valid_tuning(tuning) || !gevo_aligned(ranges, 8) ||
        !gevo_aligned(out->conic_opacity, 16) || !gevo_aligned(out->rgb_depth, 16) ||
        !gevo_aligned(out->xy, 8))
        return GEVO_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = reinterpret_cast<char*>(workspace);
    switch (pick_ppt(tuning)) {
    case 8: return launch_bwd<8>(*layout, n, *proj, vals, ranges, bg, T_final, n_contrib, dL_drgb, dL_ddepth, dL_dT, *out, tuning, ws, st);
    case 4: return launch_bwd<4>(*layout, n, *proj, vals, ranges, bg, T_final, n_contrib, dL_drgb, dL_ddepth, dL_dT, *out, tuning, ws, st);
    case 2: return launch_bwd<2>(*layout, n, *proj, vals, ranges, bg, T_final, n_contrib, dL_drgb, dL_ddepth, dL_dT, *out, tuning, ws, st);
    default: return launch_bwd<1>(*layout, n, *proj, vals, ranges, bg, T_final, n_contrib, dL_drgb, dL_ddepth, dL_dT, *out, tuning, ws, st);
    }
}

extern "C" gevo_status gevo_render_bwd_active(const gevo_layout* layout, int32_t n,
                                              const gevo_proj* proj, const uint32_t* vals,
                                              const uint32_t* ranges, const float* bg,
                                              const float* T_final, const uint32_t* n_contrib,
                                              const float* dL_drgb, const float* dL_ddepth,
                                              const float* dL_dT, const float* pix_err,
                                              float* gauss_err, const uint32_t* active,
                                              const gevo_active_state* state, gevo_grad2d* out,
                                              const gevo_tuning* tuning, void* workspace,
                                              void* stream)
{
    if (!layout || layout->n_views < 1 || n < 0 || !proj || !proj->xy || !proj->conic_opacity ||
        !proj->rgb_depth || !proj->radius || !vals || !ranges || !bg || !T_final || !n_contrib ||
        !dL_drgb || !out || !out->xy || !out->conic_opacity || !out->rgb_depth || !workspace ||
        !gevo_aligned(workspace, 256) || !valid_tuning(tuning) || !gevo_aligned(ranges, 8) ||
        !gevo_aligned(out->conic_opacity, 16) || !gevo_aligned(out->rgb_depth, 16) ||
        !gevo_aligned(out->xy, 8) || (pix_err == nullptr) != (gauss_err == nullptr))
        return GEVO_ERR_INVALID;
    if (state && (!active || pix_err || !state->last || !state->T || !state->rest ||
                  !gevo_aligned(state->rest, 16)))
        return GEVO_ERR_INVALID;
    const uint32_t* al = state ? state->last : nullptr;
    const float* aT = state ? state->T : nullptr;
    const float* ar = state ? state->rest : nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = reinterpret_cast<char*>(workspace);
    switch (pick_ppt(tuning)) {
    case 8: return launch_bwd<8>(*layout, n, *proj, vals, ranges, bg, T_final, n_contrib, dL_drgb, dL_ddepth, dL_dT, *out, tuning, ws, st, pix_err, gauss_err, active, al, aT, ar);
    case 4: return launch_bwd<4>(*layout, n, *proj, vals, ranges, bg, T_final, n_contrib, dL_drgb, dL_ddepth, dL_dT, *out, tuning, ws, st, pix_err, gauss_err, active, al, aT, ar);
    case 2: return launch_bwd<2>(*layout, n, *proj, vals, ranges, bg, T_final, n_contrib, dL_drgb, dL_ddepth, dL_dT, *out, tuning, ws, st, pix_err, gauss_err, active, al, aT, ar);
    default: return launch_bwd<1>(*layout, n, *proj, vals, ranges, bg, T_final, n_contrib, dL_drgb, dL_ddepth, dL_dT, *out, tuning, ws, st, pix_err, gauss_err, active, al, aT, ar);
    }
}

extern "C" gevo_status gevo_grad2d_zero(const gevo_layout* layout, int32_t n, const gevo_proj* proj,
                                        gevo_grad2d* out, void* stream)
{
    if (!layout || layout->n_views < 1 || n < 0 || !proj || !proj->radius || !out || !out->xy ||
        !out->conic_opacity || !out->rgb_depth || !gevo_aligned(out->conic_opacity, 16) ||
        !gevo_aligned(out->rgb_depth, 16) || !gevo_aligned(out->xy, 8))
        return GEVO_ERR_INVALID;
    const size_t total = (size_t)layout->n_views * n;
    if (total == 0) return GEVO_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = (int)std::min<size_t>((total + 255) / 256, (size_t)sm_count() * 16);
    k_zero_grad2d<<<grid, 256, 0, st>>>(total, proj->radius, reinterpret_cast<float2*>(out->xy),
                                        reinterpret_cast<float4*>(out->conic_opacity),
                                        reinterpret_cast<float4*>(out->rgb_depth));
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}
