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

#include <type_traits>

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

// One spelling for scalar and paired FP32 arithmetic, so that a kernel body
// written over V = float (one pixel) or V = f2 (two pixels of a column, the
// paired f32x2 instructions) computes exactly the same binary32 results.
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ f2 vfma(f2 a, f2 b, f2 c) { return f2_fma(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ f2 vmul(f2 a, f2 b) { return f2_mul(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ f2 vadd(f2 a, f2 b) { return f2_add(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ f2 vsub(f2 a, f2 b) { return f2_sub(a, b); }
template <class V> __device__ __forceinline__ V vsplat(float a);
template <> __device__ __forceinline__ float vsplat<float>(float a) { return a; }
template <> __device__ __forceinline__ f2 vsplat<f2>(float a) { return f2_splat(a); }
__device__ __forceinline__ float vlane(float x, int) { return x; }
__device__ __forceinline__ float vlane(f2 x, int i) { return i ? f2_hi(x) : f2_lo(x); }
template <class V> __device__ __forceinline__ V vpack(const float* a);
template <> __device__ __forceinline__ float vpack<float>(const float* a) { return a[0]; }
template <> __device__ __forceinline__ f2 vpack<f2>(const float* a) { return f2_make(a[0], a[1]); }
template <class V> struct VW { static constexpr int n = 1; };
template <> struct VW<f2> { static constexpr int n = 2; };

// Skip test of one pixel-entry: with the log2 exponent p2 of the Gaussian
// falloff and l = log2(1 / (255 o)), an entry is skipped unless l <= p2 <= 0
// (p2 > 0 is skipped by definition; p2 < l means alpha < 1/255).  The two
// bounds are one window test |p2 + m| <= m with m = -l / 2 =
// log2(255 o) / 2 stored per staged entry (m < 0 when o < 1/255: nothing
// passes).  The same window test decides the reverse walk's entries.
__device__ __forceinline__ bool window_ok(float d, float m)
{
    return fabsf(d) <= m;
}

// Where the window test passes, p2 <= 0 up to rounding, so G <= 1 + 2^-20 and
// an entry of opacity o <= 0.98 has o G < 0.99: its alpha is never clamped.
constexpr float kNoClampO = 0.98f;

// A staged list entry, every value held twice (as a pair), so that the walk
// loads its operands straight into paired registers: mean (x, y), pre-scaled
// conic (a', b', c'), opacity o, m = log2(255 o) / 2 of the window test, and
// colour and depth.
struct Staged {
    ulonglong2 p0;   // (x, x) (y, y)
    ulonglong2 p1;   // (a', a') (b', b')
    ulonglong2 p2;   // (c', c') (o, o)
    ulonglong2 p3;   // (m, m) (r, r)
    ulonglong2 p4;   // (g, g) (b, b)
    unsigned long long p5;   // (z, z)
};

__device__ __forceinline__ ulonglong2 pair2(float a, float b)
{
    return make_ulonglong2(f2_splat(a).v, f2_splat(b).v);
}

__device__ __forceinline__ void stage_entry(Staged& e, float2 m, float4 c, float4 r)
{
    const float4 cs = prescale(c);
    e.p0 = pair2(m.x, m.y);
    e.p1 = pair2(cs.x, cs.y);
    e.p2 = pair2(cs.z, cs.w);
    e.p3 = pair2(0.5f * __log2f(255.f * c.w), r.x);
    e.p4 = pair2(r.y, r.z);
    e.p5 = f2_splat(r.w).v;
}

template <class V> __device__ __forceinline__ V vget(unsigned long long x);
template <> __device__ __forceinline__ float vget<float>(unsigned long long x) { return f2_lo(f2{x}); }
template <> __device__ __forceinline__ f2 vget<f2>(unsigned long long x) { return f2{x}; }

// The operands of one staged entry at a thread's column px (pxv = px as V).
template <class V>
struct EntryOps {
    V my, cz, cx, cy, cw, mw, rx, ry, rb, rw, dx;
    float dxs, a, b, c, o, m;
};

template <class V>
__device__ __forceinline__ EntryOps<V> entry_ops(const Staged& e, V pxv)
{
    const ulonglong2 p0 = e.p0, p1 = e.p1, p2 = e.p2, p3 = e.p3, p4 = e.p4;
    const unsigned long long p5 = e.p5;
    EntryOps<V> q;
    const V mx = vget<V>(p0.x), aa = vget<V>(p1.x), bb = vget<V>(p1.y);
    q.my = vget<V>(p0.y);
    q.dx = vsub(mx, pxv);
    q.cx = vmul(vmul(aa, q.dx), q.dx);   // a' dx^2
    q.cy = vmul(bb, q.dx);               // b' dx
    q.cz = vget<V>(p2.x);
    q.cw = vget<V>(p2.y);
    q.mw = vget<V>(p3.x);
    q.rx = vget<V>(p3.y);
    q.ry = vget<V>(p4.x);
    q.rb = vget<V>(p4.y);
    q.rw = vget<V>(p5);
    q.dxs = vlane(q.dx, 0);
    q.a = f2_lo(f2{p1.x});
    q.b = f2_lo(f2{p1.y});
    q.c = f2_lo(f2{p2.x});
    q.o = f2_lo(f2{p2.y});
    q.m = f2_lo(f2{p3.x});
    return q;
}

// ACT: also record, per pixel, where the reverse walk of an active-set
// backward has to start: 1 + the list position of the last blended entry of an
// active Gaussian (0 if none), the transmittance right after it, and the colour
// (with T_final bg) and depth blended behind it.  The colour is summed in two
// parts, up to the last active entry and since it, so that the part behind
// needs no difference of two sums; the bookkeeping runs only at active
// entries (a warp-uniform branch), and the pixel colour is the sum of the two
// parts.
//
// Per pixel-entry the arithmetic runs on pairs of pixels (f32x2) where a thread
// has two or more: the exponent (2 FMAs), the window offset, o G, the
// candidate T (1 - alpha), and the branch-free blend bookkeeping: with
// b = -alpha where the entry blends at the pixel and 0 elsewhere,
//   -C <- -C + (b T) c (colour and depth summed negated, b T = -alpha T)
//   T <- T + b T       (blended: T (1 - alpha); else unchanged)
// The decisions themselves (window test, stop, done) stay per pixel.
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
    using V = typename std::conditional<(PPT >= 2), f2, float>::type;
    constexpr int W2 = VW<V>::n;
    constexpr int NV = PPT / W2;
    constexpr int NT = 256 / PPT;
    // staging batch: one record per thread (measured on the benchmark: 64
    // entries at 64 threads beat 32, 96, 128 and 256 -- a block leaves its tile
    // as soon as all its pixels stopped, which happens early in most lists)
    constexpr int kBatch = NT;
    __shared__ Staged s_e[kBatch];
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

        // per pixel pair: T, Tf, negated colour / depth sums; pixel rows
        V T[NV], Cn0[NV], Cn1[NV], Cn2[NV], Dn[NV], pyv[NV];
        float B0[PPT], B1[PPT], B2[PPT], BD[PPT], Ta[PPT];   // (negated) sums through the last active entry
        uint32_t last[PPT], cnt[PPT], la[PPT], nbl[PPT];
        bool done[PPT];
#pragma unroll
        for (int h = 0; h < NV; h++) {
            float yy[W2];
#pragma unroll
            for (int i = 0; i < W2; i++) yy[i] = (float)(py0 + h * W2 + i);
            T[h] = vsplat<V>(1.f);
            pyv[h] = vpack<V>(yy);
            Cn0[h] = Cn1[h] = Cn2[h] = Dn[h] = vsplat<V>(0.f);
        }
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            last[k] = 0u; cnt[k] = 0u; nbl[k] = 0u;
            done[k] = !(px < W && py0 + k < H);   // outside the image: nothing to blend
            if (ACT) { B0[k] = B1[k] = B2[k] = BD[k] = 0.f; Ta[k] = 1.f; la[k] = 0u; }
        }
        const V pxv = vsplat<V>((float)px);

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
                stage_entry(s_e[j], m, c, rz[id]);
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
                const uint32_t pos1 = b + j - rg.x + 1;
                const EntryOps<V> e = entry_ops<V>(s_e[j], pxv);
#pragma unroll
                for (int h = 0; h < NV; h++) {
                    const V dy = vsub(e.my, pyv[h]);
                    const V p2 = vfma(vfma(e.cz, dy, e.cy), dy, e.cx);
                    const V dwin = vadd(p2, e.mw);
                    float g[W2];
#pragma unroll
                    for (int i = 0; i < W2; i++) g[i] = ex2_approx(vlane(p2, i));
                    const V og = vmul(e.cw, vpack<V>(g));
                    float na[W2], bn[W2];
#pragma unroll
                    for (int i = 0; i < W2; i++) na[i] = fmaxf(-kAlphaMax, -vlane(og, i));   // -alpha
                    const V tn = vfma(vpack<V>(na), T[h], T[h]);                             // T (1 - alpha)
#pragma unroll
                    for (int i = 0; i < W2; i++) {
                        const int k = h * W2 + i;
                        const bool ok = !done[k] && window_ok(vlane(dwin, i), e.m);
                        const bool bl = ok && !(vlane(tn, i) < kTStop);
                        const bool stop = ok && !bl;
                        if (COUNT && stop) cnt[k] = pos1;
                        if (COUNT) nbl[k] += bl ? 1u : 0u;
                        done[k] = done[k] || stop;
                        bn[i] = bl ? na[i] : 0.f;
                        last[k] = bl ? pos1 : last[k];
                    }
                    const V bnv = vpack<V>(bn);            // -alpha where blended, else 0
                    const V nw = vmul(bnv, T[h]);          // -alpha T
                    T[h] = vfma(bnv, T[h], T[h]);          // blended: T (1 - alpha), else T
                    Cn0[h] = vfma(nw, e.rx, Cn0[h]);
                    Cn1[h] = vfma(nw, e.ry, Cn1[h]);
                    Cn2[h] = vfma(nw, e.rb, Cn2[h]);
                    Dn[h] = vfma(nw, e.rw, Dn[h]);
                }
                if (ACT && s_act[j]) {
                    // an active entry: move the part since the previous one
                    // into the part up to here (Cn holds the part since)
#pragma unroll
                    for (int h = 0; h < NV; h++) {
                        float c0[W2], c1[W2], c2[W2], dd[W2];
#pragma unroll
                        for (int i = 0; i < W2; i++) {
                            const int k = h * W2 + i;
                            const bool at = last[k] == pos1;   // blended right here
                            const float x0_ = vlane(Cn0[h], i), x1_ = vlane(Cn1[h], i),
                                        x2_ = vlane(Cn2[h], i), xd = vlane(Dn[h], i);
                            B0[k] = at ? __fadd_rn(B0[k], x0_) : B0[k];
                            B1[k] = at ? __fadd_rn(B1[k], x1_) : B1[k];
                            B2[k] = at ? __fadd_rn(B2[k], x2_) : B2[k];
                            BD[k] = at ? __fadd_rn(BD[k], xd) : BD[k];
                            c0[i] = at ? 0.f : x0_;
                            c1[i] = at ? 0.f : x1_;
                            c2[i] = at ? 0.f : x2_;
                            dd[i] = at ? 0.f : xd;
                            Ta[k] = at ? vlane(T[h], i) : Ta[k];
                            la[k] = at ? pos1 : la[k];
                        }
                        Cn0[h] = vpack<V>(c0);
                        Cn1[h] = vpack<V>(c1);
                        Cn2[h] = vpack<V>(c2);
                        Dn[h] = vpack<V>(dd);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int h = k / W2, i = k % W2;
            const int py = py0 + k;
            if (px < W && py < H) {
                const size_t pix = (size_t)py * W + px;
                const size_t gp = (size_t)L.pix_base[v] + pix;
                const float Tk = vlane(T[h], i);
                float c0 = -vlane(Cn0[h], i), c1 = -vlane(Cn1[h], i), c2 = -vlane(Cn2[h], i),
                      dp = -vlane(Dn[h], i);
                if (ACT) {
                    // c0..dp hold the part behind the last active entry
                    act_last[gp] = la[k];
                    act_T[gp] = Ta[k];
                    act_rest[gp] = la[k] ? make_float4(__fmaf_rn(Tk, bg0, c0), __fmaf_rn(Tk, bg1, c1),
                                                       __fmaf_rn(Tk, bg2, c2), dp)
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
                    c0 = __fsub_rn(c0, B0[k]);
                    c1 = __fsub_rn(c1, B1[k]);
                    c2 = __fsub_rn(c2, B2[k]);
                    dp = __fsub_rn(dp, BD[k]);
                }
                float* rgb = out_rgb + 3 * (size_t)L.pix_base[v];
                rgb[pix] = __fmaf_rn(Tk, bg0, c0);
                rgb[P + pix] = __fmaf_rn(Tk, bg1, c1);
                rgb[2 * P + pix] = __fmaf_rn(Tk, bg2, c2);
                out_d[gp] = dp;
                out_T[gp] = Tk;
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
//
// Per pixel-entry the arithmetic runs on pairs of pixels (f32x2) where a thread
// has two or more, branch-free: a pixel where the entry is not blended (list
// position at or past n_contrib, or outside the window test of the forward
// pass) takes alpha = 0 -- T / (1 - 0) = T (the hardware reciprocal of 1 is
// exact), the suffix scalar and every sum unchanged -- and the derivatives
// through alpha are kept only where o G <= 0.99 (alpha not clamped).
#ifndef GEVO_BWD8_MINB
#define GEVO_BWD8_MINB 14   // 32-thread walk: at most 146 registers (measured best of 12, 14, 16, 18)
#endif
template <int PPT, bool DD, bool DT, bool EXT>
__global__ void __launch_bounds__(256 / PPT, (PPT == 8 ? (EXT ? 16 : GEVO_BWD8_MINB) : 1))
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
    using V = typename std::conditional<(PPT >= 2), f2, float>::type;
    constexpr int W2 = VW<V>::n;
    constexpr int NV = PPT / W2;
    constexpr int NT = 256 / PPT;
    constexpr int NW = NT / 32;
    // staging batch: half a record per thread from 64 threads up (measured on
    // the benchmark: 32 entries at 64 threads beat 64, 96, 128 and 256; the walk
    // starts near each warp's last blended position, so short batches waste
    // less), two records per thread for the one-warp walk (64 entries beat 16
    // and 32 there: fewer barriers and list rounds per entry; the active-set
    // variant keeps 32, measured faster for it)
    constexpr int kBatch = NT >= 64 ? NT / 2 : (EXT ? NT : 2 * NT);
    __shared__ Staged s_e[kBatch];
    __shared__ uint32_t s_mask[kBatch];
    __shared__ uint32_t s_id[kBatch];
    // per-entry sums: the six moment products, colour and depth (10), the
    // opacity term with dL/dT_final, the error weight of Eq. 5
    constexpr int NG = 10 + (DT ? 1 : 0) + (EXT ? 1 : 0);
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
        const V pxv = vsplat<V>((float)px);

        // Only the projection of the suffix colour and depth S onto the
        // pixel's upstream gradient, Pg = dL/dC . S (+ dL/dD S_D), enters
        // dL/dalpha = T_i (dL/dC . c + dL/dD z - Pg), and it follows
        // S <- S + alpha (c - S) as Pg <- Pg + alpha (q - Pg), q = dL/dC . c +
        // dL/dD z: one scalar per pixel instead of four.
        float Tk[PPT], Pk[PPT], g0[PPT], g1[PPT], g2[PPT], gdd[PPT], gtt[PPT], pek[PPT], yk[PPT];
        uint32_t last[PPT];
        uint32_t mymax = 0;
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            const int py = py0 + k;
            Pk[k] = 0.f;
            yk[k] = (float)py;
            if (px < W && py < H) {
                const size_t pix = (size_t)py * W + px;
                const size_t gp = (size_t)L.pix_base[v] + pix;
                const float* g3 = dL_drgb + 3 * (size_t)L.pix_base[v];
                Tk[k] = T_final[gp];
                last[k] = n_contrib[gp];
                g0[k] = g3[pix]; g1[k] = g3[P + pix]; g2[k] = g3[2 * P + pix];
                gdd[k] = DD ? dL_dd[gp] : 0.f;
                gtt[k] = DT ? dL_dT[gp] * Tk[k] : 0.f;
                pek[k] = (EXT && pix_err) ? pix_err[gp] : 0.f;
                Pk[k] = g0[k] * bg0 + g1[k] * bg1 + g2[k] * bg2;
                if (EXT && act_last) {
                    // start at the last active entry: what lies behind it is
                    // summarised by the transmittance after it and the colour
                    // and depth blended behind it
                    last[k] = act_last[gp];
                    if (last[k]) {
                        const float Ta = act_T[gp];
                        const float4 q = act_rest[gp];
                        Tk[k] = Ta;
                        Pk[k] = __fdiv_rn(g0[k] * q.x + g1[k] * q.y + g2[k] * q.z + gdd[k] * q.w, Ta);
                    }
                }
            } else {
                Tk[k] = 1.f; last[k] = 0u;
                g0[k] = g1[k] = g2[k] = gdd[k] = gtt[k] = pek[k] = 0.f;
            }
            mymax = max(mymax, last[k]);
        }
        V T[NV], Pg[NV], gC0[NV], gC1[NV], gC2[NV], gD[NV], gTT[NV], pe[NV], pyv[NV];
#pragma unroll
        for (int h = 0; h < NV; h++) {
            T[h] = vpack<V>(Tk + h * W2);
            Pg[h] = vpack<V>(Pk + h * W2);
            gC0[h] = vpack<V>(g0 + h * W2);
            gC1[h] = vpack<V>(g1 + h * W2);
            gC2[h] = vpack<V>(g2 + h * W2);
            gD[h] = vpack<V>(gdd + h * W2);
            gTT[h] = vpack<V>(gtt + h * W2);
            pe[h] = vpack<V>(pek + h * W2);
            pyv[h] = vpack<V>(yk + h * W2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mymax = max(mymax, __shfl_xor_sync(0xffffffffu, mymax, o));
        if (lane == 0) s_max[warp] = mymax;
        __syncthreads();
        uint32_t bmax = 0;
#pragma unroll
        for (int w = 0; w < NW; w++) bmax = max(bmax, s_max[w]);

        const V one = vsplat<V>(1.f);
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
                stage_entry(s_e[j], m, c, rz[gid]);
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
                const EntryOps<V> e = entry_ops<V>(s_e[j], pxv);
                const float dx = e.dxs;
                const bool act = !EXT || !(s_id[j] >> 31);
                // per-thread sums over its pixels (pairs), reduced below
                V s0 = vsplat<V>(0.f), s1 = s0, s2 = s0, so = s0, sr = s0, sg = s0, sb = s0,
                  sz = s0, se = s0;
                // NC: the entry cannot reach the alpha clamp (o <= kNoClampO), so
                // alpha needs no minimum and dL/dalpha no clamp select; without
                // dL/dT_final an unused pixel's alpha = 0 already zeroes its term
                auto pixels = [&](auto nc_tag) {
                    constexpr bool NC = decltype(nc_tag)::value;
#pragma unroll
                    for (int h = 0; h < NV; h++) {
                        const V dy = vsub(e.my, pyv[h]);
                        const V p2 = vfma(vfma(e.cz, dy, e.cy), dy, e.cx);
                        const V dwin = vadd(p2, e.mw);
                        float g[W2], al[W2];
                        bool kk[W2];
#pragma unroll
                        for (int i = 0; i < W2; i++) g[i] = ex2_approx(vlane(p2, i));
                        const V G = vpack<V>(g);
                        const V og = vmul(e.cw, G);
#pragma unroll
                        for (int i = 0; i < W2; i++) {
                            const int k = h * W2 + i;
                            const float ogi = vlane(og, i);
                            const bool use = pos < last[k] && window_ok(vlane(dwin, i), e.m);
                            if (NC) {
                                kk[i] = use;
                                al[i] = use ? ogi : 0.f;
                            } else {
                                kk[i] = use && ogi <= kAlphaMax;      // alpha not clamped
                                al[i] = use ? fminf(kAlphaMax, ogi) : 0.f;
                            }
                        }
                        const V alpha = vpack<V>(al);                    // 0 where unused
                        const V om = vsub(one, alpha);
                        float ri[W2];
#pragma unroll
                        for (int i = 0; i < W2; i++) ri[i] = rcp_approx(vlane(om, i));
                        const V inv = vpack<V>(ri);
                        const V Ti = vmul(T[h], inv);
                        T[h] = Ti;
                        const V w = vmul(alpha, Ti);
                        // (c - S) . dL/dC, shared by dL/dalpha = T_i gd and the suffix update
                        V qc = vmul(gC0[h], e.rx);
                        qc = vfma(gC1[h], e.ry, qc);
                        qc = vfma(gC2[h], e.rb, qc);
                        if (DD) qc = vfma(gD[h], e.rw, qc);
                        const V gd = vsub(qc, Pg[h]);
                        Pg[h] = vfma(alpha, gd, Pg[h]);
                        if (EXT && !act) {
                            if (pix_err) se = vfma(w, pe[h], se);
                            continue;
                        }
                        if (EXT) se = vfma(w, pe[h], se);
                        sr = vfma(gC0[h], w, sr);
                        sg = vfma(gC1[h], w, sg);
                        sb = vfma(gC2[h], w, sb);
                        if (DD) sz = vfma(gD[h], w, sz);
                        V dp;
                        float dd[W2];
                        if (DT) {
                            // dL/dalpha = gd T_i - dL/dT_final T_final / (1 - alpha)
                            const V dLda = vsub(vmul(gd, Ti), vmul(gTT[h], inv));
#pragma unroll
                            for (int i = 0; i < W2; i++) dd[i] = kk[i] ? vlane(dLda, i) : 0.f;
                            const V kd = vpack<V>(dd);
                            so = vfma(kd, G, so);
                            dp = vmul(kd, alpha);
                        } else {
                            const V gw = vmul(gd, w);
                            if (NC) {
                                dp = gw;
                            } else {
#pragma unroll
                                for (int i = 0; i < W2; i++) dd[i] = kk[i] ? vlane(gw, i) : 0.f;
                                dp = vpack<V>(dd);
                            }
                        }
                        const V t = vmul(dp, dy);
                        s0 = vadd(s0, dp);
                        s1 = vadd(s1, t);
                        s2 = vfma(t, dy, s2);
                    }
                };
                if (!DT && e.o <= kNoClampO) pixels(std::true_type{});
                else pixels(std::false_type{});
                float m0 = vlane(s0, 0), m1 = vlane(s1, 0), m2 = vlane(s2, 0);
                float a_o = vlane(so, 0), a_r = vlane(sr, 0), a_g = vlane(sg, 0),
                      a_b = vlane(sb, 0), a_z = vlane(sz, 0), a_e = vlane(se, 0);
#pragma unroll
                for (int i = 1; i < W2; i++) {
                    m0 += vlane(s0, i); m1 += vlane(s1, i); m2 += vlane(s2, i);
                    a_o += vlane(so, i); a_r += vlane(sr, i); a_g += vlane(sg, i);
                    a_b += vlane(sb, i); a_z += vlane(sz, i); a_e += vlane(se, i);
                }
                if (EXT && !act) {
                    // inactive: transmittance and suffix colour only (+ the error weight)
                    if (pix_err) {
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) a_e += __shfl_xor_sync(0xffffffffu, a_e, o);
                        if (lane == 0 && a_e != 0.f) atomicAdd(&s_g[j][NG - 1], a_e);
                    }
                    continue;
                }
                // A thread's pixels share the column, so dx is the same for all
                // of them: the conic and mean gradients are linear in the
                // per-pixel dp = dL/dalpha * alpha with coefficients in 1, dy,
                // dy^2 (the moments m0, m1, m2), and across the warp's columns in
                // 1, dx, dx^2.  The warp sums the six products m0, dx m0, dx^2 m0,
                // m1, dx m1, m2, and the gradients are formed from their totals
                // once per entry when the batch is flushed.
                const float S1 = dx * m0;
                const float vals[12] = {m0, S1, dx * S1, m1, dx * m1, m2, a_r, a_g, a_b, a_z,
                                        DT ? a_o : a_e, a_e};
                int slot;
                // one warp per block: an entry's sums come from this warp alone,
                // so they are stored; several warps add theirs
                if (NG == 10) {
                    const float tot = warp_reduce10(vals, slot);
                    if (NW == 1) {
                        if (slot >= 0) s_g[j][slot] = tot;
                    } else if (slot >= 0 && tot != 0.f) {
                        atomicAdd(&s_g[j][slot], tot);
                    }
                } else {
                    const float tot = warp_reduce12(vals, slot);
                    if (NW == 1) {
                        if (slot >= 0 && slot < NG) s_g[j][slot] = tot;
                    } else if (slot >= 0 && slot < NG && tot != 0.f) {
                        atomicAdd(&s_g[j][slot], tot);
                    }
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
                if (DT) nz = nz || gg[10] != 0.f;
                if (!nz) continue;
                // d alpha / d(a, b, c) = alpha (-dx^2 / 2, -dx dy, -dy^2 / 2);
                // d alpha / d(mean) = alpha ln2 (2 a' dx + b' dy, 2 c' dy + b' dx)
                // with the pre-scaled conic (a', b', c'); without dL/dT_final,
                // dL/do = sum dL/dalpha G = m0 / o (alpha = o G on every
                // unclamped pixel)
                const float ca = f2_lo(f2{s_e[j].p1.x}), cb = f2_lo(f2{s_e[j].p1.y});
                const float cc = f2_lo(f2{s_e[j].p2.x}), op = f2_lo(f2{s_e[j].p2.y});
                const float S0 = gg[0], S1 = gg[1], S2 = gg[2], S3 = gg[3], S4 = gg[4], S5 = gg[5];
                const float gx = kLn2 * (2.f * ca * S1 + cb * S3);
                const float gy = kLn2 * (2.f * cc * S3 + cb * S1);
                const float go = DT ? gg[10] : S0 * rcp_approx(op);
                const size_t gid = vbase + (EXT ? (s_id[j] & 0x7FFFFFFFu) : s_id[j]);
                atomicAdd(g_xy + gid, make_float2(gx, gy));
                atomicAdd(g_co + gid, make_float4(-0.5f * S2, -S4, -0.5f * S5, go));
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
    if (!layout || !gevo::layout_valid(*layout) || n < 0 || !proj || !proj->xy || !proj->conic_opacity ||
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
    if (!layout || !gevo::layout_valid(*layout) || n < 0 || !proj || !proj->xy || !proj->conic_opacity ||
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
    if (!layout || !gevo::layout_valid(*layout) || n < 0 || !proj || !proj->xy || !proj->conic_opacity ||
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
    if (!layout || !gevo::layout_valid(*layout) || n < 0 || !proj || !proj->xy || !proj->conic_opacity ||
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
    if (!layout || !gevo::layout_valid(*layout) || n < 0 || !proj || !proj->xy || !proj->conic_opacity ||
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
    if (!layout || !gevo::layout_valid(*layout) || n < 0 || !proj || !proj->radius || !out || !out->xy ||
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
