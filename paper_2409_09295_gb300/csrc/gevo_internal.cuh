// Internal declarations shared by the CUDA translation units of libgevo.
// Constants are those of the 3DGS formulation the paper renders with
// (Section I "GS"); the paper itself states none of them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/gevo.h"

namespace gevo {

constexpr float kNearZ = 0.2f;          // cull at or in front of 0.2 m
constexpr float kDilation = 0.3f;       // px^2 added to the 2-D covariance
constexpr float kGuard = 1.3f;          // Jacobian clamp: 1.3x half field of view
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTStop = 1e-4f;
constexpr int kTile = GEVO_TILE;        // 16
constexpr int kTilePixels = kTile * kTile;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// Bits of the sticky device error word.
constexpr uint32_t kErrCapacity = 1u << 0;
constexpr uint32_t kErrNonFinite = 1u << 1;
constexpr uint32_t kErrTimeout = 1u << 2;    // a bounded device wait gave up

// Workspace layout (offsets in bytes from the 256-byte aligned base).
struct WsLayout {
    size_t err;          // uint32 error word + uint32 queue heads [8]
    size_t tile_count;   // uint32 [T]
    size_t tile_cursor;  // uint32 [T]
    size_t tile_order;   // uint32 [T]  heaviest first
    size_t tile_start;   // uint32 [T]  exclusive scan of counts
    size_t dup_tmp;      // uint64 [cap]  (depth bits << 32 | id), bucketed by tile
    size_t dup_tmp2;     // uint64 [cap]  ping-pong for long tiles
    size_t dxi_acc;      // float [V][6]
    size_t pb_perm;      // uint32 [n]: the projection backward's Gaussian order
    size_t pb_mask;      // uint64 [n]: visible-view mask of each, in that order
    size_t core;         // bytes up to here (the no-allocation sort uses only these)
    size_t blk_off;      // uint32 [ceil(n / 2048)][T]: each binning block's run offset per tile
    // depth-ordered binning (gevo_bin_sort on views of at most kOrdMaxTiles tiles)
    size_t ord_stat;     // uint32 [V][4]: max(~depth bits), max(depth bits), visible count
    size_t ord_seg;      // uint32 [5][V * kDepthBins (+1)]: count, start, cursor, order, and
                         // ranges [V * kDepthBins][2] of the depth segments
    size_t ord_total;    // uint64 visible entries + uint32 scratch error word
    size_t ord_b1;       // uint64 [V * n] (depth bits << 32 | id), by depth segment; once
                         // the depth sort is done, uint4 [V * n] records (id, depth bits,
                         // tile rectangle) in sorted order
    size_t ord_b2;       // uint64 [V * n] ping-pong of long segments
    size_t ord_vals;     // uint32 [V * n]: each entry's depth bits (id order) until the depth
                         // sort writes each view's visible ids in (depth bits, id) order
    size_t ord_dkeys;    // uint64 [V * n]: the depth sort's keys (segment << 32 | depth bits)
    size_t ord_pre;      // uint64 [V * n + V + 1]: first the uint2 tile rectangle of each
                         // visible entry (id order), then per view the exclusive prefix of
                         // the rectangle areas (first duplicate of each entry) and its end
    size_t ord_bsum;     // uint64 [V * (n / kOrdScanItems + 1)]: block sums of that scan
    size_t ord_units;    // uint64 [4 * (GEVO_MAX_VIEWS + 1)]: the unit table
    size_t ord_cnt;      // uint32 [(cap / kOrdUnit + V + 1) * max tiles]: per (unit, tile)
                         // counts, then their running sums over units
    size_t ord_wstart;   // uint32 [(cap / kOrdUnit + V + 1) * 8]: first entry of each warp
    size_t ord_wofs;     // uint32 [(cap / kOrdUnit + V + 1) * 8 * ceil(max tiles / 2)]: per
                         // (unit, warp, tile) the earlier warps' count, 16 bits per tile
    size_t total;
};
constexpr int kDepthBins = 256;     // depth segments per view of the per-view depth sort
constexpr int kOrdMaxTiles = 8192;  // views with more tiles take the bucket-and-sort path
constexpr int kOrdUnit = 8192;      // duplicates per block of the order-keeping passes
constexpr int kOrdScanItems = 1024; // entries per block of the prefix scan (4 per thread)
// pbwd false leaves out the projection backward's order (the no-allocation
// sort's scratch holds only what the sort uses); every field before dup_tmp has
// an offset that does not depend on cap, so calls that do not know the
// capacity (render, projection backward) pass 0.
WsLayout ws_layout(const gevo_layout& L, int32_t n, uint64_t cap, bool pbwd = true);

// Gaussians per binning block of one view (the binning kernels' chunk).
constexpr int kBinChunk = 2048;

// Queue-head slots inside the error block.
constexpr int kQueueFwd = 1;
constexpr int kQueueBwd = 2;
constexpr int kQueueSort = 3;

// Which view owns global tile t (uniform per block; at most 64 views).
__device__ __forceinline__ int view_of_tile(const gevo_layout& L, int t)
{
    int v = 0;
    while (v + 1 < L.n_views && t >= L.tile_base[v + 1]) ++v;
    return v;
}

// Tile rectangle in binary32 (identical rounding in every kernel that bins):
// [floor((m - r) / 16), floor((m + r + 15) / 16)) per axis, clamped to the grid.
__device__ __forceinline__ void tile_rect(float mx, float my, int r, int tiles_x, int tiles_y,
                                          int& x0, int& y0, int& x1, int& y1)
{
    const float rf = (float)r;
    float a = floorf(__fmul_rn(__fsub_rn(mx, rf), 0.0625f));
    float b = floorf(__fmul_rn(__fsub_rn(my, rf), 0.0625f));
    float c = floorf(__fmul_rn(__fadd_rn(__fadd_rn(mx, rf), 15.0f), 0.0625f));
    float d = floorf(__fmul_rn(__fadd_rn(__fadd_rn(my, rf), 15.0f), 0.0625f));
    x0 = (int)fminf(fmaxf(a, 0.0f), (float)tiles_x);
    y0 = (int)fminf(fmaxf(b, 0.0f), (float)tiles_y);
    x1 = (int)fminf(fmaxf(c, 0.0f), (float)tiles_x);
    y1 = (int)fminf(fmaxf(d, 0.0f), (float)tiles_y);
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x to within 1 ulp (PTX rcp.approx): the reverse walk's transmittance
// recovery, where a per-step ulp is far below the gradients' tolerance and no
// integer decision depends on the result.
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sqrt(x) to within a few ulp (PTX sqrt.approx).
__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// A layout is used only as gevo_layout_init fills it: 1..GEVO_MAX_VIEWS views of
// positive size, tile and pixel counts and the per-view bases recomputed from
// the widths and heights.  Entry points reject anything else as invalid, so a
// hand-built layout cannot make a kernel index past the tile or pixel planes.
bool layout_valid(const gevo_layout& L);

// Packed pairs of binary32 values for the paired FP32 instructions of sm_100
// and later (add / sub / mul / fma .rn.f32x2: two IEEE round-to-nearest
// results per lane and instruction, each the same as the scalar instruction's).
struct f2 {
    unsigned long long v;
};
__device__ __forceinline__ f2 f2_make(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ f2 f2_splat(float a) { return f2_make(a, a); }
__device__ __forceinline__ float f2_lo(f2 x)
{
    float a;
    asm("{\n\t.reg .f32 t;\n\tmov.b64 {%0, t}, %1;\n\t}" : "=f"(a) : "l"(x.v));
    return a;
}
__device__ __forceinline__ float f2_hi(f2 x)
{
    float b;
    asm("{\n\t.reg .f32 t;\n\tmov.b64 {t, %0}, %1;\n\t}" : "=f"(b) : "l"(x.v));
    return b;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

int sm_count();
int device_max_smem_optin();

}  // namespace gevo

#define GEVO_CHECK_LAUNCH()                                   \
    do {                                                      \
        if (cudaGetLastError() != cudaSuccess) return GEVO_ERR_CUDA; \
    } while (0)

static inline bool gevo_aligned(const void* p, size_t a)
{
    return ((uintptr_t)p % a) == 0;
}
