// Stages a2-a4 of the splatting renderer GEVO uses (Section I "GS"): emit one
// (tile, depth) key per (Gaussian, tile) pair, sort the keys bit-exactly and
// find each tile's range.
//
// Two GB300 designs instead of one 64-bit radix sort over all duplicates.
// Views of up to kOrdMaxTiles tiles take the depth-ordered path further down:
// each view's visible entries are sorted by depth once and every duplicate is
// emitted straight into its sorted place (no per-tile sort).  Larger views,
// and the no-allocation call, take the bucket-and-sort path:
//   1. k_count   : per-tile duplicate counts (one L2 atomic per duplicate);
//   2. k_scan    : one block scans the counts -> tile starts, the ranges, the
//                  total D and a heaviest-first tile order for later kernels;
//   3. k_scatter : each duplicate (depth bits << 32 | id) goes into its tile's
//                  bucket (8 bytes written per duplicate);
//   4. k_segsort : one block per tile sorts its bucket (stable LSD radix, each
//                  warp scattering its own chunk, then equal depths by id): in
//                  shared memory over 9-bit digits of the depth bits minus the
//                  tile's least, up to 2048 entries; through L2 over the
//                  varying depth bytes beyond that.  It writes the final 64-bit
//                  keys and 32-bit values.
// The tile is handled by counting, so the sort only moves the depth half; the
// result is the unique (tile, depth bits, id) order, identical to a full sort.
#include "gevo_internal.cuh"
#include <mutex>

namespace gevo {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortSmemItems = 2048;   // longer tiles sort through global memory (L2)

__global__ void __launch_bounds__(256)
k_count(gevo_layout L, int n, const float2* __restrict__ xy, const int* __restrict__ radius,
        uint32_t* __restrict__ tile_count)
{
    const size_t total = (size_t)L.n_views * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int r = radius[i];
        if (r <= 0) continue;
        const int v = (int)(i / n);
        const float2 m = xy[i];
        int x0, y0, x1, y1;
        tile_rect(m.x, m.y, r, L.tiles_x[v], L.tiles_y[v], x0, y0, x1, y1);
        const int base = L.tile_base[v];
        const int tx = L.tiles_x[v];
        for (int y = y0; y < y1; y++)
            for (int x = x0; x < x1; x++) atomicAdd(tile_count + base + y * tx + x, 1u);
    }
}

// One block of 1024 threads.  Warp w owns a contiguous chunk of the tiles and
// walks it 32 tiles at a time (coalesced loads, warp scans with a carry); the
// warps' chunk totals are scanned once in shared memory.  The heaviest-first
// order buckets tiles by floor(log2(count)); bucket counts and positions are
// taken with one shared-memory atomic per distinct bucket per warp step.  When
// a chunk is at most kScanCache steps (T <= 16384) its counts are read once,
// all at a time, and kept in registers for the three passes.
constexpr int kScanCache = 16;
__global__ void __launch_bounds__(1024)
k_scan(int T, uint64_t cap, const uint32_t* __restrict__ tile_count, uint32_t* __restrict__ tile_start,
       uint32_t* __restrict__ tile_cursor, uint32_t* __restrict__ tile_order,
       uint32_t* __restrict__ ranges, uint64_t* __restrict__ d_n_dup, uint32_t* err,
       const unsigned long long* __restrict__ known_total = nullptr)
{
    constexpr int NW = 32;
    __shared__ unsigned long long s_warp[NW];
    __shared__ uint32_t s_bucket[34];
    __shared__ uint32_t s_bucket_base[34];
    __shared__ unsigned long long s_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int chunk = ((T + NW - 1) / NW + 31) & ~31;
    const int w0 = min(T, warp * chunk), w1 = min(T, w0 + chunk);
    const uint32_t lt = (1u << lane) - 1u;
    const bool cached = chunk <= 32 * kScanCache;   // the same in every warp
    uint32_t cc[kScanCache];
    // every pass visits the chunk's steps in order; step i covers tiles
    // w0 + 32 i + lane, and f(t, valid, c) is called by the whole warp
    auto steps = [&](auto&& f) {
        if (cached) {
#pragma unroll
            for (int i = 0; i < kScanCache; i++) {
                const int b0 = w0 + 32 * i;
                if (b0 >= w1) break;
                f(b0 + lane, b0 + lane < w1, cc[i]);
            }
        } else {
            for (int b0 = w0; b0 < w1; b0 += 32) {
                const int t = b0 + lane;
                f(t, t < w1, t < w1 ? tile_count[t] : 0u);
            }
        }
    };
    if (tid < 34) s_bucket[tid] = 0;
    unsigned long long sum = 0;
    if (cached) {
#pragma unroll
        for (int i = 0; i < kScanCache; i++) {
            const int t = w0 + 32 * i + lane;
            cc[i] = t < w1 ? tile_count[t] : 0u;
        }
#pragma unroll
        for (int i = 0; i < kScanCache; i++) sum += cc[i];
    } else {
        for (int t = w0 + lane; t < w1; t += 32) sum += tile_count[t];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) s_warp[warp] = sum;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long x = s_warp[lane];
        unsigned long long incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        s_warp[lane] = incl - x;
        if (lane == 31) s_total = incl;
    }
    __syncthreads();
    // the depth-ordered path counts no duplicate when D exceeds the capacity and
    // passes the exact D instead
    const unsigned long long D = known_total ? *known_total : s_total;
    const bool overflow = D > cap;
    unsigned long long carry = s_warp[warp];
    steps([&](int t, bool valid, uint32_t c) {
        unsigned long long incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        const unsigned long long run = carry + incl - c;
        if (valid) {
            tile_start[t] = (uint32_t)run;
            tile_cursor[t] = 0u;
            const bool empty = overflow || c == 0;
            ranges[2 * t] = empty ? 0u : (uint32_t)run;
            ranges[2 * t + 1] = empty ? 0u : (uint32_t)(run + c);
        }
        carry += __shfl_sync(0xffffffffu, incl, 31);
        const int b = valid ? (c == 0 ? 0 : 32 - __clz(c)) : 34;
        const uint32_t peers = __match_any_sync(0xffffffffu, b);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&s_bucket[b], __popc(peers));
    });
    if (tid == 0) {
        *d_n_dup = D;
        if (overflow) atomicOr(err, kErrCapacity);
    }
    __syncthreads();
    if (tid == 0) {  // heaviest bucket first, empty tiles last
        uint32_t acc = 0;
        for (int b = 33; b >= 0; b--) { s_bucket_base[b] = acc; acc += s_bucket[b]; }
    }
    __syncthreads();
    steps([&](int t, bool valid, uint32_t c) {
        const int b = valid ? (c == 0 ? 0 : 32 - __clz(c)) : 34;
        const uint32_t peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (valid && lane == leader) base = atomicAdd(&s_bucket_base[b], __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (valid) tile_order[base + __popc(peers & lt)] = (uint32_t)t;
    });
}

__global__ void __launch_bounds__(256)
k_scatter(gevo_layout L, int n, const float2* __restrict__ xy, const int* __restrict__ radius,
          const float4* __restrict__ rgbz, const uint32_t* __restrict__ tile_start,
          uint32_t* __restrict__ tile_cursor, const uint64_t* __restrict__ d_n_dup, uint64_t cap,
          unsigned long long* __restrict__ bucket)
{
    if (*d_n_dup > cap) return;
    const size_t total = (size_t)L.n_views * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int r = radius[i];
        if (r <= 0) continue;
        const int v = (int)(i / n);
        const uint32_t g = (uint32_t)(i - (size_t)v * n);
        const float2 m = xy[i];
        const uint32_t dbits = __float_as_uint(rgbz[i].w);
        const unsigned long long item = ((unsigned long long)dbits << 32) | g;
        int x0, y0, x1, y1;
        tile_rect(m.x, m.y, r, L.tiles_x[v], L.tiles_y[v], x0, y0, x1, y1);
        const int base = L.tile_base[v];
        const int tx = L.tiles_x[v];
        for (int y = y0; y < y1; y++)
            for (int x = x0; x < x1; x++) {
                const int t = base + y * tx + x;
                const uint32_t slot = tile_start[t] + atomicAdd(tile_cursor + t, 1u);
                bucket[slot] = item;
            }
    }
}

// ---------------------------------------------------------------------------
// Shared-memory binning: block (c, v) handles Gaussians [c*kBinChunk, ...) of
// view v and keeps a histogram of view v's tiles in shared memory, so global
// atomics drop from one per duplicate to one per (block, touched tile).
// Rectangles wider than a warp are expanded by the whole warp (lane k takes
// tiles k, k+32, ...), so one large splat does not serialise its warp.
// ---------------------------------------------------------------------------
constexpr int kBinThreads = 256;
constexpr int kBinMaxSmemTiles = 16384;   // views with more tiles use k_count / k_scatter

// f(g, tile, depth bits of g): the depth bits are loaded with the Gaussian's
// other record fields when rgbz != NULL (0 otherwise) and handed to the lane
// that emits each duplicate by shuffle.
template <typename F>
__device__ __forceinline__ void for_each_dup(const gevo_layout& L, int v, int n, int g0, int g1,
                                             const float2* __restrict__ xy,
                                             const int* __restrict__ radius,
                                             const float4* __restrict__ rgbz, F&& f)
{
    // The duplicates of the warp's 32 Gaussians are laid end to end (warp
    // prefix sum of the rectangle areas) and dealt out round-robin to the
    // lanes, so every lane does the same amount of work whatever the sizes.
    // The Gaussians with a non-empty rectangle are packed into shared memory
    // in lane order; the owner of duplicate k0 + p of a round of 32 is then
    // (packed rectangles starting before k0) + (starts at k0 .. k0 + p) - 1,
    // from one ballot, one OR-reduction and a population count.
    __shared__ int4 s_rect[kBinThreads / 32][32];      // x0, y0, width, first duplicate
    __shared__ uint2 s_gd[kBinThreads / 32][32];       // Gaussian, depth bits
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int tx = L.tiles_x[v], ty = L.tiles_y[v];
    const size_t vb = (size_t)v * n;
    // the next group's record fields are loaded while this group is expanded
    int rn = 0;
    float2 mn = make_float2(0.f, 0.f);
    uint32_t dn = 0u;
    auto fetch = [&](int gg) {
        rn = 0;
        if (gg < g1) {
            rn = radius[vb + gg];
            mn = xy[vb + gg];
            if (rgbz) dn = __float_as_uint(__ldg(reinterpret_cast<const float*>(rgbz + vb + gg) + 3));
        }
    };
    fetch(g0 + (int)(threadIdx.x & ~31) + lane);
    for (int gs = g0 + (int)(threadIdx.x & ~31); gs < g1; gs += kBinThreads) {
        const int g = gs + lane;
        const int r = rn;
        const float2 m = mn;
        const uint32_t dbits = r > 0 ? dn : 0u;
        fetch(g + kBinThreads);
        int x0 = 0, y0 = 0, x1 = 0, y1 = 0;
        if (r > 0) tile_rect(m.x, m.y, r, tx, ty, x0, y0, x1, y1);
        const int w = x1 - x0;
        const int area = w * (y1 - y0);
        const uint32_t nz = __ballot_sync(0xffffffffu, area > 0);
        if (nz == 0u) continue;
        int incl = area;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        const int excl = incl - area;
        __syncwarp();   // the previous group's readers are done
        if (area > 0) {
            const int c = __popc(nz & lt);
            s_rect[warp][c] = make_int4(x0, y0, w, excl);
            s_gd[warp][c] = make_uint2((uint32_t)g, dbits);
        }
        __syncwarp();
        for (int k0 = 0; k0 < total; k0 += 32) {
            const int k = k0 + lane;
            const bool starts = area > 0 && excl >= k0 && excl < k0 + 32;
            const uint32_t M = __reduce_or_sync(0xffffffffu, starts ? 1u << (excl - k0) : 0u);
            const int before = __popc(__ballot_sync(0xffffffffu, area > 0 && excl < k0));
            if (k < total) {
                const int own = before + __popc(M & (0xffffffffu >> (31 - lane))) - 1;
                const int4 rc = s_rect[warp][own];
                const uint2 gd = s_gd[warp][own];
                const int local = k - rc.w;
                // local / width by an approximate reciprocal, off by at most one, then fixed
                int qy = (int)((float)local * rcp_approx((float)rc.z));
                if (qy * rc.z > local) qy--;
                else if ((qy + 1) * rc.z <= local) qy++;
                const int yy = rc.y + qy, xx = rc.x + (local - qy * rc.z);
                f((int)gd.x, yy * tx + xx, gd.y);
            }
        }
    }
}

__global__ void __launch_bounds__(kBinThreads)
k_count_smem(gevo_layout L, int n, const float2* __restrict__ xy, const int* __restrict__ radius,
             uint32_t* __restrict__ tile_count)
{
    extern __shared__ uint32_t s_hist[];
    const int v = blockIdx.y;
    const int nt = L.tiles_x[v] * L.tiles_y[v];
    for (int t = threadIdx.x; t < nt; t += kBinThreads) s_hist[t] = 0u;
    __syncthreads();
    const int g0 = blockIdx.x * kBinChunk, g1 = min(n, g0 + kBinChunk);
    for_each_dup(L, v, n, g0, g1, xy, radius, nullptr, [&](int, int t, uint32_t) { atomicAdd(s_hist + t, 1u); });
    __syncthreads();
    uint32_t* dst = tile_count + L.tile_base[v];
    for (int t = threadIdx.x; t < nt; t += kBinThreads) {
        const uint32_t c = s_hist[t];
        if (c) atomicAdd(dst + t, c);
    }
}

__global__ void __launch_bounds__(kBinThreads)
k_scatter_smem(gevo_layout L, int n, const float2* __restrict__ xy, const int* __restrict__ radius,
               const float4* __restrict__ rgbz, const uint32_t* __restrict__ tile_start,
               uint32_t* __restrict__ tile_cursor, const uint64_t* __restrict__ d_n_dup, uint64_t cap,
               unsigned long long* __restrict__ bucket)
{
    extern __shared__ uint32_t s_hist[];
    if (*d_n_dup > cap) return;
    const int v = blockIdx.y;
    const int nt = L.tiles_x[v] * L.tiles_y[v];
    const int base = L.tile_base[v];
    for (int t = threadIdx.x; t < nt; t += kBinThreads) s_hist[t] = 0u;
    __syncthreads();
    const int g0 = blockIdx.x * kBinChunk, g1 = min(n, g0 + kBinChunk);
    for_each_dup(L, v, n, g0, g1, xy, radius, nullptr, [&](int, int t, uint32_t) { atomicAdd(s_hist + t, 1u); });
    __syncthreads();
    // reserve a contiguous run of each touched tile's bucket for this block
    for (int t = threadIdx.x; t < nt; t += kBinThreads) {
        const uint32_t c = s_hist[t];
        if (c) s_hist[t] = tile_start[base + t] + atomicAdd(tile_cursor + base + t, c);
    }
    __syncthreads();
    for_each_dup(L, v, n, g0, g1, xy, radius, rgbz, [&](int g, int t, uint32_t dbits) {
        const uint32_t slot = atomicAdd(s_hist + t, 1u);
        bucket[slot] = ((unsigned long long)dbits << 32) | (uint32_t)g;
    });
}

// The same two passes with one histogram: the counting pass keeps, per
// (block, tile), the old tile count its atomicAdd returned -- the offset of this
// block's run inside the tile's bucket -- so the scatter pass only adds the
// tile start and needs neither a second histogram nor global atomics.
__global__ void __launch_bounds__(kBinThreads)
k_count_off(gevo_layout L, int n, const float2* __restrict__ xy, const int* __restrict__ radius,
            uint32_t* __restrict__ tile_count, uint32_t* __restrict__ blk_off)
{
    extern __shared__ uint32_t s_hist[];
    const int v = blockIdx.y;
    const int nt = L.tiles_x[v] * L.tiles_y[v];
    for (int t = threadIdx.x; t < nt; t += kBinThreads) s_hist[t] = 0u;
    __syncthreads();
    const int g0 = blockIdx.x * kBinChunk, g1 = min(n, g0 + kBinChunk);
    for_each_dup(L, v, n, g0, g1, xy, radius, nullptr, [&](int, int t, uint32_t) { atomicAdd(s_hist + t, 1u); });
    __syncthreads();
    uint32_t* dst = tile_count + L.tile_base[v];
    uint32_t* off = blk_off + (size_t)gridDim.x * L.tile_base[v] + (size_t)blockIdx.x * nt;
    for (int t = threadIdx.x; t < nt; t += kBinThreads) {
        const uint32_t c = s_hist[t];
        if (c) off[t] = atomicAdd(dst + t, c);
    }
}

__global__ void __launch_bounds__(kBinThreads)
k_scatter_off(gevo_layout L, int n, const float2* __restrict__ xy, const int* __restrict__ radius,
              const float4* __restrict__ rgbz, const uint32_t* __restrict__ tile_start,
              const uint32_t* __restrict__ blk_off, const uint64_t* __restrict__ d_n_dup,
              uint64_t cap, unsigned long long* __restrict__ bucket)
{
    extern __shared__ uint32_t s_hist[];
    if (*d_n_dup > cap) return;
    const int v = blockIdx.y;
    const int nt = L.tiles_x[v] * L.tiles_y[v];
    const int base = L.tile_base[v];
    const uint32_t* off = blk_off + (size_t)gridDim.x * base + (size_t)blockIdx.x * nt;
    // entries of tiles this block does not touch hold stale values and are never used
    for (int t = threadIdx.x; t < nt; t += kBinThreads) s_hist[t] = tile_start[base + t] + off[t];
    __syncthreads();
    const int g0 = blockIdx.x * kBinChunk, g1 = min(n, g0 + kBinChunk);
    for_each_dup(L, v, n, g0, g1, xy, radius, rgbz, [&](int g, int t, uint32_t dbits) {
        const uint32_t slot = atomicAdd(s_hist + t, 1u);
        bucket[slot] = ((unsigned long long)dbits << 32) | (uint32_t)g;
    });
}

// Exclusive scan of 256 values held one per thread (blockDim == 256).
__device__ __forceinline__ uint32_t block_exscan256(uint32_t v, uint32_t* s_tmp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s_tmp[warp] = incl;
    __syncthreads();
    uint32_t off = 0;
    for (int w = 0; w < warp; w++) off += s_tmp[w];
    __syncthreads();
    return off + incl - v;
}

// The lanes whose BITS-bit value equals this lane's (the top bit marks an
// empty slot), from one ballot per bit; measured faster here than the match
// instruction on rounds of low depth bits, which hold up to 32 distinct values.
template <int BITS>
__device__ __forceinline__ uint32_t match_bits(uint32_t dg)
{
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < BITS; b++) {
        const bool bit = (dg >> b) & 1u;
        const uint32_t m = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? m : ~m;
    }
    return peers;
}

// One stable LSD pass over the byte of `a` at bit `shift`, a -> b.  Warp w owns
// the contiguous chunk [w L/8, (w+1) L/8): it counts its digits, one block scan
// turns the per-warp counts into per-warp digit offsets, then each warp scatters
// its chunk in rounds of 32 with warp-synchronous ranking (match_bits).  Order is
// kept at every level (chunk, round, lane), so the pass is stable; the block
// synchronises five times per pass whatever the tile's length.
__device__ void radix_pass(const unsigned long long* a, unsigned long long* b, int L, int shift,
                           uint32_t (*s_off)[256], uint32_t* s_tmp)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int chunk = (L + kSortWarps - 1) / kSortWarps;
    const int lo = min(L, warp * chunk), hi = min(L, lo + chunk);
    for (int d = lane; d < 256; d += 32) s_off[warp][d] = 0u;
    __syncwarp();
    for (int i = lo + lane; i < hi; i += 32) atomicAdd(&s_off[warp][(a[i] >> shift) & 255u], 1u);
    __syncthreads();
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; w++) tot += s_off[w][tid];
    uint32_t run = block_exscan256(tot, s_tmp);
#pragma unroll
    for (int w = 0; w < kSortWarps; w++) {
        const uint32_t c = s_off[w][tid];
        s_off[w][tid] = run;
        run += c;
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    for (int r = lo; r < hi; r += 32) {
        const int i = r + lane;
        const bool valid = i < hi;
        const unsigned long long key = valid ? a[i] : 0ull;
        const uint32_t dg = valid ? (uint32_t)((key >> shift) & 255u) : 256u;
        const uint32_t peers = match_bits<9>(dg);
        if (valid) b[s_off[warp][dg] + __popc(peers & lt)] = key;
        __syncwarp();
        if (valid && (__ffs(peers) - 1) == lane) s_off[warp][dg] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
}

// The shared-memory pass, on (32-bit depth key, 16-bit position in the bucket)
// pairs (6 bytes an item instead of 8, so more blocks fit on an SM) and 9-bit
// digits of (key - kmin) at bit `shift`: the
// depths of one tile span a range of about 2^26 in their bit patterns, which
// three 9-bit passes cover where four byte passes were needed.  Per-warp digit
// counts and offsets are 16-bit (a tile here holds at most 2048 items), packed
// two to a word, so the 512 counters of each warp take the bytes the 256
// 32-bit ones of the byte pass take.
__device__ void radix_pass_kv9(const uint32_t* ka, const uint16_t* ia, uint32_t* kb, uint16_t* ib,
                               int L, int shift, uint32_t kmin, uint32_t (*s_off)[256],
                               uint32_t* s_tmp)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int chunk = (L + kSortWarps - 1) / kSortWarps;
    const int lo = min(L, warp * chunk), hi = min(L, lo + chunk);
    for (int d = lane; d < 256; d += 32) s_off[warp][d] = 0u;
    __syncwarp();
    for (int i = lo + lane; i < hi; i += 32) {
        const uint32_t dg = ((ka[i] - kmin) >> shift) & 511u;
        atomicAdd(&s_off[warp][dg >> 1], 1u << ((dg & 1u) * 16));
    }
    __syncthreads();
    // thread t owns digits 2t (low halves) and 2t + 1 (high halves)
    uint32_t t0 = 0, t1 = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; w++) {
        const uint32_t pr = s_off[w][tid];
        t0 += pr & 0xffffu;
        t1 += pr >> 16;
    }
    uint32_t r0 = block_exscan256(t0 + t1, s_tmp);
    uint32_t r1 = r0 + t0;
#pragma unroll
    for (int w = 0; w < kSortWarps; w++) {
        const uint32_t pr = s_off[w][tid];
        s_off[w][tid] = r0 | (r1 << 16);
        r0 += pr & 0xffffu;
        r1 += pr >> 16;
    }
    __syncthreads();
    uint16_t* off = reinterpret_cast<uint16_t*>(s_off[warp]);
    const uint32_t lt = (1u << lane) - 1u;
    for (int r = lo; r < hi; r += 32) {
        const int i = r + lane;
        const bool valid = i < hi;
        const uint32_t key = valid ? ka[i] : 0u;
        const uint16_t idx = valid ? ia[i] : (uint16_t)0;
        const uint32_t dg = valid ? (((key - kmin) >> shift) & 511u) : 512u;
        const uint32_t peers = match_bits<10>(dg);
        if (valid) {
            const uint32_t pos = off[dg] + __popc(peers & lt);
            kb[pos] = key;
            ib[pos] = idx;
        }
        __syncwarp();
        if (valid && (__ffs(peers) - 1) == lane) off[dg] = (uint16_t)(off[dg] + __popc(peers));
        __syncwarp();
    }
    __syncthreads();
}

// 40 registers: six blocks of 256 threads fit on an SM (the sort is latency-bound)
__global__ void __launch_bounds__(kSortThreads, 6)
k_segsort(const uint32_t* __restrict__ tile_order, const uint32_t* __restrict__ tile_start,
          const uint32_t* __restrict__ tile_count, const uint64_t* __restrict__ d_n_dup,
          uint64_t cap, unsigned long long* __restrict__ bucket,
          unsigned long long* __restrict__ bucket2, unsigned long long* __restrict__ keys_out,
          uint32_t* __restrict__ vals_out)
{
    // shared-memory path: keys [2][kSortSmemItems] uint32, then positions [2][..] uint16
    extern __shared__ uint32_t s_kv[];
    __shared__ uint32_t s_off[kSortWarps][256];
    __shared__ uint32_t s_tmp[kSortWarps];
    __shared__ uint32_t s_or[kSortWarps], s_and[kSortWarps], s_min[kSortWarps], s_max[kSortWarps];
    if (*d_n_dup > cap) return;
    const uint32_t tile = tile_order[blockIdx.x];
    const int L = (int)tile_count[tile];
    if (L == 0) return;
    const uint32_t s0 = tile_start[tile];
    const int tid = threadIdx.x;
    const bool small = L <= kSortSmemItems;
    unsigned long long* a = bucket + s0;
    unsigned long long* b = bucket2 + s0;
    uint32_t* ka = s_kv;
    uint32_t* kb = s_kv + kSortSmemItems;
    uint16_t* ia = reinterpret_cast<uint16_t*>(s_kv + 2 * kSortSmemItems);
    uint16_t* ib = ia + kSortSmemItems;
    // which depth bytes vary inside this tile (long tiles), and the range of
    // the depth bit patterns (short tiles)
    uint32_t o = 0u, an = 0xffffffffu, mn = 0xffffffffu, mx = 0u;
    for (int i = tid; i < L; i += kSortThreads) {
        const uint32_t hi = (uint32_t)(a[i] >> 32);
        if (small) {
            ka[i] = hi;
            ia[i] = (uint16_t)i;
        }
        o |= hi;
        an &= hi;
        mn = min(mn, hi);
        mx = max(mx, hi);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        o |= __shfl_xor_sync(0xffffffffu, o, d);
        an &= __shfl_xor_sync(0xffffffffu, an, d);
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, d));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, d));
    }
    if ((tid & 31) == 0) {
        s_or[tid >> 5] = o; s_and[tid >> 5] = an;
        s_min[tid >> 5] = mn; s_max[tid >> 5] = mx;
    }
    __syncthreads();
    uint32_t vary = 0u, kmin = 0xffffffffu, kmax = 0u;
    {
        uint32_t oo = 0u, aa = 0xffffffffu;
#pragma unroll
        for (int w = 0; w < kSortWarps; w++) {
            oo |= s_or[w]; aa &= s_and[w];
            kmin = min(kmin, s_min[w]); kmax = max(kmax, s_max[w]);
        }
        vary = oo ^ aa;
    }
    if (small) {
        if (L > 1) {
            const int bits = 32 - __clz(kmax - kmin);   // 0 when all depths are equal
            for (int shift = 0; shift < bits; shift += 9) {
                radix_pass_kv9(ka, ia, kb, ib, L, shift, kmin, s_off, s_tmp);
                uint32_t* t = ka; ka = kb; kb = t;
                uint16_t* u = ia; ia = ib; ib = u;
            }
            // equal depth bits: order by id (runs are rare and short)
            for (int i = tid; i < L; i += kSortThreads) {
                const uint32_t hi = ka[i];
                const bool start = (i == 0 || ka[i - 1] != hi);
                if (start && i + 1 < L && ka[i + 1] == hi) {
                    int e = i + 1;
                    while (e < L && ka[e] == hi) e++;
                    for (int j = i + 1; j < e; j++) {
                        const uint16_t x = ia[j];
                        const uint32_t id = (uint32_t)a[x];
                        int m = j - 1;
                        while (m >= i && (uint32_t)a[ia[m]] > id) { ia[m + 1] = ia[m]; m--; }
                        ia[m + 1] = x;
                    }
                }
            }
            __syncthreads();
        }
        const unsigned long long th = (unsigned long long)tile << 32;
        for (int i = tid; i < L; i += kSortThreads) {
            if (keys_out) keys_out[s0 + i] = th | ka[i];
            vals_out[s0 + i] = (uint32_t)a[ia[i]];
        }
        return;
    }
    if (L > 1) {
        for (int d = 0; d < 4; d++) {
            if (((vary >> (8 * d)) & 255u) == 0u) continue;
            radix_pass(a, b, L, 32 + 8 * d, s_off, s_tmp);
            unsigned long long* t = a;
            a = b;
            b = t;
        }
        // equal depth bits: order by id (runs are rare and short)
        for (int i = tid; i < L; i += kSortThreads) {
            const uint32_t hi = (uint32_t)(a[i] >> 32);
            const bool start = (i == 0 || (uint32_t)(a[i - 1] >> 32) != hi);
            if (start && i + 1 < L && (uint32_t)(a[i + 1] >> 32) == hi) {
                int e = i + 1;
                while (e < L && (uint32_t)(a[e] >> 32) == hi) e++;
                for (int j = i + 1; j < e; j++) {
                    const unsigned long long k = a[j];
                    int m = j - 1;
                    while (m >= i && a[m] > k) { a[m + 1] = a[m]; m--; }
                    a[m + 1] = k;
                }
            }
        }
        __syncthreads();
    }
    const unsigned long long th = (unsigned long long)tile << 32;
    for (int i = tid; i < L; i += kSortThreads) {
        const unsigned long long k = a[i];
        if (keys_out) keys_out[s0 + i] = th | (k >> 32);
        vals_out[s0 + i] = (uint32_t)k;
    }
}

// ---------------------------------------------------------------------------
// Depth-ordered binning.  Every tile list is the tile's duplicates in (depth
// bits, id) order, and the depth of a (view, Gaussian) entry is the same in
// every tile it touches.  So each view's visible entries are first sorted by
// (depth bits, id) once -- a few million items: one duplicate per entry into
// one of kDepthBins depth segments of its view (a monotone quantisation of the
// depth bits between the view's least and greatest), then the segment sort
// above -- and the tile duplicates are emitted in that order by an
// order-keeping scatter.  The work is divided by duplicates, not entries: in
// depth order the nearest Gaussians (the largest splats, hundreds of tiles
// each) sit together, so equal runs of entries would carry very unequal work.
// Each view's entries get a record (Gaussian, depth bits, tile rectangle) and
// the exclusive prefix of their rectangle areas -- the index of each entry's
// first duplicate.  A unit is kOrdUnit consecutive duplicates of one view
// (one block, eight warps of kOrdWarpDups); the prefix pass also writes, for
// every warp boundary, the entry holding that duplicate, so a warp starts
// without a search and may begin or end inside an entry.  Per tile, a unit's
// run starts at the sum of the earlier units' counts (a counting pass and a
// scan over units), a warp's run inside it at the earlier warps' counts (a
// counting pass inside the block), and a duplicate's place inside its warp's
// run at the number of earlier lanes of its round with the same tile (one
// ballot per tile-index bit) plus the earlier rounds' count.  The lists come out sorted: no
// per-tile sort runs at all.
// ---------------------------------------------------------------------------
constexpr int kOrdWarpDups = kOrdUnit / 8;       // duplicates per warp of a unit (8 warps)
// Words of the unit table (uint64), filled once the per-view totals are known.
constexpr int kUnitFirst = 0;                      // [V + 1]: first unit of view v; [V]: all units
constexpr int kUnitDv = GEVO_MAX_VIEWS + 1;        // [V]: duplicates of view v
constexpr int kUnitVs = 2 * (GEVO_MAX_VIEWS + 1);  // [V]: first sorted position of view v
constexpr int kUnitD = 3 * (GEVO_MAX_VIEWS + 1);   // [0]: D over all views

// Duplicates [d0, d1) of one view in order.  rec and pre are the view's records
// (Gaussian, depth bits, x0 | y0 << 16, width | height << 16) and the exclusive
// prefix of their rectangle areas (pre[M] = the view's duplicate count), in
// (depth bits, id) order; p is the entry holding duplicate d0.  The warp walks
// 32 entries per round, lays their duplicates end to end and deals them to the
// lanes 32 at a time; the round's first entry may have started before d0 and
// its last may run past d1.  f(g, local tile, depth bits, valid, single) is
// called by every lane once per 32 duplicates (valid false past the range;
// single, the same in every lane, true when one entry holds all 32), so f may
// use warp collectives.
template <typename F>
__device__ __forceinline__ void walk_dups(int tx, const uint4* __restrict__ rec,
                                          const unsigned long long* __restrict__ pre, int M,
                                          int p, unsigned long long d0, unsigned long long d1,
                                          F&& f)
{
    __shared__ int4 s_rect[8][32];     // x0, y0, width, first duplicate (from the round's start)
    __shared__ uint2 s_gd[8][32];      // Gaussian, depth bits
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    unsigned long long cur = d0;
    for (; cur < d1 && p < M; p += 32) {
        const int q = p + lane;
        uint4 r = make_uint4(0u, 0u, 0u, 0u);
        unsigned long long a;
        if (q < M) { r = rec[q]; a = pre[q]; }
        else a = pre[M];
        const int w = (int)(r.w & 0xffffu);
        const int area = w * (int)(r.w >> 16);
        const int excl = (int)(long long)(a - cur);   // negative only for a partial first entry
        const unsigned long long rend =
            min(d1, __shfl_sync(0xffffffffu, a + (unsigned long long)area, 31));
        const int total = (int)(rend - cur);
        const uint32_t nz = __ballot_sync(0xffffffffu, area > 0);
        __syncwarp();   // the previous round's readers are done
        if (area > 0) {
            const int c = __popc(nz & lt);
            s_rect[warp][c] = make_int4((int)(r.z & 0xffffu), (int)(r.z >> 16), w, excl);
            s_gd[warp][c] = make_uint2(r.x, r.y);
        }
        __syncwarp();
        for (int k0 = 0; k0 < total; k0 += 32) {
            const int k = k0 + lane;
            const bool starts = area > 0 && excl >= k0 && excl < k0 + 32;
            const uint32_t Ms = __reduce_or_sync(0xffffffffu, starts ? 1u << (excl - k0) : 0u);
            const int before = __popc(__ballot_sync(0xffffffffu, area > 0 && excl < k0));
            int tl = -1, gg = 0;
            uint32_t db = 0u;
            if (k < total) {
                const int own = before + __popc(Ms & (0xffffffffu >> (31 - lane))) - 1;
                const int4 rc = s_rect[warp][own];
                const uint2 gd = s_gd[warp][own];
                const int local = k - rc.w;
                int qy = (int)((float)local * rcp_approx((float)rc.z));
                if (qy * rc.z > local) qy--;
                else if ((qy + 1) * rc.z <= local) qy++;
                tl = (rc.y + qy) * tx + rc.x + (local - qy * rc.z);
                gg = (int)gd.x;
                db = gd.y;
            }
            // no entry but the first starts inside these 32 duplicates: one
            // entry holds them all, so their tiles are distinct
            f(gg, tl, db, k < total, (Ms & ~1u) == 0u);
        }
        cur = rend;
    }
}

// Dynamic shared-memory limits of the binning and sort kernels, raised once per
// device (the attribute belongs to the device's context) and only upwards.
// Host threads may sort concurrently, so the record sits behind a mutex.
static std::mutex g_attr_mu;

// Per view: max(~depth bits) (so the least depth is its complement), max(depth
// bits) and the count of visible entries (radius > 0); per entry its depth bits
// dk (kInvisible when radius <= 0: the bits of a positive depth are below it)
// and, when visible, its tile rectangle rect (x0 | y0 << 16, width | height <<
// 16).  Block (x, v) reduces 1024 entries of view v.
constexpr uint32_t kInvisible = 0xffffffffu;
__global__ void __launch_bounds__(256)
k_ord_stat(gevo_layout L, int n, const float2* __restrict__ xy, const int* __restrict__ radius,
           const float4* __restrict__ rgbz, uint32_t* __restrict__ stat,
           uint32_t* __restrict__ dk, uint2* __restrict__ rect)
{
    __shared__ uint32_t s_r[3][8];
    const int v = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t vb = (size_t)v * n;
    const int tx = L.tiles_x[v], ty = L.tiles_y[v];
    uint32_t nmin = 0u, mx = 0u, cnt = 0u;
    int rr[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {   // the four radii in flight together
        const int g = blockIdx.x * 1024 + i * 256 + threadIdx.x;
        rr[i] = g < n ? radius[vb + g] : 0;
    }
    // then the visible entries' depths and means, all four before any use
    uint32_t dd[4];
    float2 mm[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int g = blockIdx.x * 1024 + i * 256 + threadIdx.x;
        dd[i] = 0u;
        mm[i] = make_float2(0.f, 0.f);
        if (rr[i] > 0) {
            dd[i] = __float_as_uint(__ldg(reinterpret_cast<const float*>(rgbz + vb + g) + 3));
            mm[i] = xy[vb + g];
        }
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int g = blockIdx.x * 1024 + i * 256 + threadIdx.x;
        if (g >= n) break;
        const int r = rr[i];
        if (r <= 0) { dk[vb + g] = kInvisible; continue; }
        const uint32_t d = dd[i];
        const float2 m = mm[i];
        int x0, y0, x1, y1;
        tile_rect(m.x, m.y, r, tx, ty, x0, y0, x1, y1);
        dk[vb + g] = d;
        rect[vb + g] = make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16),
                                  (uint32_t)(x1 - x0) | ((uint32_t)(y1 - y0) << 16));
        nmin = max(nmin, ~d);
        mx = max(mx, d);
        cnt++;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nmin = max(nmin, __shfl_xor_sync(0xffffffffu, nmin, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) { s_r[0][warp] = nmin; s_r[1][warp] = mx; s_r[2][warp] = cnt; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; w++) {
            nmin = max(nmin, s_r[0][w]); mx = max(mx, s_r[1][w]); cnt += s_r[2][w];
        }
        if (cnt) {
            atomicMax(stat + 4 * v, nmin);
            atomicMax(stat + 4 * v + 1, mx);
            atomicAdd(stat + 4 * v + 2, cnt);
        }
    }
}

// Depth segments of view v: d -> ((d - least) mul) >> 32 with
// mul = floor(2^32 kDepthBins / (greatest - least + 1)), a monotone map of the
// view's depth bits onto 0 .. kDepthBins - 1 (the product stays below
// kDepthBins 2^32) with one division per block instead of one per entry.
__device__ __forceinline__ unsigned long long depth_mul(const uint32_t* stat, int v)
{
    const uint32_t lo = ~stat[4 * v], hi = stat[4 * v + 1];
    return ((unsigned long long)kDepthBins << 32) / ((unsigned long long)(hi - lo) + 1ull);
}

__device__ __forceinline__ int depth_segment(uint32_t lo, unsigned long long mul, uint32_t d)
{
    return (int)(((unsigned long long)(d - lo) * mul) >> 32);
}

// Count (SCATTER false) or place (SCATTER true) each visible entry in its depth
// segment; block (x, v) takes kOrdSegChunk entries of view v, kOrdSegChunk / 256
// per thread.  The block counts its entries per segment in shared memory (the
// shared atomic's old value ranks an entry inside the block's share); placing,
// it reserves one run per (block, segment) with a single global atomic.  The
// order inside a segment is left to the segment sort.
constexpr int kOrdSegChunk = 4096;   // entries per block of the depth-segment passes
                                     // (measured: 4096 a little faster than 1024 and 2048)

template <bool SCATTER>
__global__ void __launch_bounds__(256)
k_ord_seg(int n, const uint32_t* __restrict__ dk, const uint32_t* __restrict__ stat,
          uint32_t* __restrict__ seg_count, const uint32_t* __restrict__ seg_start,
          uint32_t* __restrict__ seg_cursor, unsigned long long* __restrict__ b1)
{
    constexpr int PER = kOrdSegChunk / 256;
    __shared__ uint32_t s_h[kDepthBins];
    __shared__ unsigned long long s_mul;
    const int v = blockIdx.y;
    const size_t vb = (size_t)v * n;
    for (int i = threadIdx.x; i < kDepthBins; i += blockDim.x) s_h[i] = 0u;
    if (threadIdx.x == 0) s_mul = depth_mul(stat, v);
    __syncthreads();
    const uint32_t lo = ~stat[4 * v];
    const unsigned long long mul = s_mul;
    uint32_t d[PER];
    int rank[PER];
#pragma unroll
    for (int i = 0; i < PER; i++) {   // every load in flight before the first atomic
        const int g = blockIdx.x * kOrdSegChunk + i * 256 + threadIdx.x;
        d[i] = g < n ? dk[vb + g] : kInvisible;
    }
#pragma unroll
    for (int i = 0; i < PER; i++) {
        rank[i] = d[i] != kInvisible
                      ? (int)atomicAdd(s_h + depth_segment(lo, mul, d[i]), 1u)
                      : 0;
    }
    __syncthreads();
    if constexpr (!SCATTER) {
        for (int i = threadIdx.x; i < kDepthBins; i += blockDim.x)
            if (s_h[i]) atomicAdd(seg_count + v * kDepthBins + i, s_h[i]);
    } else {
#pragma unroll
        for (int i = threadIdx.x; i < kDepthBins; i += 256)   // the block's reservations together
            if (s_h[i]) s_h[i] = seg_start[v * kDepthBins + i] +
                                 atomicAdd(seg_cursor + v * kDepthBins + i, s_h[i]);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < PER; i++) {
            if (d[i] == kInvisible) continue;
            const int g = blockIdx.x * kOrdSegChunk + i * 256 + threadIdx.x;
            const int sg = depth_segment(lo, mul, d[i]);
            b1[s_h[sg] + rank[i]] = ((unsigned long long)d[i] << 32) | (uint32_t)g;
        }
    }
}

// First sorted position of view v (the visible entries of earlier views).
// Called by whole warps: the lanes load the earlier views' counts at once.
__device__ __forceinline__ uint32_t view_start(const uint32_t* stat, int v)
{
    const int lane = threadIdx.x & 31;
    uint32_t s = 0u;
    for (int u0 = 0; u0 < v; u0 += 32) {
        const int u = u0 + lane;
        s += __reduce_add_sync(0xffffffffu, u < v ? stat[4 * u + 2] : 0u);
    }
    return s;
}

// Exclusive scan over the NT threads of the block; total gets the block's sum.
// Every thread of the block must call it (it holds two barriers).
template <int NT>
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long x,
                                                              unsigned long long& total)
{
    __shared__ unsigned long long s_w[NT / 32 + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long y = lane < NT / 32 ? s_w[lane] : 0ull;
        unsigned long long wi = y;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long z = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += z;
        }
        if (lane < NT / 32) s_w[lane] = wi - y;
        if (lane == 31) s_w[NT / 32] = wi;
    }
    __syncthreads();
    const unsigned long long r = s_w[warp] + incl - x;
    total = s_w[NT / 32];
    __syncthreads();   // s_w is free for the next call
    return r;
}

// Per sorted entry p of view v: its record (Gaussian, depth bits,
// x0 | y0 << 16, width | height << 16 of its tile rectangle) -- the depth bits
// from the depth sort's keys, the rectangle gathered from the stat pass's; per
// block of kOrdScanItems entries the sum of the rectangle areas, at
// bsum[v gridDim.x + blockIdx.x].
__global__ void __launch_bounds__(256)
k_ord_rec(int n, const uint32_t* __restrict__ stat, const uint32_t* __restrict__ sorted,
          const unsigned long long* __restrict__ dkeys, const uint2* __restrict__ rect,
          uint4* __restrict__ rec, unsigned long long* __restrict__ bsum)
{
    const int v = blockIdx.y;
    const int M = (int)stat[4 * v + 2];
    const int p0 = blockIdx.x * kOrdScanItems;
    if (p0 >= M) return;   // the whole block: before any barrier
    const uint32_t vs = view_start(stat, v);
    const size_t vb = (size_t)v * n;
    constexpr int PER = kOrdScanItems / 256;
    unsigned long long sum = 0ull;
    uint32_t g[PER];
#pragma unroll
    for (int i = 0; i < PER; i++) {   // the ids, then the gathers, all in flight together
        const int p = p0 + i * 256 + threadIdx.x;
        g[i] = p < M ? sorted[vs + p] : 0u;
    }
#pragma unroll
    for (int i = 0; i < PER; i++) {
        const int p = p0 + i * 256 + threadIdx.x;
        if (p < M) {
            const uint2 rc = rect[vb + g[i]];
            rec[vs + p] = make_uint4(g[i], (uint32_t)dkeys[vs + p], rc.x, rc.y);
            sum += (unsigned long long)((rc.y & 0xffffu) * (rc.y >> 16));
        }
    }
    unsigned long long total;
    block_excl_scan<256>(sum, total);
    if (threadIdx.x == 0) bsum[(size_t)v * gridDim.x + blockIdx.x] = total;
}

// One block.  Per view (one warp each): the block sums become their exclusive
// running sums (in place) and the total is the view's duplicate count D_v.
// Then, in one thread, the unit table -- first unit of each view
// (ceil(D_v / kOrdUnit) units each), D_v, the view's first sorted position and D
// -- and each view's prefix end pre[vs + v + M_v] = D_v.  When D exceeds the
// capacity no unit is made, so the counting and scatter passes do nothing and
// only D is reported.
__global__ void __launch_bounds__(1024)
k_ord_bscan(int V, int nbs, uint64_t cap, const uint32_t* __restrict__ stat,
            unsigned long long* __restrict__ bsum, unsigned long long* __restrict__ units,
            unsigned long long* __restrict__ pre)
{
    __shared__ unsigned long long s_dv[GEVO_MAX_VIEWS];
    __shared__ uint32_t s_m[GEVO_MAX_VIEWS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = warp; v < V; v += 32) {
        const uint32_t M = stat[4 * v + 2];
        const int nb = (int)((M + kOrdScanItems - 1) / kOrdScanItems);
        unsigned long long* bs = bsum + (size_t)v * nbs;
        unsigned long long carry = 0ull;
        for (int c0 = 0; c0 < nb; c0 += 128) {   // four steps' loads at a time
            unsigned long long xs[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int i = c0 + 32 * k + lane;
                xs[k] = i < nb ? bs[i] : 0ull;
            }
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int i = c0 + 32 * k + lane;
                const unsigned long long x = xs[k];
                unsigned long long incl = x;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (i < nb) bs[i] = carry + incl - x;
                carry += __shfl_sync(0xffffffffu, incl, 31);
            }
        }
        if (lane == 0) {
            s_dv[v] = carry;
            s_m[v] = M;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long D = 0ull, vs = 0ull;
        for (int v = 0; v < V; v++) D += s_dv[v];
        const bool overflow = D > cap;
        unsigned long long u = 0ull;
        for (int v = 0; v < V; v++) {
            const uint32_t M = s_m[v];
            units[kUnitFirst + v] = u;
            units[kUnitDv + v] = s_dv[v];
            units[kUnitVs + v] = vs;
            pre[vs + v + M] = s_dv[v];
            if (!overflow) u += (s_dv[v] + kOrdUnit - 1) / kOrdUnit;
            vs += M;
        }
        units[kUnitFirst + V] = u;
        units[kUnitD] = D;
    }
}

// Per sorted entry p of view v: pre[vs + v + p] = the index of its first
// duplicate among the view's duplicates (the exclusive prefix of the areas in
// (depth bits, id) order); and for every warp boundary j kOrdWarpDups that
// falls inside its duplicates, wstart[8 (first unit of v) + j] = p.  Thread i
// of block (x, v) takes the kOrdScanItems / 256 consecutive entries from
// x kOrdScanItems + i kOrdScanItems / 256.
__global__ void __launch_bounds__(256)
k_ord_pre(const uint32_t* __restrict__ stat, const unsigned long long* __restrict__ units,
          const uint4* __restrict__ rec, const unsigned long long* __restrict__ bsum,
          uint64_t cap, unsigned long long* __restrict__ pre, uint32_t* __restrict__ wstart)
{
    constexpr int PER = kOrdScanItems / 256;
    const int v = blockIdx.y;
    const int M = (int)stat[4 * v + 2];
    const int p0 = blockIdx.x * kOrdScanItems;
    if (p0 >= M) return;   // the whole block: before any barrier
    const unsigned long long vs = units[kUnitVs + v];
    const bool keep = units[kUnitD] <= cap;
    uint32_t* ws = wstart + units[kUnitFirst + v] * 8ull;
    const uint32_t* wh = reinterpret_cast<const uint32_t*>(rec + vs) + 3;   // .w of each record
    const int q0 = p0 + threadIdx.x * PER;
    const unsigned long long base = bsum[(size_t)v * gridDim.x + blockIdx.x];   // before the barriers
    uint32_t area[PER];
    unsigned long long sum = 0ull;
#pragma unroll
    for (int i = 0; i < PER; i++) {
        const int q = q0 + i;
        uint32_t a = 0u;
        if (q < M) {
            const uint32_t x = wh[4 * (size_t)q];
            a = (x & 0xffffu) * (x >> 16);
        }
        area[i] = a;
        sum += a;
    }
    unsigned long long tot;
    unsigned long long run = base + block_excl_scan<256>(sum, tot);
    unsigned long long* pv = pre + vs + v;
#pragma unroll
    for (int i = 0; i < PER; i++) {
        const int q = q0 + i;
        if (q < M) {
            pv[q] = run;
            if (keep && area[i] > 0u)
                for (unsigned long long j = (run + kOrdWarpDups - 1) / kOrdWarpDups;
                     j * kOrdWarpDups < run + area[i]; j++)
                    ws[j] = (uint32_t)q;
        }
        run += area[i];
    }
}

// The view v of unit u, first[v] <= u < first[v + 1] (the table's end is the
// unit count): the number of views whose successor's first unit is at or
// below u (first units rise with the view).  Called by whole warps: the
// lanes read the table at once and count by ballot, one memory latency instead
// of one per view.
__device__ __forceinline__ int view_of_unit(const unsigned long long* units, int n_views, int u)
{
    const int lane = threadIdx.x & 31;
    int v = 0;
    for (int k0 = 0; k0 < n_views; k0 += 32) {
        const int k = k0 + lane;
        const bool below = k < n_views && units[kUnitFirst + k + 1] <= (unsigned long long)u;
        v += __popc(__ballot_sync(0xffffffffu, below));
    }
    return v;
}

// Per unit u and tile t of its view: the unit's duplicate count, at
// cnt[u max_tiles + t], and per warp w of the unit the number of the unit's
// duplicates of tile t that earlier warps hold -- 16 bits, two tiles to a word,
// at wofs[(8u + w) rwm + t / 2] with rwm = ceil(max_tiles / 2).  A warp's
// kOrdWarpDups duplicates hold at most that many of one tile and the unit at
// most kOrdUnit, so 16 bits hold every count and offset.  A persistent grid
// walks the units.
__global__ void __launch_bounds__(256)
k_ord_count(gevo_layout L, int max_tiles, const uint32_t* __restrict__ stat,
            const unsigned long long* __restrict__ units, const uint4* __restrict__ rec,
            const unsigned long long* __restrict__ pre, const uint32_t* __restrict__ wstart,
            uint32_t* __restrict__ cnt, uint32_t* __restrict__ wofs)
{
    extern __shared__ uint32_t s_rel[];   // [8][rw] per-warp counts, 16 bits per tile
    const int warp = threadIdx.x >> 5;
    const int rwm = (max_tiles + 1) / 2;
    const int n_units = (int)units[kUnitFirst + L.n_views];
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const int v = view_of_unit(units, L.n_views, u);
        const int nt = L.tiles_x[v] * L.tiles_y[v];
        const int rw = (nt + 1) / 2;
        for (int i = threadIdx.x; i < 8 * rw; i += blockDim.x) s_rel[i] = 0u;
        __syncthreads();
        const unsigned long long Dv = units[kUnitDv + v];
        const unsigned long long w0 =
            (unsigned long long)(u - (int)units[kUnitFirst + v]) * kOrdUnit +
            (unsigned long long)warp * kOrdWarpDups;
        if (w0 < Dv) {
            const unsigned long long vs = units[kUnitVs + v];
            uint32_t* my = s_rel + warp * rw;
            walk_dups(L.tiles_x[v], rec + vs, pre + vs + v, (int)stat[4 * v + 2],
                      (int)wstart[(size_t)u * 8 + warp], w0, min(Dv, w0 + kOrdWarpDups),
                      [&](int, int t, uint32_t, bool ok, bool) {
                          if (ok) atomicAdd(my + (t >> 1), 1u << ((t & 1) * 16));
                      });
        }
        __syncthreads();
        uint32_t* wo = wofs + (size_t)u * 8 * rwm;
        uint32_t* dst = cnt + (size_t)u * max_tiles;
        for (int q = threadIdx.x; q < rw; q += blockDim.x) {
            uint32_t r0 = 0u, r1 = 0u;
#pragma unroll
            for (int w = 0; w < 8; w++) {
                const uint32_t c = s_rel[w * rw + q];
                wo[(size_t)w * rwm + q] = r0 | (r1 << 16);
                r0 += c & 0xffffu;
                r1 += c >> 16;
            }
            dst[2 * q] = r0;
            if (2 * q + 1 < nt) dst[2 * q + 1] = r1;
        }
        __syncthreads();
    }
}

// The same counts from the entries' rectangles instead of their duplicates.
// A warp's duplicates of one entry are a run of the entry's row-major tile
// indices, so they cover at most three rectangles of tiles (the rest of a first
// row, whole rows, the start of a last row) -- one for an entry the warp holds
// whole.  Each rectangle adds its four corners to a 2-D difference array
// (per warp, th rows of stride S = tw | 1 words, odd so that the row and column
// passes below meet no bank conflicts), and two running-sum passes (along the
// rows, then down the columns) turn it into the per-tile counts.  A word holds
// the +1 corners in its low half and the -1 corners in its high half: each of a
// warp's at most 1024 entries (every one holds at least one of its 1024
// duplicates) adds at most three rectangles of two corners of either sign, so
// no running sum of a half passes 6144, the halves never carry, and a count is
// low - high.  It executes about 60% of the instructions of the walk over the
// duplicates (9.5M against 15.8M on four 640 x 480 views of 500k Gaussians);
// the arrays take 32 S th bytes of shared memory, so larger views keep
// k_ord_count.
__device__ __forceinline__ void diff_rect(uint32_t* a, int S, int tw, int th, int xa, int xb,
                                          int ya, int yb)
{
    // tiles xa..xb x ya..yb (inclusive); corners past the grid change nothing
    atomicAdd(a + ya * S + xa, 1u);
    if (xb + 1 < tw) atomicAdd(a + ya * S + xb + 1, 0x10000u);
    if (yb + 1 < th) {
        atomicAdd(a + (yb + 1) * S + xa, 0x10000u);
        if (xb + 1 < tw) atomicAdd(a + (yb + 1) * S + xb + 1, 1u);
    }
}

__global__ void __launch_bounds__(256)
k_ord_count_rect(gevo_layout L, int max_tiles, int cells, const uint32_t* __restrict__ stat,
                 const unsigned long long* __restrict__ units, const uint4* __restrict__ rec,
                 const unsigned long long* __restrict__ pre, const uint32_t* __restrict__ wstart,
                 uint32_t* __restrict__ cnt, uint32_t* __restrict__ wofs)
{
    extern __shared__ uint32_t s_d[];   // [8][cells]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rwm = (max_tiles + 1) / 2;
    const int n_units = (int)units[kUnitFirst + L.n_views];
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const int v = view_of_unit(units, L.n_views, u);
        const int tw = L.tiles_x[v], th = L.tiles_y[v], S = tw | 1;
        const int nt = tw * th, rw = (nt + 1) / 2;
        uint32_t* a = s_d + warp * cells;
        for (int i = lane; i < th * S; i += 32) a[i] = 0u;
        __syncwarp();
        const unsigned long long Dv = units[kUnitDv + v];
        const unsigned long long w0 =
            (unsigned long long)(u - (int)units[kUnitFirst + v]) * kOrdUnit +
            (unsigned long long)warp * kOrdWarpDups;
        if (w0 < Dv) {
            const unsigned long long w1 = min(Dv, w0 + kOrdWarpDups);
            const unsigned long long vs = units[kUnitVs + v];
            const uint4* rv = rec + vs;
            const unsigned long long* pv = pre + vs + v;
            const int M = (int)stat[4 * v + 2];
            // chunks of 4 x 32 entries with every load issued before any use (one
            // memory latency per chunk; a warp's ~116 entries are mostly one chunk)
            constexpr int kChunk = 4;
            for (int p = (int)wstart[(size_t)u * 8 + warp] + lane;; p += 32 * kChunk) {
                unsigned long long pa[kChunk];
                uint4 rr[kChunk];
#pragma unroll
                for (int i = 0; i < kChunk; i++) {
                    const int q = p + 32 * i;
                    pa[i] = q < M ? pv[q] : ~0ull;            // past the view: past the warp
                    rr[i] = q < M ? rv[q] : make_uint4(0u, 0u, 0u, 0u);
                }
#pragma unroll
                for (int i = 0; i < kChunk; i++) {
                    if (pa[i] >= w1) continue;        // starts past the warp's duplicates
                    const uint4 r = rr[i];
                    const int w = (int)(r.w & 0xffffu), area = w * (int)(r.w >> 16);
                    const int lo = pa[i] >= w0 ? 0 : (int)(w0 - pa[i]);
                    const int hi = (int)min((unsigned long long)area, w1 - pa[i]);
                    if (lo >= hi) continue;           // no tiles, or all before the warp's first
                    const int x0 = (int)(r.z & 0xffffu), y0 = (int)(r.z >> 16);
                    if (lo == 0 && hi == area) {      // the whole rectangle
                        diff_rect(a, S, tw, th, x0, x0 + w - 1, y0, y0 + (int)(r.w >> 16) - 1);
                        continue;
                    }
                    const int r0 = lo / w, c0 = lo - r0 * w, r1 = (hi - 1) / w,
                              c1 = hi - 1 - r1 * w;
                    if (r0 == r1) {
                        diff_rect(a, S, tw, th, x0 + c0, x0 + c1, y0 + r0, y0 + r0);
                    } else {
                        diff_rect(a, S, tw, th, x0 + c0, x0 + w - 1, y0 + r0, y0 + r0);
                        if (r1 > r0 + 1)
                            diff_rect(a, S, tw, th, x0, x0 + w - 1, y0 + r0 + 1, y0 + r1 - 1);
                        diff_rect(a, S, tw, th, x0, x0 + c1, y0 + r1, y0 + r1);
                    }
                }
                // entries start in order: go on while the chunk's last one starts inside
                if (__shfl_sync(0xffffffffu, pa[kChunk - 1], 31) >= w1) break;
            }
        }
        __syncwarp();
        // running sums along each row, then down each column; four loads ahead of
        // their stores, so that they overlap
        for (int y = lane; y < th; y += 32) {
            uint32_t run = 0u;
            uint32_t* row = a + y * S;
            int x = 0;
            for (; x + 4 <= tw; x += 4) {
                const uint32_t c0 = row[x], c1 = row[x + 1], c2 = row[x + 2], c3 = row[x + 3];
                row[x] = run += c0;
                row[x + 1] = run += c1;
                row[x + 2] = run += c2;
                row[x + 3] = run += c3;
            }
            for (; x < tw; x++) row[x] = run += row[x];
        }
        __syncwarp();
        for (int x = lane; x < tw; x += 32) {
            uint32_t run = 0u;
            uint32_t* col = a + x;
            int y = 0;
            for (; y + 4 <= th; y += 4) {
                const uint32_t c0 = col[y * S], c1 = col[(y + 1) * S], c2 = col[(y + 2) * S],
                               c3 = col[(y + 3) * S];
                col[y * S] = run += c0;
                col[(y + 1) * S] = run += c1;
                col[(y + 2) * S] = run += c2;
                col[(y + 3) * S] = run += c3;
            }
            for (; y < th; y++) col[y * S] = run += col[y * S];
        }
        __syncthreads();
        uint32_t* wo = wofs + (size_t)u * 8 * rwm;
        uint32_t* dst = cnt + (size_t)u * max_tiles;
        for (int q = threadIdx.x; q < rw; q += blockDim.x) {
            const int t0 = 2 * q, y = t0 / tw, x = t0 - y * tw;
            const int i0 = y * S + x;
            const bool two = t0 + 1 < nt;
            const int i1 = x + 1 < tw ? i0 + 1 : i0 + S - x;   // the next row's first tile
            uint32_t r0 = 0u, r1 = 0u;
#pragma unroll
            for (int w = 0; w < 8; w++) {
                wo[(size_t)w * rwm + q] = r0 | (r1 << 16);
                const uint32_t c0 = s_d[w * cells + i0];
                r0 += (c0 & 0xffffu) - (c0 >> 16);
                if (two) {
                    const uint32_t c1 = s_d[w * cells + i1];
                    r1 += (c1 & 0xffffu) - (c1 >> 16);
                }
            }
            dst[t0] = r0;
            if (two) dst[t0 + 1] = r1;
        }
        __syncthreads();
    }
}

// Per tile of a view: its unit counts become their exclusive running sums (in
// unit order, in place) and the total is the tile's count.  Block (x, v) takes
// the 32 tiles 32x .. 32x + 31 of view v, one per lane; its eight warps split
// the view's units into eight runs, sum their run per tile, and after the
// warps' sums are scanned in shared memory write the running sums.
__global__ void __launch_bounds__(256)
k_ord_scan(gevo_layout L, int max_tiles, const unsigned long long* __restrict__ units,
           uint32_t* __restrict__ cnt, uint32_t* __restrict__ tile_count)
{
    __shared__ uint32_t s_sum[8][32];
    const int v = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nt = L.tiles_x[v] * L.tiles_y[v];
    const int t = blockIdx.x * 32 + lane;
    if (blockIdx.x * 32 >= nt) return;   // the whole block: before any barrier
    const int u0 = (int)units[kUnitFirst + v], nu = (int)units[kUnitFirst + v + 1] - u0;
    const int a = u0 + (int)((long long)nu * warp / 8), b = u0 + (int)((long long)nu * (warp + 1) / 8);
    uint32_t* c = cnt + t;
    const size_t mt = (size_t)max_tiles;
    uint32_t sum = 0u;
    if (t < nt) {
#pragma unroll 4
        for (int u = a; u < b; u++) sum += c[(size_t)u * mt];
    }
    s_sum[warp][lane] = sum;
    __syncthreads();
    uint32_t run = 0u;
    for (int w = 0; w < warp; w++) run += s_sum[w][lane];
    if (t < nt) {
        int u = a;
        for (; u + 4 <= b; u += 4) {   // four loads ahead of their stores
            const uint32_t x0 = c[u * mt], x1 = c[(u + 1) * mt], x2 = c[(u + 2) * mt],
                           x3 = c[(u + 3) * mt];
            c[u * mt] = run;
            c[(u + 1) * mt] = run += x0;
            c[(u + 2) * mt] = run += x1;
            c[(u + 3) * mt] = run += x2;
            run += x3;
        }
        for (; u < b; u++) {
            const uint32_t x = c[u * mt];
            c[u * mt] = run;
            run += x;
        }
        if (warp == 7) tile_count[L.tile_base[v] + t] = run;
    }
}

// The order-keeping scatter, one unit per block at a time.  Shared memory: the
// unit's first slot per tile [T_v], then per warp and tile the 16-bit running
// offset (two tiles to a 32-bit word) that starts as the counting pass's count
// of the earlier warps' duplicates and grows by each round's.
__global__ void __launch_bounds__(256)
k_ord_scatter(gevo_layout L, int max_tiles, const uint32_t* __restrict__ stat,
              const unsigned long long* __restrict__ units, const uint4* __restrict__ rec,
              const unsigned long long* __restrict__ pre, const uint32_t* __restrict__ wstart,
              const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ wofs,
              const uint32_t* __restrict__ tile_start, unsigned long long* __restrict__ keys,
              uint32_t* __restrict__ vals)
{
    extern __shared__ uint32_t s_dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int rwm = (max_tiles + 1) / 2;
    const int n_units = (int)units[kUnitFirst + L.n_views];
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const int v = view_of_unit(units, L.n_views, u);
        const int nt = L.tiles_x[v] * L.tiles_y[v];
        const int rw = (nt + 1) / 2;   // words per warp row
        uint32_t* s_base = s_dyn;
        uint32_t* s_rel = s_dyn + 2 * rw;
        // the unit's first slot per tile and the warps' running offsets
        const int tb = L.tile_base[v];
        const uint32_t* off = cnt + (size_t)u * max_tiles;
        for (int t = threadIdx.x; t < nt; t += blockDim.x) s_base[t] = tile_start[tb + t] + off[t];
        // each warp its own row of running offsets
        const uint32_t* wo = wofs + ((size_t)u * 8 + warp) * rwm;
        for (int q = lane; q < rw; q += 32) s_rel[warp * rw + q] = wo[q];
        __syncthreads();
        const unsigned long long Dv = units[kUnitDv + v];
        const unsigned long long w0 =
            (unsigned long long)(u - (int)units[kUnitFirst + v]) * kOrdUnit +
            (unsigned long long)warp * kOrdWarpDups;
        if (w0 < Dv) {
            const unsigned long long vs = units[kUnitVs + v];
            // the warp's offsets, one 16-bit word per tile (tile t is the half of
            // word t / 2 that the packing puts it in: little-endian)
            uint16_t* my = reinterpret_cast<uint16_t*>(s_rel + warp * rw);
            // the lanes of a round with the same tile, by one ballot per bit of the
            // tile index (the match instruction's cost grows with the distinct
            // values a round holds: up to 32 here; measured 0.10 ms slower)
            const int tbits = 32 - __clz(max(nt - 1, 1));
            walk_dups(L.tiles_x[v], rec + vs, pre + vs + v, (int)stat[4 * v + 2],
                      (int)wstart[(size_t)u * 8 + warp], w0, min(Dv, w0 + kOrdWarpDups),
                      [&](int g, int t, uint32_t dbits, bool ok, bool single) {
                uint32_t peers = 1u << lane;
                if (!single) {
                    peers = __ballot_sync(0xffffffffu, ok);
                    for (int b = 0; b < tbits; b++) {
                        const bool bit = (t >> b) & 1;
                        const uint32_t B = __ballot_sync(0xffffffffu, bit);
                        peers &= bit ? B : ~B;
                    }
                }
                const uint32_t rank = __popc(peers & lt);
                uint32_t o = 0u;
                if (ok) {
                    o = my[t];
                    const uint32_t slot = s_base[t] + o + rank;
                    if (keys) keys[slot] = ((unsigned long long)(tb + t) << 32) | dbits;
                    vals[slot] = (uint32_t)g;
                }
                __syncwarp();   // every peer has read the tile's offset
                if (ok && (peers >> lane) == 1u) my[t] = (uint16_t)(o + rank + 1u);   // last peer
                __syncwarp();
            });
        }
        __syncthreads();
    }
}

static void bin_attributes(size_t bin_smem)
{
    static size_t done[256] = {0};
    int dev = 0;
    if (bin_smem <= 48 * 1024 || cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256)
        return;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (bin_smem > done[dev]) {
        cudaFuncSetAttribute(k_count_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bin_smem);
        cudaFuncSetAttribute(k_scatter_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bin_smem);
        cudaFuncSetAttribute(k_count_off, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bin_smem);
        cudaFuncSetAttribute(k_scatter_off, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bin_smem);
        done[dev] = bin_smem;
    }
}

static void segsort_attributes(size_t smem)
{
    static bool done[256] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (!done[dev]) {
        cudaFuncSetAttribute(k_segsort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        done[dev] = true;
    }
}

static void ord_attributes(size_t smem)
{
    static size_t done[256] = {0};
    int dev = 0;
    if (smem <= 48 * 1024 || cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (smem > done[dev]) {
        cudaFuncSetAttribute(k_ord_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_ord_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        done[dev] = smem;
    }
}

// Shared memory of the rectangle count, at most; views needing more count by
// walking their duplicates (k_ord_count).  112 KB hold the difference arrays of
// views up to 3584 words a warp (75 x 43 tiles: 1200 x 680 pixels).
constexpr size_t kOrdRectSmem = 112 * 1024;

static void count_rect_attributes(size_t smem)
{
    static size_t done[256] = {0};
    int dev = 0;
    if (smem <= 48 * 1024 || cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (smem > done[dev]) {
        cudaFuncSetAttribute(k_ord_count_rect, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        done[dev] = smem;
    }
}

// gevo_bin_sort on layouts whose views have at most kOrdMaxTiles tiles: the
// per-view depth sort, then the order-keeping scatter (see above).
static gevo_status bin_sort_ordered(const gevo_layout& L, int32_t n, const gevo_proj& proj,
                                    uint64_t cap, uint64_t* keys, uint32_t* vals,
                                    uint32_t* ranges, uint64_t* d_n_dup, char* ws,
                                    const WsLayout& w, cudaStream_t st)
{
    const int V = L.n_views, T = L.total_tiles, S = V * kDepthBins;
    uint32_t* err = reinterpret_cast<uint32_t*>(ws + w.err);
    uint32_t* tile_count = reinterpret_cast<uint32_t*>(ws + w.tile_count);
    uint32_t* tile_cursor = reinterpret_cast<uint32_t*>(ws + w.tile_cursor);
    uint32_t* tile_order = reinterpret_cast<uint32_t*>(ws + w.tile_order);
    uint32_t* tile_start = reinterpret_cast<uint32_t*>(ws + w.tile_start);
    uint32_t* stat = reinterpret_cast<uint32_t*>(ws + w.ord_stat);
    uint32_t* seg = reinterpret_cast<uint32_t*>(ws + w.ord_seg);
    uint32_t* seg_count = seg;
    uint32_t* seg_start = seg + S;
    uint32_t* seg_cursor = seg + 2 * S + 1;
    uint32_t* seg_order = seg + 3 * S + 1;
    uint32_t* seg_ranges = seg + 4 * S + 1;
    uint64_t* n_vis = reinterpret_cast<uint64_t*>(ws + w.ord_total);
    uint32_t* err1 = reinterpret_cast<uint32_t*>(ws + w.ord_total + 8);
    auto* b1 = reinterpret_cast<unsigned long long*>(ws + w.ord_b1);
    auto* b2 = reinterpret_cast<unsigned long long*>(ws + w.ord_b2);
    uint32_t* sorted = reinterpret_cast<uint32_t*>(ws + w.ord_vals);
    auto* rec = reinterpret_cast<uint4*>(ws + w.ord_b1);   // b1 is free once the depth sort ends
    uint32_t* dk = reinterpret_cast<uint32_t*>(ws + w.ord_vals);   // read before the sort writes ids
    auto* rect = reinterpret_cast<uint2*>(ws + w.ord_pre);         // read before the prefix is written
    auto* dkeys = reinterpret_cast<unsigned long long*>(ws + w.ord_dkeys);
    auto* pre = reinterpret_cast<unsigned long long*>(ws + w.ord_pre);
    auto* bsum = reinterpret_cast<unsigned long long*>(ws + w.ord_bsum);
    auto* units = reinterpret_cast<unsigned long long*>(ws + w.ord_units);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(ws + w.ord_cnt);
    uint32_t* wstart = reinterpret_cast<uint32_t*>(ws + w.ord_wstart);
    uint32_t* wofs = reinterpret_cast<uint32_t*>(ws + w.ord_wofs);
    const auto* xy = reinterpret_cast<const float2*>(proj.xy);
    const auto* rgbz = reinterpret_cast<const float4*>(proj.rgb_depth);
    const uint64_t cap1 = (uint64_t)V * (uint64_t)n;
    int max_tiles = 0;
    for (int v = 0; v < V; v++) max_tiles = std::max(max_tiles, L.tiles_x[v] * L.tiles_y[v]);
    const int nbx = (n + kOrdSegChunk - 1) / kOrdSegChunk;
    const int nbs = (n + kOrdScanItems - 1) / kOrdScanItems;

    if (cudaMemsetAsync(stat, 0, 16 * (size_t)V, st) != cudaSuccess) return GEVO_ERR_CUDA;
    if (n > 0) {
        // 1. each view's visible entries in (depth bits, id) order
        if (cudaMemsetAsync(seg_count, 0, 4 * (size_t)S, st) != cudaSuccess) return GEVO_ERR_CUDA;
        k_ord_stat<<<dim3((n + 1023) / 1024, V), 256, 0, st>>>(L, n, xy, proj.radius, rgbz, stat,
                                                                dk, rect);
        GEVO_CHECK_LAUNCH();
        k_ord_seg<false><<<dim3(nbx, V), 256, 0, st>>>(n, dk, stat, seg_count, nullptr, nullptr,
                                                        nullptr);
        GEVO_CHECK_LAUNCH();
        k_scan<<<1, 1024, 0, st>>>(S, cap1, seg_count, seg_start, seg_cursor, seg_order,
                                   seg_ranges, n_vis, err1);
        GEVO_CHECK_LAUNCH();
        k_ord_seg<true><<<dim3(nbx, V), 256, 0, st>>>(n, dk, stat, nullptr, seg_start, seg_cursor,
                                                       b1);
        GEVO_CHECK_LAUNCH();
        const size_t ssmem = (sizeof(uint32_t) + sizeof(uint16_t)) * 2 * kSortSmemItems;
        segsort_attributes(ssmem);
        k_segsort<<<S, kSortThreads, ssmem, st>>>(seg_order, seg_start, seg_count, n_vis, cap1,
                                                  b1, b2, dkeys, sorted);
        GEVO_CHECK_LAUNCH();
        // 2. records and the block sums of their areas
        k_ord_rec<<<dim3(nbs, V), 256, 0, st>>>(n, stat, sorted, dkeys, rect, rec, bsum);
        GEVO_CHECK_LAUNCH();
    }
    // 3. per-view totals, the unit table, the duplicate prefix and warp starts
    k_ord_bscan<<<1, 1024, 0, st>>>(V, nbs, cap, stat, bsum, units, pre);
    GEVO_CHECK_LAUNCH();
    if (n > 0) {
        k_ord_pre<<<dim3(nbs, V), 256, 0, st>>>(stat, units, rec, bsum, cap, pre, wstart);
        GEVO_CHECK_LAUNCH();
    }
    // 4. per (unit, tile) counts, their running sums over units, the tile totals
    const size_t osmem = sizeof(uint32_t) * 10 * (size_t)((max_tiles + 1) / 2);
    ord_attributes(osmem);
    const uint64_t unit_rows = cap / kOrdUnit + (uint64_t)V + 1;
    const int ugrid = (int)std::max<uint64_t>(1, std::min<uint64_t>(unit_rows, (uint64_t)sm_count() * 32));
    int cells = 0;   // the rectangle count's difference arrays: th (tw | 1) words a warp
    for (int v = 0; v < V; v++) cells = std::max(cells, L.tiles_y[v] * (L.tiles_x[v] | 1));
    const size_t rsmem = sizeof(uint32_t) * 8 * (size_t)cells;
    if (rsmem <= kOrdRectSmem) {
        count_rect_attributes(rsmem);
        k_ord_count_rect<<<ugrid, 256, rsmem, st>>>(L, max_tiles, cells, stat, units, rec, pre,
                                                     wstart, cnt, wofs);
    } else {
        k_ord_count<<<ugrid, 256, sizeof(uint32_t) * 8 * (size_t)((max_tiles + 1) / 2), st>>>(
            L, max_tiles, stat, units, rec, pre, wstart, cnt, wofs);
    }
    GEVO_CHECK_LAUNCH();
    k_ord_scan<<<dim3((max_tiles + 31) / 32, V), 256, 0, st>>>(L, max_tiles, units, cnt,
                                                                tile_count);
    GEVO_CHECK_LAUNCH();
    // 5. tile starts, ranges, D, heaviest-first order, the capacity check
    k_scan<<<1, 1024, 0, st>>>(T, cap, tile_count, tile_start, tile_cursor, tile_order, ranges,
                               d_n_dup, err, units + kUnitD);
    GEVO_CHECK_LAUNCH();
    // 6. the duplicates, emitted in order
    if (cap > 0) {
        k_ord_scatter<<<ugrid, 256, osmem, st>>>(L, max_tiles, stat, units, rec, pre, wstart, cnt,
                                                 wofs, tile_start,
                                                 reinterpret_cast<unsigned long long*>(keys), vals);
        GEVO_CHECK_LAUNCH();
    }
    return GEVO_OK;
}

}  // namespace gevo

using namespace gevo;

extern "C" int32_t gevo_bin_sort_launches(const gevo_layout* layout, int32_t n,
                                          uint64_t dup_capacity)
{
    if (!layout || !gevo::layout_valid(*layout) || n < 0) return -1;
    int mt = 0;
    for (int v = 0; v < layout->n_views; v++)
        mt = std::max(mt, layout->tiles_x[v] * layout->tiles_y[v]);
    const bool work = n > 0, room = dup_capacity > 0;
    if (mt <= kOrdMaxTiles)   // the launches of bin_sort_ordered
        return (work ? 6 : 0) + 1 + (work ? 1 : 0) + 3 + (room ? 1 : 0);
    return (work ? 1 : 0) + 1 + (work && room ? 2 : 0);
}

extern "C" gevo_status gevo_bin_sort(const gevo_layout* layout, int32_t n, const gevo_proj* proj,
                                     uint64_t dup_capacity, uint64_t* keys, uint32_t* vals,
                                     uint32_t* ranges, uint64_t* d_n_dup, void* workspace,
                                     void* stream)
{
    if (!layout || !gevo::layout_valid(*layout) || n < 0 || !proj || !proj->xy || !proj->radius ||
        !proj->rgb_depth || !ranges || !d_n_dup || !workspace || !gevo_aligned(workspace, 256) ||
        (dup_capacity > 0 && !vals) || dup_capacity > 0xffffffffull)
        return GEVO_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    const WsLayout w = ws_layout(*layout, n, dup_capacity);
    char* ws = reinterpret_cast<char*>(workspace);
    uint32_t* err = reinterpret_cast<uint32_t*>(ws + w.err);
    uint32_t* tile_count = reinterpret_cast<uint32_t*>(ws + w.tile_count);
    uint32_t* tile_cursor = reinterpret_cast<uint32_t*>(ws + w.tile_cursor);
    uint32_t* tile_order = reinterpret_cast<uint32_t*>(ws + w.tile_order);
    uint32_t* tile_start = reinterpret_cast<uint32_t*>(ws + w.tile_start);
    auto* bucket = reinterpret_cast<unsigned long long*>(ws + w.dup_tmp);
    auto* bucket2 = reinterpret_cast<unsigned long long*>(ws + w.dup_tmp2);
    uint32_t* blk_off = reinterpret_cast<uint32_t*>(ws + w.blk_off);
    const int T = layout->total_tiles;
    {
        int mt = 0;
        for (int v = 0; v < layout->n_views; v++)
            mt = std::max(mt, layout->tiles_x[v] * layout->tiles_y[v]);
        if (mt <= kOrdMaxTiles)
            return bin_sort_ordered(*layout, n, *proj, dup_capacity, keys, vals, ranges, d_n_dup,
                                    ws, w, st);
    }

    if (cudaMemsetAsync(tile_count, 0, sizeof(uint32_t) * T, st) != cudaSuccess) return GEVO_ERR_CUDA;
    const size_t total = (size_t)layout->n_views * n;
    const int sms = sm_count();
    const int grid = (int)std::min<size_t>((total + 255) / 256, (size_t)sms * 8);
    int max_tiles = 0;
    for (int v = 0; v < layout->n_views; v++)
        max_tiles = std::max(max_tiles, layout->tiles_x[v] * layout->tiles_y[v]);
    const bool smem_bins = max_tiles <= kBinMaxSmemTiles;
    const dim3 bin_grid((n + kBinChunk - 1) / kBinChunk, layout->n_views);
    const size_t bin_smem = sizeof(uint32_t) * (size_t)max_tiles;
    if (smem_bins) bin_attributes(bin_smem);
    if (total > 0) {
        if (smem_bins)
            k_count_off<<<bin_grid, kBinThreads, bin_smem, st>>>(
                *layout, n, reinterpret_cast<const float2*>(proj->xy), proj->radius, tile_count,
                blk_off);
        else
            k_count<<<std::max(grid, 1), 256, 0, st>>>(*layout, n,
                                                       reinterpret_cast<const float2*>(proj->xy),
                                                       proj->radius, tile_count);
        GEVO_CHECK_LAUNCH();
    }
    k_scan<<<1, 1024, 0, st>>>(T, dup_capacity, tile_count, tile_start, tile_cursor, tile_order,
                               ranges, d_n_dup, err);
    GEVO_CHECK_LAUNCH();
    if (total > 0 && dup_capacity > 0) {
        if (smem_bins)
            k_scatter_off<<<bin_grid, kBinThreads, bin_smem, st>>>(
                *layout, n, reinterpret_cast<const float2*>(proj->xy), proj->radius,
                reinterpret_cast<const float4*>(proj->rgb_depth), tile_start, blk_off, d_n_dup,
                dup_capacity, bucket);
        else
            k_scatter<<<std::max(grid, 1), 256, 0, st>>>(
                *layout, n, reinterpret_cast<const float2*>(proj->xy), proj->radius,
                reinterpret_cast<const float4*>(proj->rgb_depth), tile_start, tile_cursor, d_n_dup,
                dup_capacity, bucket);
        GEVO_CHECK_LAUNCH();
        const size_t smem = (sizeof(uint32_t) + sizeof(uint16_t)) * 2 * kSortSmemItems;
        segsort_attributes(smem);
        k_segsort<<<T, kSortThreads, smem, st>>>(tile_order, tile_start, tile_count, d_n_dup,
                                                 dup_capacity, bucket, bucket2,
                                                 reinterpret_cast<unsigned long long*>(keys), vals);
        GEVO_CHECK_LAUNCH();
    }
    return GEVO_OK;
}

// ---------------------------------------------------------------------------
// gevo_bin_sort_noalloc: the same sort for callers that cannot allocate device
// memory (for example plug-ins of a host application that owns every device
// allocation, or real-time loops that must not call an allocator).  Its
// scratch is the static array below; the launch sequence is that of
// gevo_bin_sort with workspace pointers into the array.
// ---------------------------------------------------------------------------
namespace gevo {
static __device__ __align__(256) unsigned char g_noalloc_scratch[GEVO_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device ordinal.  In host code the
// array's name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress with the device current.
static void* noalloc_scratch_address()
{
    static std::mutex mu;
    static void* addr[256] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
        addr[dev] = p;
    }
    return addr[dev];
}
}  // namespace gevo

extern "C" gevo_status gevo_bin_sort_noalloc(const gevo_layout* layout, int32_t n,
                                             const gevo_proj* proj, uint64_t dup_capacity,
                                             uint64_t* keys, uint32_t* vals, uint32_t* ranges,
                                             uint64_t* d_n_dup, void* stream)
{
    if (!layout || !gevo::layout_valid(*layout) || n < 0 || !proj || !proj->xy || !proj->radius ||
        !proj->rgb_depth || !ranges || !d_n_dup || (dup_capacity > 0 && !vals))
        return GEVO_ERR_INVALID;
    if (dup_capacity > GEVO_NOALLOC_MAX_DUPS || layout->total_tiles > GEVO_NOALLOC_MAX_TILES)
        return GEVO_ERR_SCRATCH_LIMIT;
    const WsLayout w = ws_layout(*layout, n, dup_capacity, false);
    if (w.core > GEVO_NOALLOC_SCRATCH_BYTES) return GEVO_ERR_SCRATCH_LIMIT;
    char* ws = reinterpret_cast<char*>(noalloc_scratch_address());
    if (!ws) return GEVO_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* err = reinterpret_cast<uint32_t*>(ws + w.err);
    uint32_t* tile_count = reinterpret_cast<uint32_t*>(ws + w.tile_count);
    uint32_t* tile_cursor = reinterpret_cast<uint32_t*>(ws + w.tile_cursor);
    uint32_t* tile_order = reinterpret_cast<uint32_t*>(ws + w.tile_order);
    uint32_t* tile_start = reinterpret_cast<uint32_t*>(ws + w.tile_start);
    auto* bucket = reinterpret_cast<unsigned long long*>(ws + w.dup_tmp);
    auto* bucket2 = reinterpret_cast<unsigned long long*>(ws + w.dup_tmp2);
    const int T = layout->total_tiles;
    // the array keeps the previous call's contents: zero the error word and the
    // tile counts; every other scratch field is fully written before it is read
    if (cudaMemsetAsync(err, 0, 64, st) != cudaSuccess) return GEVO_ERR_CUDA;
    if (cudaMemsetAsync(tile_count, 0, sizeof(uint32_t) * T, st) != cudaSuccess) return GEVO_ERR_CUDA;
    const size_t total = (size_t)layout->n_views * n;
    const int grid = (int)std::min<size_t>((total + 255) / 256, (size_t)sm_count() * 8);
    int max_tiles = 0;
    for (int v = 0; v < layout->n_views; v++)
        max_tiles = std::max(max_tiles, layout->tiles_x[v] * layout->tiles_y[v]);
    const bool smem_bins = max_tiles <= kBinMaxSmemTiles;
    const dim3 bin_grid((n + kBinChunk - 1) / kBinChunk, layout->n_views);
    const size_t bin_smem = sizeof(uint32_t) * (size_t)max_tiles;
    if (smem_bins) bin_attributes(bin_smem);
    if (total > 0) {
        if (smem_bins)
            k_count_smem<<<bin_grid, kBinThreads, bin_smem, st>>>(
                *layout, n, reinterpret_cast<const float2*>(proj->xy), proj->radius, tile_count);
        else
            k_count<<<std::max(grid, 1), 256, 0, st>>>(*layout, n,
                                                       reinterpret_cast<const float2*>(proj->xy),
                                                       proj->radius, tile_count);
        GEVO_CHECK_LAUNCH();
    }
    k_scan<<<1, 1024, 0, st>>>(T, dup_capacity, tile_count, tile_start, tile_cursor, tile_order,
                               ranges, d_n_dup, err);
    GEVO_CHECK_LAUNCH();
    if (total > 0 && dup_capacity > 0) {
        if (smem_bins)
            k_scatter_smem<<<bin_grid, kBinThreads, bin_smem, st>>>(
                *layout, n, reinterpret_cast<const float2*>(proj->xy), proj->radius,
                reinterpret_cast<const float4*>(proj->rgb_depth), tile_start, tile_cursor,
                d_n_dup, dup_capacity, bucket);
        else
            k_scatter<<<std::max(grid, 1), 256, 0, st>>>(
                *layout, n, reinterpret_cast<const float2*>(proj->xy), proj->radius,
                reinterpret_cast<const float4*>(proj->rgb_depth), tile_start, tile_cursor, d_n_dup,
                dup_capacity, bucket);
        GEVO_CHECK_LAUNCH();
        const size_t smem = (sizeof(uint32_t) + sizeof(uint16_t)) * 2 * kSortSmemItems;
        segsort_attributes(smem);
        k_segsort<<<T, kSortThreads, smem, st>>>(tile_order, tile_start, tile_count, d_n_dup,
                                                 dup_capacity, bucket, bucket2,
                                                 reinterpret_cast<unsigned long long*>(keys), vals);
        GEVO_CHECK_LAUNCH();
    }
    return GEVO_OK;
}
