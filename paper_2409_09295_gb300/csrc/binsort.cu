// Stages a2-a4 of the splatting renderer GEVO uses (Section I "GS"): emit one
// (tile, depth) key per (Gaussian, tile) pair, sort the keys bit-exactly and
// find each tile's range.
//
// GB300 design (instead of one 64-bit radix sort over all duplicates):
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
// taken with one shared-memory atomic per distinct bucket per warp step.
__global__ void __launch_bounds__(1024)
k_scan(int T, uint64_t cap, const uint32_t* __restrict__ tile_count, uint32_t* __restrict__ tile_start,
       uint32_t* __restrict__ tile_cursor, uint32_t* __restrict__ tile_order,
       uint32_t* __restrict__ ranges, uint64_t* __restrict__ d_n_dup, uint32_t* err)
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
    if (tid < 34) s_bucket[tid] = 0;
    unsigned long long sum = 0;
    for (int t = w0 + lane; t < w1; t += 32) sum += tile_count[t];
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
    const unsigned long long D = s_total;
    const bool overflow = D > cap;
    unsigned long long carry = s_warp[warp];
    for (int b0 = w0; b0 < w1; b0 += 32) {
        const int t = b0 + lane;
        const bool valid = t < w1;
        const uint32_t c = valid ? tile_count[t] : 0u;
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
    }
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
    for (int b0 = w0; b0 < w1; b0 += 32) {
        const int t = b0 + lane;
        const bool valid = t < w1;
        const uint32_t c = valid ? tile_count[t] : 0u;
        const int b = valid ? (c == 0 ? 0 : 32 - __clz(c)) : 34;
        const uint32_t peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (valid && lane == leader) base = atomicAdd(&s_bucket_base[b], __popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (valid) tile_order[base + __popc(peers & lt)] = (uint32_t)t;
    }
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
            keys_out[s0 + i] = th | ka[i];
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
        keys_out[s0 + i] = th | (k >> 32);
        vals_out[s0 + i] = (uint32_t)k;
    }
}

// Dynamic shared-memory limits of the binning and sort kernels, raised once per
// device (the attribute belongs to the device's context) and only upwards.
// Host threads may sort concurrently, so the record sits behind a mutex.
static std::mutex g_attr_mu;

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

}  // namespace gevo

using namespace gevo;

extern "C" gevo_status gevo_bin_sort(const gevo_layout* layout, int32_t n, const gevo_proj* proj,
                                     uint64_t dup_capacity, uint64_t* keys, uint32_t* vals,
                                     uint32_t* ranges, uint64_t* d_n_dup, void* workspace,
                                     void* stream)
{
    if (!layout || !gevo::layout_valid(*layout) || n < 0 || !proj || !proj->xy || !proj->radius ||
        !proj->rgb_depth || !ranges || !d_n_dup || !workspace || !gevo_aligned(workspace, 256) ||
        (dup_capacity > 0 && (!keys || !vals)) || dup_capacity > 0xffffffffull)
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
        !proj->rgb_depth || !ranges || !d_n_dup || (dup_capacity > 0 && (!keys || !vals)))
        return GEVO_ERR_INVALID;
    if (dup_capacity > GEVO_NOALLOC_MAX_DUPS || layout->total_tiles > GEVO_NOALLOC_MAX_TILES)
        return GEVO_ERR_SCRATCH_LIMIT;
    const WsLayout w = ws_layout(*layout, n, dup_capacity);
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
