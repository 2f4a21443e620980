// Host-side set-up, workspace sizing and status calls of the C ABI.
#include <string.h>

#include "gevo_internal.cuh"

namespace gevo {

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

WsLayout ws_layout(const gevo_layout& L, int32_t n, uint64_t cap, bool pbwd)
{
    WsLayout w;
    size_t T = (size_t)L.total_tiles;
    size_t o = 0;
    w.err = o;          o = align256(o + 64);
    w.tile_count = o;   o = align256(o + 4 * T);
    w.tile_cursor = o;  o = align256(o + 4 * T);
    w.tile_order = o;   o = align256(o + 4 * T);
    w.tile_start = o;   o = align256(o + 4 * (T + 1));
    const size_t nn = pbwd ? (size_t)(n > 0 ? n : 0) : 0;
    w.pb_perm = o;      o = align256(o + 4 * nn);
    w.pb_mask = o;      o = align256(o + 8 * nn);
    w.dup_tmp = o;      o = align256(o + 8 * (size_t)cap);
    w.dup_tmp2 = o;     o = align256(o + 8 * (size_t)cap);
    w.dxi_acc = o;      o = align256(o + 4 * 6 * (size_t)GEVO_MAX_VIEWS);
    w.core = o;
    const size_t nbx = ((size_t)(n > 0 ? n : 0) + kBinChunk - 1) / kBinChunk;
    w.blk_off = o;      o = align256(o + 4 * nbx * T);
    const size_t V = (size_t)L.n_views, VN = V * (size_t)(n > 0 ? n : 0);
    const size_t S = V * kDepthBins;
    w.ord_stat = o;     o = align256(o + 16 * V);
    w.ord_seg = o;      o = align256(o + 4 * (5 * S + 1) + 4 * S);
    w.ord_total = o;    o = align256(o + 16);
    w.ord_b1 = o;       o = align256(o + 16 * VN);   // later the uint4 records
    w.ord_b2 = o;       o = align256(o + 8 * VN);
    w.ord_vals = o;     o = align256(o + 4 * VN);
    w.ord_dkeys = o;    o = align256(o + 8 * VN);
    w.ord_pre = o;      o = align256(o + 8 * (VN + V + 1));
    w.ord_bsum = o;     o = align256(o + 8 * V * ((size_t)(n > 0 ? n : 0) / kOrdScanItems + 1));
    w.ord_units = o;    o = align256(o + 8 * 4 * (GEVO_MAX_VIEWS + 1));
    size_t max_tiles = 0;
    for (int v = 0; v < L.n_views; v++)
        max_tiles = std::max(max_tiles, (size_t)L.tiles_x[v] * L.tiles_y[v]);
    const size_t unit_rows = (size_t)(cap / kOrdUnit) + V + 1;
    w.ord_cnt = o;      o = align256(o + 4 * unit_rows * max_tiles);
    w.ord_wstart = o;   o = align256(o + 4 * 8 * unit_rows);
    w.ord_wofs = o;     o = align256(o + 4 * 8 * ((max_tiles + 1) / 2) * unit_rows);
    w.total = o;
    return w;
}

bool layout_valid(const gevo_layout& L)
{
    if (L.n_views < 1 || L.n_views > GEVO_MAX_VIEWS) return false;
    int64_t tiles = 0, pix = 0;
    for (int v = 0; v < L.n_views; v++) {
        const int32_t w = L.width[v], h = L.height[v];
        if (w <= 0 || h <= 0 || w > 65536 || h > 65536) return false;
        if (L.tiles_x[v] != (w + GEVO_TILE - 1) / GEVO_TILE ||
            L.tiles_y[v] != (h + GEVO_TILE - 1) / GEVO_TILE)
            return false;
        if (L.tile_base[v] != tiles || L.pix_base[v] != pix) return false;
        tiles += (int64_t)L.tiles_x[v] * L.tiles_y[v];
        pix += (int64_t)w * h;
        if (tiles > (1 << 30)) return false;
    }
    return L.tile_base[L.n_views] == tiles && L.pix_base[L.n_views] == pix &&
           L.total_tiles == tiles && L.total_pixels == pix;
}

int sm_count()
{
    static int cached = 0;
    if (!cached) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached = v > 0 ? v : 1;
    }
    return cached;
}

int device_max_smem_optin()
{
    static int cached = 0;
    if (!cached) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cached = v > 0 ? v : 48 * 1024;
    }
    return cached;
}

}  // namespace gevo

extern "C" {

gevo_status gevo_layout_init(gevo_layout* layout, int32_t n_views, const int32_t* width,
                             const int32_t* height)
{
    if (!layout || !width || !height || n_views < 1 || n_views > GEVO_MAX_VIEWS)
        return GEVO_ERR_INVALID;
    memset(layout, 0, sizeof(*layout));
    layout->n_views = n_views;
    int64_t tiles = 0, pix = 0;
    for (int v = 0; v < n_views; v++) {
        if (width[v] <= 0 || height[v] <= 0 || width[v] > 65536 || height[v] > 65536)
            return GEVO_ERR_INVALID;
        layout->width[v] = width[v];
        layout->height[v] = height[v];
        layout->tiles_x[v] = (width[v] + GEVO_TILE - 1) / GEVO_TILE;
        layout->tiles_y[v] = (height[v] + GEVO_TILE - 1) / GEVO_TILE;
        layout->tile_base[v] = (int32_t)tiles;
        layout->pix_base[v] = pix;
        tiles += (int64_t)layout->tiles_x[v] * layout->tiles_y[v];
        pix += (int64_t)width[v] * height[v];
        if (tiles > (1 << 30)) return GEVO_ERR_INVALID;
    }
    layout->tile_base[n_views] = (int32_t)tiles;
    layout->pix_base[n_views] = pix;
    layout->total_tiles = (int32_t)tiles;
    layout->total_pixels = pix;
    return GEVO_OK;
}

size_t gevo_workspace_bytes(const gevo_layout* layout, int32_t n, uint64_t dup_capacity)
{
    if (!layout || !gevo::layout_valid(*layout)) return 0;
    return gevo::ws_layout(*layout, n, dup_capacity).total;
}

gevo_status gevo_last_error(void* workspace, void* stream)
{
    if (!workspace) return GEVO_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t word = 0;
    if (cudaMemcpyAsync(&word, workspace, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return GEVO_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GEVO_ERR_CUDA;
    if (word) {
        if (cudaMemsetAsync(workspace, 0, 4, s) != cudaSuccess) return GEVO_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return GEVO_ERR_CUDA;
    }
    if (word & gevo::kErrCapacity) return GEVO_ERR_CAPACITY;
    if (word & gevo::kErrNonFinite) return GEVO_ERR_NONFINITE;
    if (word & gevo::kErrTimeout) return GEVO_ERR_TIMEOUT;
    return GEVO_OK;
}

const char* gevo_status_str(gevo_status s)
{
    switch (s) {
    case GEVO_OK: return "ok";
    case GEVO_ERR_INVALID: return "invalid argument";
    case GEVO_ERR_CAPACITY: return "duplicate capacity exceeded";
    case GEVO_ERR_CUDA: return "CUDA error";
    case GEVO_ERR_TIMEOUT: return "device wait timed out";
    case GEVO_ERR_NONFINITE: return "non-finite value culled";
    case GEVO_ERR_SCRATCH_LIMIT: return "size exceeds the fixed no-allocation scratch";
    }
    return "unknown status";
}

int32_t gevo_version(void) { return GEVO_VERSION; }

}  // extern "C"
