/*
 * gevo.h -- C ABI of the GB300 (sm_103a) differentiable Gaussian-splatting
 * rasterizer behind GEVO's map optimisation, tracking and rendered keyframes.
 *
 * The paper (GEVO, arXiv 2409.09295) renders with the 3DGS rasterizer it cites
 * in Section I ("GS") and optimises the map and the camera pose T_k through it
 * (Section III-B, Eq. 2 local stage and Eq. 3 global stage); Eq. 6 (E_pc)
 * compares renders R(M'_t, T_kl) of four past keyframes against stop-gradient
 * renders of the previous map, which is what the batched multi-view calls are
 * for.  Every operation below is one stage of that renderer:
 *
 *   gevo_project      projection: 3-D covariance, EWA 2-D conic, depth, radius,
 *                     colour, tiles touched                          (stage a1)
 *   gevo_bin_sort     (tile, depth) keys, bit-exact sort, tile ranges (a2-a4)
 *   gevo_render_fwd   front-to-back alpha blending: RGB, depth, final T (a5)
 *   gevo_render_bwd   reverse walk: gradients of the 2-D records     (a6)
 *   gevo_project_bwd  gradients of the Gaussian parameters and of the camera
 *                     pose as an se(3) twist                          (a7)
 *   gevo_loss_l1      L1 photometric (+ depth) loss and its gradient  (a8)
 *
 * Conventions shared by every call
 *  - Device pointers are caller-owned device memory (for example torch
 *    tensors); the library never allocates, frees or synchronises inside these
 *    calls, and launches only on the given stream.  Host pointers are read
 *    before the call returns.
 *  - float arrays are IEEE binary32, row-major, tightly packed, 16-byte
 *    aligned unless stated otherwise.
 *  - A call returns GEVO_ERR_INVALID without launching anything on host-
 *    detectable misuse (NULL where a pointer is required, negative sizes,
 *    sh_degree outside 0..3, a layout with no views, misaligned pointers).
 *    GEVO_ERR_CUDA means a launch failed (cudaGetLastError after the launch).
 *  - Conditions only the device can see (duplicate count above capacity)
 *    set a sticky error word in the workspace; outputs that depend on them are
 *    then defined as stated per call.  gevo_last_error() reads and clears it.
 *  - No kernel waits on another kernel or block.  The only device-side wait is
 *    the tensor-core GEMM's wait for its own MMAs (bounded: it gives up after
 *    about a second, records GEVO_ERR_TIMEOUT and frees its tensor memory).
 *
 * Numerical constants of the formulation (3DGS defaults; the paper gives none):
 *   near plane z > 0.2, 2-D dilation 0.3 px^2, Jacobian guard band 1.3x the
 *   half field of view, alpha clamp 0.99, skip alpha < 1/255, stop before
 *   T < 1e-4, 16 x 16 pixel tiles, radius ceil(3 sqrt(lambda_max)).
 */
#ifndef GEVO_H
#define GEVO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GEVO_VERSION 1
#define GEVO_MAX_VIEWS 64
#define GEVO_TILE 16

typedef enum {
    GEVO_OK = 0,
    GEVO_ERR_INVALID = 1,   /* bad argument, nothing launched                    */
    GEVO_ERR_CAPACITY = 2,  /* device: duplicate count exceeded dup_capacity     */
    GEVO_ERR_CUDA = 3,      /* a CUDA runtime call or launch failed              */
    GEVO_ERR_TIMEOUT = 4,   /* device: a bounded tensor-core completion wait gave up */
    GEVO_ERR_NONFINITE = 5, /* device: a non-finite projected value was culled   */
    GEVO_ERR_SCRATCH_LIMIT = 6 /* sizes exceed gevo_bin_sort_noalloc's fixed scratch */
} gevo_status;

/* Pinhole camera of one view, world -> camera: p_c = R * p_w + t, camera x
 * right, y down, z forward.  Pixel i is sampled at coordinate i, so the image
 * mean of a point is (fx X/Z + cx - 0.5, fy Y/Z + cy - 0.5).  An array of these
 * lives in DEVICE memory (16 floats = 64 bytes each) so that poses can change
 * between replays of a captured graph. */
typedef struct {
    float R[9];   /* row-major */
    float t[3];
    float fx, fy, cx, cy;
} gevo_camera;

/* Image geometry of a batch of views (HOST memory, fixed for a captured graph).
 * Tiles are numbered view-major: global tile = tile_base[v] + ty * tiles_x[v]
 * + tx.  Per-pixel outputs are view-major planes: view v's pixel (x, y) is
 * element pix_base[v] + y * width[v] + x of a [total_pixels] plane; an RGB
 * output holds three such planes per view, R then G then B, starting at
 * 3 * pix_base[v]. */
typedef struct {
    int32_t n_views;
    int32_t total_tiles;
    int64_t total_pixels;
    int32_t width[GEVO_MAX_VIEWS];
    int32_t height[GEVO_MAX_VIEWS];
    int32_t tiles_x[GEVO_MAX_VIEWS];
    int32_t tiles_y[GEVO_MAX_VIEWS];
    int32_t tile_base[GEVO_MAX_VIEWS + 1];
    int64_t pix_base[GEVO_MAX_VIEWS + 1];
} gevo_layout;

/* Gaussian parameters, DEVICE memory, structure of arrays over n Gaussians.
 * Exactly one of sh / rgb is non-NULL.  rgb colours are used as given; SH
 * colours are max(0, sum_k Y_k(d) sh[k] + 0.5) with d the unit direction from
 * the camera centre to the mean and Y the real SH basis up to sh_degree. */
typedef struct {
    const float* means;      /* [n][3] world position                            */
    const float* scales;     /* [n][3] activated (positive) standard deviations  */
    const float* quats;      /* [n][4] rotation (w, x, y, z), any non-zero norm  */
    const float* opacities;  /* [n]    activated opacity in (0, 1)               */
    const float* sh;         /* [n][(sh_degree+1)^2][3] or NULL                  */
    const float* rgb;        /* [n][3] or NULL                                   */
    int32_t n;
    int32_t sh_degree;       /* 0..3, used with sh                               */
} gevo_gaussians;

/* Gradients w.r.t. gevo_gaussians, same shapes, DEVICE memory, written (not
 * accumulated) by gevo_project_bwd.  sh must be non-NULL iff the parameters
 * have sh, rgb iff they have rgb. */
typedef struct {
    float* means;
    float* scales;
    float* quats;
    float* opacities;
    float* sh;
    float* rgb;
} gevo_gaussian_grads;

/* Per (view, Gaussian) projection records, DEVICE memory, entry v * n + g. */
typedef struct {
    float* xy;             /* [V*n][2] image-space mean                          */
    float* conic_opacity;  /* [V*n][4] inverse 2-D covariance (a, b, c), opacity */
    float* rgb_depth;      /* [V*n][4] colour, camera-frame depth                 */
    int32_t* radius;       /* [V*n]    pixel radius, 0 = culled                   */
    uint32_t* tiles_touched; /* [V*n]  tiles in the rectangle, 0 if culled        */
} gevo_proj;

/* Gradients of a scalar loss w.r.t. the records, DEVICE memory, entry v*n+g. */
typedef struct {
    float* xy;             /* [V*n][2]                                           */
    float* conic_opacity;  /* [V*n][4] d/da, d/db, d/dc (as in the power), d/do  */
    float* rgb_depth;      /* [V*n][4] d/dr, d/dg, d/db, d/ddepth                 */
} gevo_grad2d;

/* Launch shape for the per-tile kernels (chosen by the autotuner).
 * threads_per_tile in {32, 64, 128, 256}: each thread owns 256 / threads pixels of
 * its 16 x 16 tile.  persistent != 0: one grid of blocks_per_sm * SMs blocks
 * pulls (view, tile) work items heaviest first from a device counter; 0: one
 * block per tile.  NULL = {256, 0, 0}. */
typedef struct {
    int32_t threads_per_tile;
    int32_t persistent;
    int32_t blocks_per_sm;   /* 0 = as many as fit */
} gevo_tuning;

/* ---------------------------------------------------------------------- */
/* Set-up (host only; no device work)                                      */
/* ---------------------------------------------------------------------- */

/* Fills *layout for n_views views of the given pixel sizes (host arrays).
 * Returns GEVO_ERR_INVALID if n_views is not in 1..GEVO_MAX_VIEWS or a size is
 * not positive or the totals overflow 32-bit tile / 31-bit list indices. */
gevo_status gevo_layout_init(gevo_layout* layout, int32_t n_views, const int32_t* width,
                             const int32_t* height);

/* Bytes of device workspace the calls below need for n Gaussians, this layout
 * and a duplicate capacity of dup_capacity (Gaussian, tile) pairs.  The
 * workspace must be 256-byte aligned, is owned by the caller, and carries
 * state between calls of one pipeline (tile counts, the heaviest-first tile
 * order and the sticky error word): use one workspace per pipeline and do not
 * run two pipelines on it concurrently.  It must be zero-filled once before
 * its first use (cudaMemset). */
size_t gevo_workspace_bytes(const gevo_layout* layout, int32_t n, uint64_t dup_capacity);

/* ---------------------------------------------------------------------- */
/* Stage a1: projection (Section I "GS"; Section III-B Eq. 2/3 render R(M,T)) */
/* ---------------------------------------------------------------------- */

/* For every view v and Gaussian g: p = R mu + t; cull if p.z <= 0.2;
 * Sigma3 = Rq diag(s)^2 Rq^T; J = EWA Jacobian of the pinhole map at p (x/z and
 * y/z clamped to 1.3x the half field of view); Sigma2 = J R Sigma3 R^T J^T +
 * 0.3 I; cull if det <= 0; conic = Sigma2^-1; radius = ceil(3 sqrt(lambda_max))
 * with lambda_max = mid + sqrt(max(0.1, mid^2 - det)); tile rectangle (see
 * gevo_bin_sort); cull if it is empty; colour from rgb or SH.  Culled entries
 * get radius = 0 and tiles_touched = 0 (other fields undefined).
 * Each Gaussian is read once for all views.  cams: DEVICE array [n_views]. */
gevo_status gevo_project(const gevo_layout* layout, const gevo_gaussians* g,
                         const gevo_camera* cams, gevo_proj* out, void* workspace,
                         void* stream);

/* Parts of gevo_project_part and gevo_project_bwd_part. */
#define GEVO_PART_ALL 0       /* the whole call, as gevo_project / gevo_project_bwd */
#define GEVO_PART_GEOMETRY 1  /* everything but the colour                          */
#define GEVO_PART_COLOUR 2    /* the colour only                                    */

/* Range unit of gevo_project_bwd_part (see there). */
#define GEVO_PART_RANGE 1024

/* gevo_project in two parts and over Gaussian ranges, so that a caller whose
 * parameters arrive in pieces (host-to-device copies) can project each piece
 * as it lands, and start the sort while the colour parameters (the SH
 * coefficients, most of the bytes) are still in flight: the sort reads no
 * colour.  Only Gaussians g_begin <= g < g_end (0 <= g_begin <= g_end <= n)
 * are projected, for every view; the records of the others are untouched.
 * GEVO_PART_GEOMETRY writes xy, conic_opacity, radius, tiles_touched and the
 * depth (w) of rgb_depth, with rgb_depth x, y, z = 0; it reads means, scales,
 * quats and opacities only (sh / rgb may still be in flight, but one of them
 * must be non-NULL).  GEVO_PART_COLOUR, after it on the stream (or after an
 * event recorded after it), writes x, y, z of rgb_depth for every entry with
 * radius > 0 and nothing else -- so gevo_bin_sort, which reads only w, may run
 * concurrently.  The parts, over any ranges covering the map, give bit for
 * bit what gevo_project gives.  part outside 0..2 or a bad range:
 * GEVO_ERR_INVALID. */
gevo_status gevo_project_part(const gevo_layout* layout, const gevo_gaussians* g,
                              const gevo_camera* cams, gevo_proj* out, int32_t part,
                              int32_t g_begin, int32_t g_end, void* workspace, void* stream);

/* gevo_project_part (part GEVO_PART_ALL or GEVO_PART_GEOMETRY) that also zeroes,
 * for every entry it finds visible (radius > 0), that entry's rows of *grad2d
 * -- the rows gevo_render_bwd then accumulates into and gevo_project_bwd reads
 * -- in the same pass, so that a step needs no separate gevo_grad2d_zero.
 * Rows of culled entries are left as they are.  GEVO_PART_COLOUR, a NULL or
 * misaligned grad2d: GEVO_ERR_INVALID. */
gevo_status gevo_project_zero(const gevo_layout* layout, const gevo_gaussians* g,
                              const gevo_camera* cams, gevo_proj* out, gevo_grad2d* grad2d,
                              int32_t part, int32_t g_begin, int32_t g_end, void* workspace,
                              void* stream);

/* ---------------------------------------------------------------------- */
/* Stages a2-a4: keys, bit-exact sort, tile ranges                          */
/* ---------------------------------------------------------------------- */

/* Tile rectangle of entry (v, g), in binary32: per axis
 * [floor((m - r) / 16), floor((m + r + 15) / 16)) clamped to the tile grid.
 * Every tile t of it yields one duplicate with key = (tile_base[v] + t) << 32 |
 * bit pattern of the binary32 depth, value = g.  Output: keys / vals sorted by
 * key, equal keys by value, of length D = sum tiles_touched; ranges[2 t],
 * ranges[2 t + 1] = [start, end) of global tile t in that order, (0, 0) for an
 * empty tile.  *d_n_dup (DEVICE uint64) receives D.
 * If D > dup_capacity: the error word gets GEVO_ERR_CAPACITY, *d_n_dup still
 * receives the true D, every range is (0, 0) and keys / vals are undefined.
 * keys: [dup_capacity] uint64 or NULL, vals: [dup_capacity] uint32, ranges:
 * [total_tiles][2] uint32 (DEVICE).  With keys NULL only vals is written: the
 * key of position i is implied (its tile is the range holding i, its depth bits
 * those of entry (v, vals[i])), and the blending and backward stages read only
 * vals and ranges. */
gevo_status gevo_bin_sort(const gevo_layout* layout, int32_t n, const gevo_proj* proj,
                          uint64_t dup_capacity, uint64_t* keys, uint32_t* vals,
                          uint32_t* ranges, uint64_t* d_n_dup, void* workspace, void* stream);

/* Number of kernels gevo_bin_sort launches for these sizes (for sizing CUDA
 * graphs and accounting launches): the views' largest tile count picks the
 * implementation -- up to 8192 tiles per view, each view's visible entries are
 * sorted by depth once and the duplicates emitted in order (12 kernels); above
 * that, duplicates are bucketed by tile and each bucket sorted (4 kernels).
 * Fewer when n or dup_capacity is 0.  -1 for an invalid layout or n < 0. */
int32_t gevo_bin_sort_launches(const gevo_layout* layout, int32_t n, uint64_t dup_capacity);

/* Same operation and outputs as gevo_bin_sort (keys may be NULL there too),
 * for callers that cannot allocate device memory: no workspace argument, and the call itself allocates
 * nothing (no cudaMalloc, no allocating library routine).  Such callers include
 * plug-ins hosted by a renderer or an inference server that owns every device
 * allocation, and real-time loops where an allocator call, with its latency
 * and implicit synchronisation, is not allowed.  The paper has no counterpart:
 * this is a deployment variant of stages a2-a4.
 * Scratch: a file-scope static device array of GEVO_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library holds until the process exits.  It caps
 * dup_capacity at GEVO_NOALLOC_MAX_DUPS and the layout at GEVO_NOALLOC_MAX_TILES
 * tiles; larger sizes return GEVO_ERR_SCRATCH_LIMIT without launching.
 * The array is reserved in device memory when the CUDA runtime loads this
 * library's kernels on a device.  Under lazy module loading (the default of
 * CUDA 12 and later) that can be the first call of this function on that
 * device, so that first call may fail with GEVO_ERR_CUDA when the device has no
 * memory left.  A caller whose allocation-free region must not reserve
 * anything makes one call outside it first, for example with dup_capacity 0
 * (which counts the duplicates only).
 * The first call on a device also looks up the array's device address (once
 * per device, with that device current) and keeps it for the process; make
 * that first call before any stream capture.  cudaDeviceReset on that device
 * unloads the array, after which this function must not be called again in
 * the process.  Every call shares the one array and clears the parts that must
 * start at zero, so calls whose GPU work overlaps (other streams, other host
 * threads) race and must be serialised by the caller.  A duplicate count above
 * dup_capacity is reported only through *d_n_dup > dup_capacity (the ranges are
 * then all (0, 0)); there is no workspace for gevo_last_error to read. */
#define GEVO_NOALLOC_MAX_DUPS (1ull << 21)
#define GEVO_NOALLOC_MAX_TILES (1 << 16)
#define GEVO_NOALLOC_SCRATCH_BYTES ((size_t)35 << 20)
gevo_status gevo_bin_sort_noalloc(const gevo_layout* layout, int32_t n, const gevo_proj* proj,
                                  uint64_t dup_capacity, uint64_t* keys, uint32_t* vals,
                                  uint32_t* ranges, uint64_t* d_n_dup, void* stream);

/* ---------------------------------------------------------------------- */
/* Stage a5: front-to-back blending (R(M, T) of Eq. 2, 3 and 6)             */
/* ---------------------------------------------------------------------- */

/* Per pixel (x, y) of view v, walk its tile's list in order: d = xy - (x, y);
 * power = -1/2 (a dx^2 + c dy^2) - b dx dy; skip if power > 0;
 * alpha = min(0.99, o exp(power)); skip if alpha < 1/255; stop (without
 * blending) if T (1 - alpha) < 1e-4; else C += alpha T c, D += alpha T z,
 * T *= 1 - alpha.  Finally C += T bg.
 * Outputs (DEVICE planes, see gevo_layout): rgb [3 * total_pixels], depth,
 * T_final [total_pixels] float; n_contrib [total_pixels] uint32 = 1 + list
 * position of the last blended entry (0 if none); n_eval (nullable) = list
 * entries examined including skips and the stopping entry.
 * bg: HOST float[3].  workspace: the one gevo_bin_sort used (persistent mode
 * reads its tile order). */
gevo_status gevo_render_fwd(const gevo_layout* layout, int32_t n, const gevo_proj* proj,
                            const uint32_t* vals, const uint32_t* ranges, const float* bg,
                            float* rgb, float* depth, float* T_final, uint32_t* n_contrib,
                            uint32_t* n_eval, const gevo_tuning* tuning, void* workspace,
                            void* stream);

/* gevo_render_fwd with n_eval and, in n_blend (DEVICE uint32[total_pixels],
 * written), the number of entries each pixel blends: the counts the work of
 * the blend and of its reverse walk is measured in. */
gevo_status gevo_render_fwd_counts(const gevo_layout* layout, int32_t n, const gevo_proj* proj,
                                   const uint32_t* vals, const uint32_t* ranges, const float* bg,
                                   float* rgb, float* depth, float* T_final, uint32_t* n_contrib,
                                   uint32_t* n_eval, uint32_t* n_blend, const gevo_tuning* tuning,
                                   void* workspace, void* stream);

/* ---------------------------------------------------------------------- */
/* Stage a6: reverse walk                                                   */
/* ---------------------------------------------------------------------- */

/* Gradients of a scalar loss L w.r.t. every record that gevo_render_fwd
 * blended, given dL/drgb [3 * total_pixels], dL/ddepth [total_pixels] and
 * dL/dT_final [total_pixels] (dL_ddepth and dL_dT nullable = 0).  Walks each
 * pixel's list from n_contrib - 1 down to 0, recomputing alpha and recovering
 * T by T / (1 - alpha) from T_final; per-Gaussian sums are warp-reduced and
 * added with FP32 atomics (summation order is not deterministic).
 * out: accumulated (+=) -- clear it first with gevo_grad2d_zero; rows of culled
 * entries are never touched.  Launches exactly one kernel. */
gevo_status gevo_render_bwd(const gevo_layout* layout, int32_t n, const gevo_proj* proj,
                            const uint32_t* vals, const uint32_t* ranges, const float* bg,
                            const float* T_final, const uint32_t* n_contrib,
                            const float* dL_drgb, const float* dL_ddepth, const float* dL_dT,
                            gevo_grad2d* out, const gevo_tuning* tuning, void* workspace,
                            void* stream);

/* Zeroes the rows of *out that belong to entries with radius > 0 (the only
 * rows gevo_render_bwd accumulates into and gevo_project_bwd reads). */
gevo_status gevo_grad2d_zero(const gevo_layout* layout, int32_t n, const gevo_proj* proj,
                             gevo_grad2d* out, void* stream);

/* ---------------------------------------------------------------------- */
/* Stage a7: projection derivative incl. the se(3) pose gradient            */
/* ---------------------------------------------------------------------- */

/* Chains dL/d(records) back to the Gaussian parameters (summed over views,
 * written to *out) and, if dxi != NULL, to a left se(3) perturbation
 * xi = (rho, phi) of each view's world->camera transform, T <- Exp(xi) T at
 * xi = 0 (dxi: DEVICE float [n_views][6], written).  The pose enters through
 * the camera-frame mean, through R in Sigma2 and through the camera centre in
 * the SH view direction.  Clamped SH channels and clamped Jacobian directions
 * get zero gradient. */
gevo_status gevo_project_bwd(const gevo_layout* layout, const gevo_gaussians* g,
                             const gevo_camera* cams, const gevo_proj* proj,
                             const gevo_grad2d* grad2d, gevo_gaussian_grads* out, float* dxi,
                             void* workspace, void* stream);

/* gevo_project_bwd in two parts and over Gaussian ranges, so that a caller
 * copying the gradients to the host can start with the SH gradients (most of
 * the bytes) of the first range while later ranges and the geometry part
 * still run.  Ranges [g_begin, g_end) start and end at multiples of
 * GEVO_PART_RANGE (or end at n).  GEVO_PART_COLOUR, for SH colours, writes
 * out->sh and the view-direction share of out->means for the range and adds
 * the camera centre's share to dxi; on the range starting at 0 it also zeroes
 * dxi and stores in the workspace the order in which both parts walk the
 * Gaussians, so it runs first.  GEVO_PART_GEOMETRY, on ranges whose colour
 * part has run (same stream, same workspace), writes out->scales, quats,
 * opacities and rgb, adds the rest of out->means (writes it for rgb colours)
 * and adds to dxi.  The SH gradients of a range are final once its colour part
 * has run.  Over ranges covering the map the parts give what gevo_project_bwd
 * gives (dxi sums in another order; every other output bit for bit).  part
 * outside 0..2 or a bad range: GEVO_ERR_INVALID. */
gevo_status gevo_project_bwd_part(const gevo_layout* layout, const gevo_gaussians* g,
                                  const gevo_camera* cams, const gevo_proj* proj,
                                  const gevo_grad2d* grad2d, gevo_gaussian_grads* out,
                                  float* dxi, int32_t part, int32_t g_begin, int32_t g_end,
                                  void* workspace, void* stream);

/* ---------------------------------------------------------------------- */
/* Stage a8: L1 loss with stop-gradient targets (E_pho of Eq. 2, E_pc of Eq. 6) */
/* ---------------------------------------------------------------------- */

/* L = sum_v [ mean_px,ch |rgb - target_rgb| + lambda_depth mean_px |depth -
 * target_depth| ] over the views of the layout; dL_drgb = sign(.) / (3 P_v),
 * dL_ddepth = lambda_depth sign(.) / P_v, sign(0) = 0.  depth / target_depth /
 * dL_ddepth may be NULL when lambda_depth == 0 (dL_ddepth is then untouched).
 * loss: DEVICE float[n_views] per-view terms (written).  All DEVICE. */
gevo_status gevo_loss_l1(const gevo_layout* layout, const float* rgb, const float* target_rgb,
                         const float* depth, const float* target_depth, float lambda_depth,
                         float* dL_drgb, float* dL_ddepth, float* loss, void* workspace,
                         void* stream);

/* ---------------------------------------------------------------------- */
/* Active set of the global stage (Section III-B2, Eq. 5)                   */
/* ---------------------------------------------------------------------- */
/* The global stage optimises only an active subset A_t = M~_t u E_t of the
 * map: the newly inserted Gaussians and E_t = {g : max_k E_k(g) > eps} over
 * the window's keyframes k, with the per-Gaussian rendering error
 *     E_k(g) = sum_u w(g, u) e_k(u),
 * w(g, u) = alpha T the blending weight of g at pixel u and e_k(u) the
 * per-pixel error |R - C_k|(u), read as the mean over the three colour
 * channels of the absolute difference.  Section IV-C states the active set
 * holds under 15% of the map and that a rasterizer specialised to it would cut
 * latency; these four calls are that path. */

/* gevo_loss_l1 plus the per-pixel error: pix_err[pix_base[v] + p] =
 * (|dr| + |dg| + |db|) / 3 of rgb - target_rgb (DEVICE float[total_pixels],
 * written).  Same loss and gradients as gevo_loss_l1. */
gevo_status gevo_loss_l1_err(const gevo_layout* layout, const float* rgb,
                             const float* target_rgb, const float* depth,
                             const float* target_depth, float lambda_depth, float* dL_drgb,
                             float* dL_ddepth, float* loss, float* pix_err, void* workspace,
                             void* stream);

/* Where the reverse walk of an active-set backward starts, per pixel (DEVICE,
 * planes of total_pixels, written by gevo_render_fwd_active):
 *   last[p]  1 + list position of the last blended entry of an active
 *            Gaussian, 0 if the pixel blends none;
 *   T[p]     transmittance right after that entry (1 if none);
 *   rest[p]  float4: colour blended behind that entry plus T_final bg, and
 *            depth blended behind it (0 if none); 16-byte aligned. */
typedef struct {
    uint32_t* last;
    float* T;
    float* rest;
} gevo_active_state;

/* gevo_render_fwd (same outputs, same values) that also fills *state for the
 * active set `active` (bit mask as in gevo_render_bwd_active).  With it the
 * reverse walk skips every list entry behind a pixel's last active entry:
 * their only effect on the active Gaussians' gradients is through the
 * transmittance and the colour behind, which *state carries. */
gevo_status gevo_render_fwd_active(const gevo_layout* layout, int32_t n, const gevo_proj* proj,
                                   const uint32_t* vals, const uint32_t* ranges, const float* bg,
                                   float* rgb, float* depth, float* T_final, uint32_t* n_contrib,
                                   const uint32_t* active, gevo_active_state* state,
                                   const gevo_tuning* tuning, void* workspace, void* stream);

/* gevo_render_bwd with optional additions, fused into the same reverse walk
 * (one kernel):
 *  - pix_err != NULL (DEVICE float[total_pixels], e.g. from gevo_loss_l1_err):
 *    gauss_err[v * n + g] += sum over view v's pixels u of w(g, u) pix_err[u]
 *    (E_k(g) of Eq. 5; DEVICE float[n_views * n], accumulated -- clear it
 *    first; rows of culled entries are never touched).  gauss_err must be
 *    non-NULL iff pix_err is.
 *  - active != NULL (DEVICE uint32[(n + 31) / 32], bit g % 32 of word g / 32
 *    set = Gaussian g active): rows of *out of inactive Gaussians are not
 *    touched; active rows get exactly what gevo_render_bwd gives them (the
 *    inactive Gaussians still occlude and are still blended).  Inactive list
 *    entries only recover T and the suffix colour, so the walk costs less in
 *    proportion to the inactive share.  An all-zero mask with pix_err gives
 *    the error pass alone.
 *  - state != NULL (requires active, and pix_err == NULL; from
 *    gevo_render_fwd_active with the same mask): each pixel's walk starts at
 *    its last active entry instead of n_contrib - 1.  Active rows get the same
 *    gradients up to rounding (the colour behind comes from the forward pass
 *    instead of the walk).
 * Everything else as gevo_render_bwd. */
gevo_status gevo_render_bwd_active(const gevo_layout* layout, int32_t n, const gevo_proj* proj,
                                   const uint32_t* vals, const uint32_t* ranges, const float* bg,
                                   const float* T_final, const uint32_t* n_contrib,
                                   const float* dL_drgb, const float* dL_ddepth,
                                   const float* dL_dT, const float* pix_err, float* gauss_err,
                                   const uint32_t* active, const gevo_active_state* state,
                                   gevo_grad2d* out, const gevo_tuning* tuning, void* workspace,
                                   void* stream);

/* Words of the `counts` argument of gevo_active_set for n Gaussians. */
#define GEVO_ACTIVE_COUNT_WORDS(n) (((size_t)(n) + 1023) / 1024 + 1)

/* Active set: Gaussian g is active iff gauss_err[k * n + g] > eps for some
 * k < n_views (strict), or bit g of `force` is set (force: DEVICE
 * uint32[(n + 31) / 32] or NULL -- the newly inserted Gaussians).  Writes
 * active (DEVICE uint32[(n + 31) / 32], the bit mask; bits >= n are 0),
 * active_list (DEVICE uint32[n]: the active indices in ascending order in
 * its first counts[0] entries) and counts (DEVICE uint32
 * [GEVO_ACTIVE_COUNT_WORDS(n)]: counts[0] = number of active Gaussians, the
 * rest scratch).  Three kernels, no host synchronisation. */
gevo_status gevo_active_set(int32_t n_views, int32_t n, const float* gauss_err, float eps,
                            const uint32_t* force, uint32_t* active, uint32_t* active_list,
                            uint32_t* counts, void* stream);

/* gevo_project_bwd restricted to the Gaussians active_list[0 .. counts[0])
 * (the outputs of gevo_active_set): their rows of *out are written exactly as
 * gevo_project_bwd writes them; other rows are not touched.  dxi (nullable)
 * is the pose gradient through the listed Gaussians only: with a grad2d from
 * gevo_render_bwd_active, the derivative with the inactive Gaussians' records
 * held fixed. */
gevo_status gevo_project_bwd_active(const gevo_layout* layout, const gevo_gaussians* g,
                                    const gevo_camera* cams, const gevo_proj* proj,
                                    const gevo_grad2d* grad2d, const uint32_t* active_list,
                                    const uint32_t* counts, gevo_gaussian_grads* out, float* dxi,
                                    void* workspace, void* stream);

/* ---------------------------------------------------------------------- */
/* Learned depth prior (spec addition; the paper initialises new      */
/* Gaussians from a cost volume + belief propagation, Section III-A)        */
/* ---------------------------------------------------------------------- */

/* C[M x N] = A[M x K] B[N x K]^T (+ bias[N]) (+ beta * C) (ReLU if relu) on the
 * tcgen05 tensor cores: A, B BF16 row-major with K contiguous (K > 0 and lda,
 * ldb multiples of 8, 16-byte aligned), FP32 accumulation in tensor memory, C
 * FP32 (out_bf16 = 0) or BF16 (out_bf16 = 1) row-major.  bias: DEVICE float[N]
 * or NULL.  workspace: any gevo workspace (its error word records
 * GEVO_ERR_TIMEOUT if an MMA completion wait gives up).  All DEVICE. */
gevo_status gevo_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, int32_t lda,
                           const void* B, int32_t ldb, void* C, int32_t ldc, int32_t out_bf16,
                           const float* bias, int32_t relu, float beta, void* workspace,
                           void* stream);

/* ---------------------------------------------------------------------- */
/* Status                                                                   */
/* ---------------------------------------------------------------------- */

/* Synchronises the stream, returns the sticky device error word (GEVO_OK if
 * clear) and clears it.  Not capturable (it copies to the host). */
gevo_status gevo_last_error(void* workspace, void* stream);

const char* gevo_status_str(gevo_status s);
int32_t gevo_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GEVO_H */
