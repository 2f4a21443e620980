/*
 * gevo_map.h -- C ABI of the map and pose optimisation steps of GEVO's two
 * mapping stages: the local stage (Section III-B1, Eq. 2: E_pho + E_iso over
 * the sliding window, the local map and the window poses) and the global
 * stage (Section III-B2, Eq. 3: E_pho + E_iso + E_pc over the active set and
 * the window poses, then pruning of low-opacity Gaussians).  The rasterizer
 * of gevo.h supplies the gradients; these calls turn them into parameter and
 * pose updates, and compact the map after pruning.
 *
 * Optimisation parameters (DEVICE float, caller-owned): means [n][3],
 * log_scales [n][3], raw quaternions [n][4], opacity logits [n] and colour
 * coefficients [n][K][3] (SH of degree d with K = (d + 1)^2, or plain RGB with
 * K = 1).  The rasterizer consumes scales = exp(log_scales) and opacities =
 * sigmoid(logits).  Every call launches on `stream` only, allocates nothing and
 * returns GEVO_ERR_INVALID without launching on bad arguments.
 */
#ifndef GEVO_MAP_H
#define GEVO_MAP_H

#include "gevo.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    float* means;
    float* log_scales;
    float* quats;
    float* logit_opacities;
    float* colours;
} gevo_map_params;

/* Adam hyper-parameters per parameter group; a learning rate of 0 freezes the
 * group.  lambda_iso weighs the isotropic loss E_iso of Eq. 2. */
typedef struct {
    float lr_means, lr_log_scales, lr_quats, lr_logit_opacities, lr_colour_dc, lr_colour_rest;
    float beta1, beta2, eps;
    float lambda_iso;
} gevo_map_adam;

/* scales = exp(log_scales) [n][3], opacities = sigmoid(logits) [n]. */
gevo_status gevo_map_activate(int32_t n, const float* log_scales, const float* logit_opacities,
                              float* scales, float* opacities, void* stream);

/* One Adam step (bias-corrected, step >= 1) of the rows being optimised --
 * rows[0 .. counts[0]) (the list and count of gevo_active_set or
 * gevo_prune_keep), or every Gaussian if rows == NULL -- from the gradients
 * w.r.t. the rasterizer inputs (grads: gevo_project_bwd's output; colour
 * gradients in grads->sh, or grads->rgb when K == 1 and sh is NULL):
 *   dL/dlog s = (dL/ds + dE_iso/ds) s,  dL/dlogit = dL/do o (1 - o),
 *   E_iso = lambda_iso / R * sum over the R rows of sum_a |s_a - mean(s)|.
 * params, m, v: updated in place (m, v zero before the first step); scales,
 * opacities: the rows' activated values rewritten for the next render;
 * iso_loss (nullable, DEVICE float): E_iso added (+=).  Rows not listed are
 * not touched. */
gevo_status gevo_map_step(int32_t n, int32_t K, gevo_map_params* params,
                          const gevo_gaussian_grads* grads, gevo_map_params* m,
                          gevo_map_params* v, const gevo_map_adam* cfg, int32_t step,
                          const uint32_t* rows, const uint32_t* counts, float* scales,
                          float* opacities, float* iso_loss, void* stream);

/* Adam on the left-perturbation twist xi = (rho, phi) of each view's pose
 * (dxi: gevo_project_bwd's [n_views][6]; m, v: [n_views][6]), then the
 * retraction R <- Rod(phi) R, t <- Rod(phi) t + rho applied to cams
 * [n_views][16] in place (R row-major, then t).  Views with fixed[v] != 0
 * (fixed nullable) keep their pose and moments. */
gevo_status gevo_pose_step(int32_t n_views, float* cams, const float* dxi, float* m, float* v,
                           float lr_rho, float lr_phi, float beta1, float beta2, float eps,
                           int32_t step, const uint8_t* fixed, void* stream);

/* Pruning after the global stage: Gaussian g is kept unless it is a candidate
 * (bit g of `candidates`, DEVICE uint32[(n + 31) / 32], NULL = every Gaussian)
 * and opacities[g] < threshold.  Writes keep (bit mask), keep_list (kept
 * indices ascending, first counts[0] entries) and counts
 * (GEVO_ACTIVE_COUNT_WORDS(n) words), like gevo_active_set. */
gevo_status gevo_prune_keep(int32_t n, const float* opacities, const uint32_t* candidates,
                            float threshold, uint32_t* keep, uint32_t* keep_list,
                            uint32_t* counts, void* stream);

/* Row gather: dst[i][0 .. width) = src[list[i]][0 .. width) for i < counts[0]
 * (at most n_max rows).  Compacts every per-Gaussian array after pruning
 * (src and dst must not overlap). */
gevo_status gevo_gather_rows(int32_t n_max, const uint32_t* list, const uint32_t* counts,
                             int32_t width, const float* src, float* dst, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GEVO_MAP_H */
