/*
 * gevo_prior.h -- C ABI of the learned depth prior: a small BF16 U-Net whose
 * convolutions run on the tcgen05 tensor cores (FP32 accumulation in tensor
 * memory).  It proposes depths for the Gaussians of a newly observed region
 * from one RGB image, trained on (RGB, depth) pairs rendered from the map
 * itself.  The paper initialises those Gaussians from a photometric cost
 * volume (Eq. 1) + belief propagation + SPGF* (Section III-A); this learned
 * proposal is an addition the paper does not make, judged against that plain
 * initialisation after the same optimisation.
 *
 * Layouts: activations NHWC BF16, channels a multiple of 8; activation
 * gradients NHWC FP32; 3x3 weights Wt[Cout][ky][kx][Cin] BF16 (K-major rows of
 * 9 Cin); FP32 masters for optimisation.  "ld" arguments are row strides in
 * elements, so an NHWC tensor can be a channel slice of a wider buffer (the
 * U-Net's skip concatenation costs no copy).  All pointers are caller-owned
 * DEVICE memory; every call launches on `stream` only, allocates nothing and
 * returns GEVO_ERR_INVALID without launching on bad arguments.
 */
#ifndef GEVO_PRIOR_H
#define GEVO_PRIOR_H

#include "gevo.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Y = act(conv3x3(X) + bias) + beta * Y, stride 1, zero padding 1: an implicit
 * GEMM (rows = nb*H*W pixels, columns = Cout, depth = 9*Cin) whose A tiles are
 * gathered from X's 3x3 neighbourhoods straight into shared memory.  X:
 * [nb][H][W][Cin] BF16, Cin % 8 == 0; Wt: [Cout][9*Cin]; bias: float[Cout] or
 * NULL; Y: rows of stride ldy (BF16 if out_bf16 else FP32); act = ReLU if relu.
 * The data gradient of a convolution is this call on dZ with gevo_flip3x3
 * weights (no bias, no ReLU, FP32 out).  Sizes: H < 32768, W < 65536 and
 * nb*H*W < 2^31, else GEVO_ERR_INVALID. */
gevo_status gevo_conv3x3(int32_t nb, int32_t H, int32_t W, int32_t Cin, const void* X,
                         int32_t Cout, const void* Wt, const float* bias, void* Y, int32_t ldy,
                         int32_t out_bf16, int32_t relu, float beta, void* workspace,
                         void* stream);

/* Weight gradient dWt[co][(tap, ci)] = sum_p dZ[p][co] col(X)[p][(tap, ci)]
 * (Wt's own layout; FP32, written).  dZt: dZ transposed, [Cout][nb*H*W] BF16
 * (nb*H*W a multiple of 8).  An implicit GEMM (rows = 9*Cin taps x channels,
 * columns = Cout, depth = pixels) whose A tiles are gathered from X's shifted
 * pixels straight into shared memory, with no im2col in memory; the
 * contraction over pixels is split across CTAs and summed with FP32 atomics.
 * Cin % 8 == 0, Cout % 8 == 0; sizes as for gevo_conv3x3. */
gevo_status gevo_conv3x3_wgrad(int32_t nb, int32_t H, int32_t W, int32_t Cin, const void* X,
                               int32_t Cout, const void* dZt, float* dWt, void* workspace,
                               void* stream);

/* dZ = dY * [Y > 0] (BF16 [P][C]); dZt = its transpose (BF16 [C][P], may be NULL);
 * db += sum over pixels of dZ (FP32 [C]).  C <= 128. */
gevo_status gevo_relu_bwd(int64_t P, int32_t C, const float* dY, int32_t lddy, const void* Y,
                          int32_t ldy, void* dZ, void* dZt, float* db, void* stream);

/* 2x2 max pool of X (rows of stride ldx) into Y [nb][H/2][W/2][C]; and its
 * gradient: the first maximum of each window (row-major scan) receives dY,
 * dX = beta * dX + that. */
gevo_status gevo_maxpool2(int32_t nb, int32_t H, int32_t W, int32_t C, const void* X, int32_t ldx,
                          void* Y, void* stream);
gevo_status gevo_maxpool2_bwd(int32_t nb, int32_t H, int32_t W, int32_t C, const void* X,
                              int32_t ldx, const float* dY, float* dX, int32_t lddx, float beta,
                              void* stream);

/* Nearest x2 upsample of X [nb][h][w][C] into rows of stride ldy; its gradient
 * sums the four copies (dX written). */
gevo_status gevo_upsample2(int32_t nb, int32_t h, int32_t w, int32_t C, const void* X, void* Y,
                           int32_t ldy, void* stream);
gevo_status gevo_upsample2_bwd(int32_t nb, int32_t h, int32_t w, int32_t C, const float* dY,
                               int32_t lddy, float* dX, void* stream);

/* Wf[ci][tap][co] = Wt[co][8 - tap][ci]. */
gevo_status gevo_flip3x3(int32_t Cout, int32_t Cin, const void* Wt, void* Wf, void* stream);

/* Planar FP32 RGB renders [nb][3][H][W] -> NHWC BF16 with 8 channels: the
 * network input rgb - 0.5 (centred) in channels 0..2, zeros in 3..7. */
gevo_status gevo_rgb_pack(int32_t nb, int32_t H, int32_t W, const float* rgb, void* X,
                          void* stream);

/* 1x1 head to one channel: pred[p] = sum_c w[c] X[p][c] + b[0] (C <= 16), and
 * its gradient (dX written [P][C] FP32; dw, db written). */
gevo_status gevo_head_fwd(int64_t P, int32_t C, const void* X, const float* w, const float* b,
                          float* pred, void* stream);
gevo_status gevo_head_bwd(int64_t P, int32_t C, const void* X, const float* w, const float* dpred,
                          float* dX, float* dw, float* db, void* stream);

/* Target log-depth from a render: log(D / (1 - T)) where 1 - T >= 0.5 (weight
 * 1), else weight 0. */
gevo_status gevo_depth_target(int64_t P, const float* depth, const float* T_final, float* target,
                              float* weight, void* stream);

/* L = (1/P) sum_p weight |pred - target| (loss: float[1], written) and its
 * gradient (sign(0) = 0). */
gevo_status gevo_depth_l1(int64_t P, const float* pred, const float* target, const float* weight,
                          float* loss, float* grad, void* stream);

/* One Adam step (bias-corrected, step >= 1) on FP32 masters; param_bf16 (may
 * be NULL) receives a BF16 copy of the updated values. */
gevo_status gevo_adam(int64_t n, float* param, const float* grad, float* m, float* v,
                      void* param_bf16, float lr, float beta1, float beta2, float eps,
                      int32_t step, void* stream);

/* Plain initialisation of Section III-A: the photometric cost volume of Eq. 1
 * for reference keyframe `ref` of nk keyframes rgb [nk][3][H][W] (H, W
 * multiples of 4) with cameras cams [nk][16] (R, t, fx, fy, cx, cy), at 1/4
 * resolution over nd depth hypotheses spaced linearly on [d0, d1]:
 * volume[(y * W/4 + x) * nd + k] = mean over the other keyframes, where the
 * sample falls inside the image, of |grey_ref(u) - grey_i(pi(u, d_k))|
 * (grey = mean of RGB after a 4x4 box average, bilinear sampling; 1.0 where
 * no keyframe sees the point).  grey: scratch [nk][H/4][W/4].  depth
 * [H][W]: winner-take-all hypothesis (lowest cost, then lowest k), nearest x4
 * upsampled -- standing in for the belief propagation and edge-aware
 * upsampling the paper cites. */
gevo_status gevo_cost_volume(int32_t nk, int32_t ref, int32_t H, int32_t W, const float* rgb,
                             const float* cams, int32_t nd, float d0, float d1, float* grey,
                             float* volume, float* depth, void* stream);

/* New Gaussians from a depth map (z-depth of pixel (x, y) sampled at
 * coordinate x, camera cam[16]): every pixel with mask > 0.5 whose 32-bit hash
 * (seeded) is <= keep becomes one Gaussian -- mean at its back-projection,
 * colour SH DC (rgb - 0.5) / Y00 with higher bands 0, isotropic scale
 * scale_px * depth / fx, identity rotation, the given opacity -- written at
 * slot atomicAdd(counter, 1) if that slot is below cap (order unspecified).
 * rgb planar [3][H][W]. */
/* Belief propagation over a cost volume (Section III-A2, the min-sum algorithm
 * of Felzenszwalb and Huttenlocher the paper cites): labels are the nd <= 64
 * depth hypotheses of volume [h][w][nd] (gevo_cost_volume's layout, the data
 * cost), neighbours on the 4-connected grid pay min(s |f_p - f_q|, tau),
 * messages start at zero and all are updated together for `iters`
 * iterations (each shifted to minimum 0).  Writes depth [4h][4w] (the label
 * minimising data cost + incoming messages, lowest on ties, as
 * d0 + (d1 - d0) f / (nd - 1), nearest x4), and if non-NULL labels [h][w] and
 * beliefs [h][w][nd].  msgs: scratch of 2 * 4 * h * w * nd floats. */
gevo_status gevo_depth_bp(int32_t h, int32_t w, int32_t nd, const float* volume, float s,
                          float tau, int32_t iters, float d0, float d1, float* msgs, float* depth,
                          int32_t* labels, float* beliefs, void* stream);

gevo_status gevo_unproject(int32_t H, int32_t W, const float* rgb, const float* depth,
                           const float* mask, const float* cam, uint32_t keep, uint32_t seed,
                           float scale_px, float opacity, int32_t sh_degree, uint32_t* counter,
                           int32_t cap, float* means, float* scales, float* quats,
                           float* opacities, float* sh, void* stream);

/* y = bf16(x). */
gevo_status gevo_to_bf16(int64_t n, const float* x, void* y, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GEVO_PRIOR_H */
