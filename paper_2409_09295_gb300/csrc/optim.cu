// Map and pose optimisation steps of the local stage (Section III-B1, Eq. 2)
// and the global stage (Section III-B2, Eq. 3): Adam on the Gaussian
// parameters with the isotropic loss fused into the scale gradient, Adam on
// the pose twists with the left-multiplied retraction, and the row gather
// that compacts the map after pruning.
#include "../../include/gevo_map.h"
#include "gevo_internal.cuh"

namespace gevo {

struct AdamC {
    float b1, b2, eps, bc1, bc2;
};

__device__ __forceinline__ float adam1(float p, float g, float* m, float* v, float lr, const AdamC& c)
{
    const float mi = c.b1 * *m + (1.f - c.b1) * g;
    const float vi = c.b2 * *v + (1.f - c.b2) * g * g;
    *m = mi;
    *v = vi;
    return p - lr * (mi / c.bc1) / (sqrtf(vi / c.bc2) + c.eps);
}

__device__ __forceinline__ float sigmoidf(float x) { return 1.f / (1.f + expf(-x)); }

__global__ void k_map_activate(int n, const float* __restrict__ ls, const float* __restrict__ lo,
                               float* __restrict__ s, float* __restrict__ o)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        s[3 * i] = expf(ls[3 * i]);
        s[3 * i + 1] = expf(ls[3 * i + 1]);
        s[3 * i + 2] = expf(ls[3 * i + 2]);
        o[i] = sigmoidf(lo[i]);
    }
}

// One thread per optimised row: means, log-scales (with E_iso), quaternions,
// opacity logit.
__global__ void __launch_bounds__(256)
k_map_step_geo(int n, gevo_map_params P, gevo_gaussian_grads G, gevo_map_params M, gevo_map_params V,
               gevo_map_adam cfg, AdamC c, const uint32_t* __restrict__ rows,
               const uint32_t* __restrict__ counts, float* __restrict__ scales,
               float* __restrict__ opac, float* __restrict__ iso_loss)
{
    const int R = rows ? (int)counts[0] : n;
    const float lam = R > 0 ? cfg.lambda_iso / (float)R : 0.f;
    float e_iso = 0.f;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        const int g = rows ? (int)rows[r] : r;
        if (cfg.lr_means != 0.f)
            for (int a = 0; a < 3; a++)
                P.means[3 * g + a] = adam1(P.means[3 * g + a], G.means[3 * g + a], M.means + 3 * g + a,
                                           V.means + 3 * g + a, cfg.lr_means, c);
        float s[3];
        for (int a = 0; a < 3; a++) s[a] = expf(P.log_scales[3 * g + a]);
        const float mean = (s[0] + s[1] + s[2]) * (1.f / 3.f);
        float sg[3], sgs = 0.f;
        for (int a = 0; a < 3; a++) {
            const float d = s[a] - mean;
            sg[a] = (float)((d > 0.f) - (d < 0.f));
            sgs += sg[a];
            e_iso += lam * fabsf(d);
        }
        if (cfg.lr_log_scales != 0.f)
            for (int a = 0; a < 3; a++) {
                const float gs = (G.scales[3 * g + a] + lam * (sg[a] - sgs * (1.f / 3.f))) * s[a];
                const float nl = adam1(P.log_scales[3 * g + a], gs, M.log_scales + 3 * g + a,
                                       V.log_scales + 3 * g + a, cfg.lr_log_scales, c);
                P.log_scales[3 * g + a] = nl;
                scales[3 * g + a] = expf(nl);
            }
        if (cfg.lr_quats != 0.f)
            for (int a = 0; a < 4; a++)
                P.quats[4 * g + a] = adam1(P.quats[4 * g + a], G.quats[4 * g + a], M.quats + 4 * g + a,
                                           V.quats + 4 * g + a, cfg.lr_quats, c);
        if (cfg.lr_logit_opacities != 0.f) {
            const float o = sigmoidf(P.logit_opacities[g]);
            const float nl = adam1(P.logit_opacities[g], G.opacities[g] * o * (1.f - o),
                                   M.logit_opacities + g, V.logit_opacities + g,
                                   cfg.lr_logit_opacities, c);
            P.logit_opacities[g] = nl;
            opac[g] = sigmoidf(nl);
        }
    }
    if (iso_loss) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e_iso += __shfl_xor_sync(0xffffffffu, e_iso, o);
        if ((threadIdx.x & 31) == 0 && e_iso != 0.f) atomicAdd(iso_loss, e_iso);
    }
}

// Colour coefficients, flat over (row, coefficient, channel) so that a warp
// reads contiguous memory; the degree-0 row has its own learning rate.
__global__ void __launch_bounds__(256)
k_map_step_colour(int n, int K, float* __restrict__ p, const float* __restrict__ grad,
                  float* __restrict__ m, float* __restrict__ v, float lr_dc, float lr_rest, AdamC c,
                  const uint32_t* __restrict__ rows, const uint32_t* __restrict__ counts)
{
    const int R = rows ? (int)counts[0] : n;
    const size_t per = (size_t)3 * K;
    const size_t total = (size_t)R * per;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / per, e = i - r * per;
        const size_t g = rows ? (size_t)rows[r] : r;
        const float lr = e < 3 ? lr_dc : lr_rest;
        if (lr == 0.f) continue;
        const size_t j = g * per + e;
        p[j] = adam1(p[j], grad[j], m + j, v + j, lr, c);
    }
}

// One thread per view: Adam on the twist from a zero start, then
// R <- Rod(phi) R, t <- Rod(phi) t + rho.
__global__ void k_pose_step(int V, float* __restrict__ cams, const float* __restrict__ dxi,
                            float* __restrict__ m, float* __restrict__ v, float lr_rho, float lr_phi,
                            AdamC c, const uint8_t* __restrict__ fixed)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= V || (fixed && fixed[k])) return;
    float xi[6];
    for (int j = 0; j < 6; j++)
        xi[j] = adam1(0.f, dxi[6 * k + j], m + 6 * k + j, v + 6 * k + j, j < 3 ? lr_rho : lr_phi, c);
    const float px = xi[3], py = xi[4], pz = xi[5];
    const float th2 = px * px + py * py + pz * pz;
    float A, B;   // Rod = I + A [phi]x + B [phi]x^2
    if (th2 < 1e-8f) {
        A = 1.f - th2 * (1.f / 6.f);
        B = 0.5f - th2 * (1.f / 24.f);
    } else {
        const float th = sqrtf(th2);
        const float sh = sinf(0.5f * th);
        A = sinf(th) / th;
        B = 2.f * sh * sh / th2;   // (1 - cos th) / th^2 without cancellation
    }
    const float K[9] = {0.f, -pz, py, pz, 0.f, -px, -py, px, 0.f};
    float K2[9], Rx[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            float acc = 0.f;
            for (int l = 0; l < 3; l++) acc += K[3 * i + l] * K[3 * l + j];
            K2[3 * i + j] = acc;
        }
    for (int i = 0; i < 9; i++) Rx[i] = (i % 4 == 0 ? 1.f : 0.f) + A * K[i] + B * K2[i];
    float* cam = cams + 16 * k;
    float R[9], t[3];
    for (int i = 0; i < 9; i++) R[i] = cam[i];
    for (int i = 0; i < 3; i++) t[i] = cam[9 + i];
    for (int i = 0; i < 3; i++) {
        for (int j = 0; j < 3; j++)
            cam[3 * i + j] = Rx[3 * i] * R[j] + Rx[3 * i + 1] * R[3 + j] + Rx[3 * i + 2] * R[6 + j];
        cam[9 + i] = Rx[3 * i] * t[0] + Rx[3 * i + 1] * t[1] + Rx[3 * i + 2] * t[2] + xi[i];
    }
}

__global__ void k_gather_rows(int n_max, const uint32_t* __restrict__ list,
                              const uint32_t* __restrict__ counts, int width,
                              const float* __restrict__ src, float* __restrict__ dst)
{
    const size_t rows = min((size_t)counts[0], (size_t)n_max);
    const size_t total = rows * (size_t)width;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / width, e = i - r * width;
        dst[i] = src[(size_t)list[r] * width + e];
    }
}

static int grid_of(size_t n)
{
    return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, (size_t)sm_count() * 8));
}

static AdamC adam_consts(const gevo_map_adam& cfg, int step)
{
    AdamC c;
    c.b1 = cfg.beta1;
    c.b2 = cfg.beta2;
    c.eps = cfg.eps;
    c.bc1 = 1.f - powf(cfg.beta1, (float)step);
    c.bc2 = 1.f - powf(cfg.beta2, (float)step);
    return c;
}

}  // namespace gevo

using namespace gevo;

extern "C" {

gevo_status gevo_map_activate(int32_t n, const float* log_scales, const float* logit_opacities,
                              float* scales, float* opacities, void* stream)
{
    if (n < 0 || !log_scales || !logit_opacities || !scales || !opacities) return GEVO_ERR_INVALID;
    if (n == 0) return GEVO_OK;
    k_map_activate<<<grid_of((size_t)n), 256, 0, (cudaStream_t)stream>>>(n, log_scales, logit_opacities,
                                                                         scales, opacities);
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}

gevo_status gevo_map_step(int32_t n, int32_t K, gevo_map_params* params,
                          const gevo_gaussian_grads* grads, gevo_map_params* m,
                          gevo_map_params* v, const gevo_map_adam* cfg, int32_t step,
                          const uint32_t* rows, const uint32_t* counts, float* scales,
                          float* opacities, float* iso_loss, void* stream)
{
    auto full = [](const gevo_map_params* p) {
        return p && p->means && p->log_scales && p->quats && p->logit_opacities && p->colours;
    };
    if (n < 0 || K < 1 || K > 16 || !full(params) || !full(m) || !full(v) || !grads || !cfg ||
        step < 1 || !scales || !opacities || (rows && !counts) || !grads->means || !grads->scales ||
        !grads->quats || !grads->opacities)
        return GEVO_ERR_INVALID;
    const float* gcol = grads->sh ? grads->sh : (K == 1 ? grads->rgb : nullptr);
    if (!gcol) return GEVO_ERR_INVALID;
    if (n == 0) return GEVO_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const AdamC c = adam_consts(*cfg, step);
    gevo_gaussian_grads G = *grads;
    k_map_step_geo<<<grid_of((size_t)n), 256, 0, st>>>(n, *params, G, *m, *v, *cfg, c, rows, counts,
                                                       scales, opacities, iso_loss);
    GEVO_CHECK_LAUNCH();
    if (cfg->lr_colour_dc != 0.f || cfg->lr_colour_rest != 0.f) {
        k_map_step_colour<<<grid_of((size_t)n * 3 * K), 256, 0, st>>>(
            n, K, params->colours, gcol, m->colours, v->colours, cfg->lr_colour_dc,
            cfg->lr_colour_rest, c, rows, counts);
        GEVO_CHECK_LAUNCH();
    }
    return GEVO_OK;
}

gevo_status gevo_pose_step(int32_t n_views, float* cams, const float* dxi, float* m, float* v,
                           float lr_rho, float lr_phi, float beta1, float beta2, float eps,
                           int32_t step, const uint8_t* fixed, void* stream)
{
    if (n_views < 1 || !cams || !dxi || !m || !v || step < 1) return GEVO_ERR_INVALID;
    gevo_map_adam cfg{};
    cfg.beta1 = beta1;
    cfg.beta2 = beta2;
    cfg.eps = eps;
    const AdamC c = adam_consts(cfg, step);
    k_pose_step<<<(n_views + 63) / 64, 64, 0, (cudaStream_t)stream>>>(n_views, cams, dxi, m, v,
                                                                       lr_rho, lr_phi, c, fixed);
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}

gevo_status gevo_gather_rows(int32_t n_max, const uint32_t* list, const uint32_t* counts,
                             int32_t width, const float* src, float* dst, void* stream)
{
    if (n_max < 0 || width < 1 || !list || !counts || !src || !dst) return GEVO_ERR_INVALID;
    if (n_max == 0) return GEVO_OK;
    k_gather_rows<<<grid_of((size_t)n_max * width), 256, 0, (cudaStream_t)stream>>>(
        n_max, list, counts, width, src, dst);
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}

}  // extern "C"
