// Stage a1 (projection) and stage a7 (its derivative, including the camera
// pose as an se(3) twist) of the splatting renderer GEVO optimises through
// (Section I "GS"; Section III-B, Eq. 2 and Eq. 3 optimise the map and T_k).
//
// One thread per Gaussian; the thread loops over every view of the batch, so
// the Gaussian's parameters (up to 236 bytes with degree-3 SH) are read from HBM
// once for all views and the 3-D covariance factor is built once.
//
// Numerics: the 2-D covariance is formed as Sigma2 = T T^T + 0.3 I with
// T = J W Rq diag(s) (2x3), and its determinant as |T0 x T1|^2 + 0.3 (|T0|^2 +
// |T1|^2) + 0.09 (Lagrange identity): every term is non-negative, so the
// determinant of a thin, elongated splat keeps full binary32 precision.
#include "gevo_internal.cuh"

namespace gevo {

// Real SH basis constants (closed forms 1/(2 sqrt(pi)), sqrt(3/(4 pi)), ...).
__constant__ float kSH[16] = {
    0.28209479177387814f,
    -0.4886025119029199f, 0.4886025119029199f, -0.4886025119029199f,
    1.0925484305920792f, -1.0925484305920792f, 0.31539156525252005f, -1.0925484305920792f,
    0.5462742152960396f,
    -0.5900435899266435f, 2.890611442640554f, -0.4570457994644658f, 0.3731763325901154f,
    -0.4570457994644658f, 1.445305721320277f, -0.5900435899266435f};

template <int DEG>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float Y[16])
{
    Y[0] = kSH[0];
    if (DEG >= 1) {
        Y[1] = kSH[1] * y; Y[2] = kSH[2] * z; Y[3] = kSH[3] * x;
    }
    if (DEG >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kSH[4] * x * y; Y[5] = kSH[5] * y * z; Y[6] = kSH[6] * (2.f * zz - xx - yy);
        Y[7] = kSH[7] * x * z; Y[8] = kSH[8] * (xx - yy);
        if (DEG >= 3) {
            Y[9] = kSH[9] * y * (3.f * xx - yy);
            Y[10] = kSH[10] * x * y * z;
            Y[11] = kSH[11] * y * (4.f * zz - xx - yy);
            Y[12] = kSH[12] * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = kSH[13] * x * (4.f * zz - xx - yy);
            Y[14] = kSH[14] * z * (xx - yy);
            Y[15] = kSH[15] * x * (xx - 3.f * yy);
        }
    }
}

// Gradient of sum_k Y_k(d) w_k with respect to d, for per-basis weights w_k.
template <int DEG>
__device__ __forceinline__ void sh_grad_dir(float x, float y, float z, const float w[16],
                                            float& gx, float& gy, float& gz)
{
    gx = gy = gz = 0.f;
    if (DEG >= 1) {
        gy += kSH[1] * w[1]; gz += kSH[2] * w[2]; gx += kSH[3] * w[3];
    }
    if (DEG >= 2) {
        gx += kSH[4] * y * w[4];           gy += kSH[4] * x * w[4];
        gy += kSH[5] * z * w[5];           gz += kSH[5] * y * w[5];
        gx += -2.f * kSH[6] * x * w[6];    gy += -2.f * kSH[6] * y * w[6];
        gz += 4.f * kSH[6] * z * w[6];
        gx += kSH[7] * z * w[7];           gz += kSH[7] * x * w[7];
        gx += 2.f * kSH[8] * x * w[8];     gy += -2.f * kSH[8] * y * w[8];
    }
    if (DEG >= 3) {
        const float xx = x * x, yy = y * y, zz = z * z;
        gx += kSH[9] * 6.f * x * y * w[9];
        gy += kSH[9] * 3.f * (xx - yy) * w[9];
        gx += kSH[10] * y * z * w[10]; gy += kSH[10] * x * z * w[10]; gz += kSH[10] * x * y * w[10];
        gx += kSH[11] * -2.f * x * y * w[11];
        gy += kSH[11] * (4.f * zz - xx - 3.f * yy) * w[11];
        gz += kSH[11] * 8.f * y * z * w[11];
        gx += kSH[12] * -6.f * x * z * w[12];
        gy += kSH[12] * -6.f * y * z * w[12];
        gz += kSH[12] * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
        gx += kSH[13] * (4.f * zz - 3.f * xx - yy) * w[13];
        gy += kSH[13] * -2.f * x * y * w[13];
        gz += kSH[13] * 8.f * x * z * w[13];
        gx += kSH[14] * 2.f * x * z * w[14]; gy += kSH[14] * -2.f * y * z * w[14];
        gz += kSH[14] * (xx - yy) * w[14];
        gx += kSH[15] * 3.f * (xx - yy) * w[15]; gy += kSH[15] * -6.f * x * y * w[15];
    }
}

// Camera block in shared memory: R[9], t[3], fx, fy, cx, cy, centre[3],
// guard limits (lx, ly).
struct CamS {
    float R[9], t[3], fx, fy, cx, cy, c[3], lx, ly;
};

__device__ __forceinline__ void load_cams(const gevo_layout& L, const gevo_camera* cams,
                                          CamS* s)
{
    for (int v = threadIdx.x; v < L.n_views; v += blockDim.x) {
        const gevo_camera k = cams[v];
        CamS o;
#pragma unroll
        for (int i = 0; i < 9; i++) o.R[i] = k.R[i];
        o.t[0] = k.t[0]; o.t[1] = k.t[1]; o.t[2] = k.t[2];
        o.fx = k.fx; o.fy = k.fy; o.cx = k.cx; o.cy = k.cy;
#pragma unroll
        for (int i = 0; i < 3; i++)
            o.c[i] = -(k.R[i] * k.t[0] + k.R[3 + i] * k.t[1] + k.R[6 + i] * k.t[2]);
        o.lx = kGuard * 0.5f * (float)L.width[v] / k.fx;
        o.ly = kGuard * 0.5f * (float)L.height[v] / k.fy;
        s[v] = o;
    }
}

__device__ __forceinline__ void quat_to_rot(float4 q, float R[9], float qn[4], float& inv_norm)
{
    inv_norm = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float w = q.x * inv_norm, x = q.y * inv_norm, y = q.z * inv_norm, z = q.w * inv_norm;
    qn[0] = w; qn[1] = x; qn[2] = y; qn[3] = z;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

template <int DEG, bool HAS_RGB>
__device__ __forceinline__ void load_colour(const float* __restrict__ coef, int g, float k[16][3])
{
    constexpr int K = (DEG + 1) * (DEG + 1);
    if (HAS_RGB) {
        k[0][0] = coef[3 * g]; k[0][1] = coef[3 * g + 1]; k[0][2] = coef[3 * g + 2];
    } else if ((K * 3) % 4 == 0) {
        const float4* p = reinterpret_cast<const float4*>(coef + (size_t)g * K * 3);
        float tmp[K * 3];
#pragma unroll
        for (int i = 0; i < K * 3 / 4; i++) {
            float4 u = __ldg(p + i);
            tmp[4 * i] = u.x; tmp[4 * i + 1] = u.y; tmp[4 * i + 2] = u.z; tmp[4 * i + 3] = u.w;
        }
#pragma unroll
        for (int i = 0; i < K; i++) { k[i][0] = tmp[3 * i]; k[i][1] = tmp[3 * i + 1]; k[i][2] = tmp[3 * i + 2]; }
    } else {
#pragma unroll
        for (int i = 0; i < K; i++)
#pragma unroll
            for (int ch = 0; ch < 3; ch++) k[i][ch] = __ldg(coef + ((size_t)g * K + i) * 3 + ch);
    }
}

// Everything the forward computes for one (view, Gaussian), reused by the
// backward so both take identical binary32 decisions.
struct Geo {
    float p[3];      // camera-frame mean
    float iz;
    float txz, tyz;  // (clamped) x/z, y/z
    bool clx, cly;   // clamp active
    float J00, J02, J11, J12;
    float M[6];      // J W
    float T[6];      // M Rq diag(s)
    float a, b, c, det;
};

__device__ __forceinline__ void geometry(const CamS& cam, const float mu[3], const float N[9], Geo& G)
{
#pragma unroll
    for (int i = 0; i < 3; i++)
        G.p[i] = cam.R[3 * i] * mu[0] + cam.R[3 * i + 1] * mu[1] + cam.R[3 * i + 2] * mu[2] + cam.t[i];
    G.iz = 1.f / G.p[2];
    const float rx = G.p[0] * G.iz, ry = G.p[1] * G.iz;
    G.clx = (rx > cam.lx) || (rx < -cam.lx);
    G.cly = (ry > cam.ly) || (ry < -cam.ly);
    G.txz = fminf(fmaxf(rx, -cam.lx), cam.lx);
    G.tyz = fminf(fmaxf(ry, -cam.ly), cam.ly);
    G.J00 = cam.fx * G.iz;
    G.J02 = -cam.fx * G.txz * G.iz;
    G.J11 = cam.fy * G.iz;
    G.J12 = -cam.fy * G.tyz * G.iz;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        G.M[i] = G.J00 * cam.R[i] + G.J02 * cam.R[6 + i];
        G.M[3 + i] = G.J11 * cam.R[3 + i] + G.J12 * cam.R[6 + i];
    }
#pragma unroll
    for (int r = 0; r < 2; r++)
#pragma unroll
        for (int k = 0; k < 3; k++)
            G.T[3 * r + k] = G.M[3 * r] * N[k] + G.M[3 * r + 1] * N[3 + k] + G.M[3 * r + 2] * N[6 + k];
    const float n0 = G.T[0] * G.T[0] + G.T[1] * G.T[1] + G.T[2] * G.T[2];
    const float n1 = G.T[3] * G.T[3] + G.T[4] * G.T[4] + G.T[5] * G.T[5];
    const float cx_ = G.T[1] * G.T[5] - G.T[2] * G.T[4];
    const float cy_ = G.T[2] * G.T[3] - G.T[0] * G.T[5];
    const float cz_ = G.T[0] * G.T[4] - G.T[1] * G.T[3];
    G.a = n0 + kDilation;
    G.c = n1 + kDilation;
    G.b = G.T[0] * G.T[3] + G.T[1] * G.T[4] + G.T[2] * G.T[5];
    G.det = (cx_ * cx_ + cy_ * cy_ + cz_ * cz_) + kDilation * (n0 + n1) + kDilation * kDilation;
}

// Colour of a Gaussian with mean mu seen from camera centre c: its rgb, or
// max(0, sum_k Y_k(d) k_k + 0.5) with d the unit direction from c to mu.
template <int DEG, bool HAS_RGB>
__device__ __forceinline__ void colour_of(const float mu[3], const float c[3],
                                          const float k[16][3], float rgb[3])
{
    constexpr int K = (DEG + 1) * (DEG + 1);
    if (HAS_RGB) {
        rgb[0] = k[0][0]; rgb[1] = k[0][1]; rgb[2] = k[0][2];
    } else {
        float dx = mu[0] - c[0], dy = mu[1] - c[1], dz = mu[2] - c[2];
        const float inl = rsqrtf(dx * dx + dy * dy + dz * dz);
        dx *= inl; dy *= inl; dz *= inl;
        float Y[16];
        sh_eval<DEG>(dx, dy, dz, Y);
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            float acc = 0.5f;
#pragma unroll
            for (int i = 0; i < K; i++) acc += Y[i] * k[i][ch];
            rgb[ch] = fmaxf(acc, 0.f);
        }
    }
}

// COLOUR false: the geometry part alone (colours left 0, the colour part writes
// them); the colour parameters are not read.
template <int DEG, bool HAS_RGB, bool COLOUR>
__global__ void __launch_bounds__(128)
k_project_fwd(gevo_layout L, int n, const float* __restrict__ means, const float* __restrict__ scales,
              const float4* __restrict__ quats, const float* __restrict__ opac,
              const float* __restrict__ coef, const gevo_camera* __restrict__ cams,
              float2* __restrict__ out_xy, float4* __restrict__ out_co, float4* __restrict__ out_rz,
              int* __restrict__ out_r, uint32_t* __restrict__ out_tiles, uint32_t* err,
              int g_begin, int g_end, float2* __restrict__ z_xy, float4* __restrict__ z_co,
              float4* __restrict__ z_rz)
{
    __shared__ CamS s_cam[GEVO_MAX_VIEWS];
    load_cams(L, cams, s_cam);
    __syncthreads();
    const int g = g_begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= g_end) return;

    const float mu[3] = {means[3 * g], means[3 * g + 1], means[3 * g + 2]};
    const float s[3] = {scales[3 * g], scales[3 * g + 1], scales[3 * g + 2]};
    const float o = opac[g];
    float Rq[9], qn[4], qinv;
    quat_to_rot(__ldg(quats + g), Rq, qn, qinv);
    float N[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) N[3 * i + k] = Rq[3 * i + k] * s[k];
    float k[16][3];
    if (COLOUR) load_colour<DEG, HAS_RGB>(coef, g, k);

    bool nonfinite = false;
    for (int v = 0; v < L.n_views; v++) {
        const CamS& cam = s_cam[v];
        const size_t idx = (size_t)v * n + g;
        Geo G;
        geometry(cam, mu, N, G);
        int r = 0;
        uint32_t area = 0;
        if (G.p[2] > kNearZ) {
            const float idet = 1.f / G.det;
            const float ca = G.c * idet, cb = -G.b * idet, cc = G.a * idet;
            const float half = 0.5f * (G.a - G.c);
            const float lmax = 0.5f * (G.a + G.c) + sqrtf(fmaxf(0.1f, half * half + G.b * G.b));
            const float rr = ceilf(3.f * sqrtf(lmax));
            const float mx = cam.fx * G.p[0] * G.iz + (cam.cx - 0.5f);
            const float my = cam.fy * G.p[1] * G.iz + (cam.cy - 0.5f);
            const bool fin = isfinite(mx) && isfinite(my) && isfinite(ca) && isfinite(cb) &&
                             isfinite(cc) && isfinite(rr);
            if (!fin) {
                nonfinite = true;
            } else if (G.det > 0.f) {
                r = (int)fminf(rr, 1.0e7f);
                int x0, y0, x1, y1;
                tile_rect(mx, my, r, L.tiles_x[v], L.tiles_y[v], x0, y0, x1, y1);
                area = (uint32_t)((x1 - x0) * (y1 - y0));
                if (area == 0) {
                    r = 0;
                } else {
                    float rgb[3] = {0.f, 0.f, 0.f};
                    if (COLOUR) colour_of<DEG, HAS_RGB>(mu, cam.c, k, rgb);
                    out_xy[idx] = make_float2(mx, my);
                    out_co[idx] = make_float4(ca, cb, cc, o);
                    out_rz[idx] = make_float4(rgb[0], rgb[1], rgb[2], G.p[2]);
                    if (z_xy) {   // the reverse walk accumulates into exactly these rows
                        z_xy[idx] = make_float2(0.f, 0.f);
                        z_co[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
                        z_rz[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
        } else if (!(G.p[2] == G.p[2])) {
            nonfinite = true;
        }
        out_r[idx] = r;
        out_tiles[idx] = area;
    }
    if (nonfinite) atomicOr(err, kErrNonFinite);
}

// ---------------------------------------------------------------------------
// Backward.
// ---------------------------------------------------------------------------
// Visible views of Gaussian g as a bit mask (at most 64 views).
__device__ __forceinline__ unsigned long long visible_views(const gevo_layout& L, int n, int g,
                                                            const int* __restrict__ radius)
{
    unsigned long long m = 0ull;
    for (int v = 0; v < L.n_views; v++)
        if (radius[(size_t)v * n + g] > 0) m |= 1ull << v;
    return m;
}

// Colour part of the projection: for every entry the geometry part left
// visible (radius > 0) the colour, written to x, y, z of rgb_depth only -- its
// w (the depth) may be read meanwhile, by the sort.
template <int DEG, bool HAS_RGB>
__global__ void __launch_bounds__(128)
k_project_colour(gevo_layout L, int n, const float* __restrict__ means,
                 const float* __restrict__ coef, const gevo_camera* __restrict__ cams,
                 const int* __restrict__ radius, float4* __restrict__ out_rz, int g_begin, int g_end)
{
    __shared__ CamS s_cam[GEVO_MAX_VIEWS];
    load_cams(L, cams, s_cam);
    __syncthreads();
    const int g = g_begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= g_end) return;
    unsigned long long vis = visible_views(L, n, g, radius);
    if (!vis) return;
    const float mu[3] = {means[3 * g], means[3 * g + 1], means[3 * g + 2]};
    float k[16][3];
    load_colour<DEG, HAS_RGB>(coef, g, k);
    while (vis) {
        const int v = __ffsll((long long)vis) - 1;
        vis &= vis - 1;
        float rgb[3];
        colour_of<DEG, HAS_RGB>(mu, s_cam[v].c, k, rgb);
        float* rz = reinterpret_cast<float*>(out_rz + (size_t)v * n + g);
        *reinterpret_cast<float2*>(rz) = make_float2(rgb[0], rgb[1]);
        rz[2] = rgb[2];
    }
}

// The order the projection backward walks the Gaussians in.  Each lane of its
// kernels walks its own Gaussian's visible views, so a warp takes as many
// iterations as its busiest lane: in id order that is 2.25 times the mean on
// the 16-view benchmark (10.3 against 4.6 views).  Here each range of
// kPbwdRange (1024) consecutive Gaussians is put in order of decreasing
// visible-view count (1.06 times the mean; 1.13 for ranges of 512, measured
// slower), and each Gaussian's visible-view mask is stored
// beside it, so the kernels read one word instead of a radius per view.  The
// order inside a count is the order of a shared-memory atomic (each Gaussian is
// still handled once); loads stay within the range's window.
constexpr int kPbwdRange = GEVO_PART_RANGE;
__global__ void __launch_bounds__(kPbwdRange)
k_pbwd_order(gevo_layout L, int n, const int* __restrict__ radius, uint32_t* __restrict__ perm,
             unsigned long long* __restrict__ vmask)
{
    __shared__ uint32_t s_n[GEVO_MAX_VIEWS + 1];
    const int g = blockIdx.x * kPbwdRange + threadIdx.x;
    for (int i = threadIdx.x; i <= L.n_views; i += blockDim.x) s_n[i] = 0u;
    __syncthreads();
    const unsigned long long m = g < n ? visible_views(L, n, g, radius) : 0ull;
    const int b = L.n_views - __popcll(m);   // the busiest first
    const uint32_t r = g < n ? atomicAdd(s_n + b, 1u) : 0u;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0u;
        for (int i = 0; i <= L.n_views; i++) {
            const uint32_t c = s_n[i];
            s_n[i] = acc;
            acc += c;
        }
    }
    __syncthreads();
    if (g < n) {
        const int pos = blockIdx.x * kPbwdRange + (int)(s_n[b] + r);
        perm[pos] = (uint32_t)g;
        vmask[pos] = m;
    }
}

// Per-view pose-gradient sums are kept in shared memory in kDxiCopies copies,
// lane l adding into copy l % kDxiCopies: lanes of a warp that reach the same
// view at once would otherwise serialise on one address.
constexpr int kDxiCopies = 16;

// Geometry part of the projection derivative: mean (through the camera-frame
// mean, the image mean, the depth and the EWA Jacobian), scale and rotation
// (through Sigma3), opacity, RGB colours if given, and the pose twist except
// its colour term.  Each lane walks only its own visible views, so a warp does
// max-over-lanes rather than all-views iterations; the per-view twist sums go
// through shared-memory atomics.
template <bool HAS_RGB, bool ADD_MEANS>
__global__ void __launch_bounds__(128)
k_project_bwd_geo(gevo_layout L, int n, const float* __restrict__ means,
                  const float* __restrict__ scales, const float4* __restrict__ quats,
                  const gevo_camera* __restrict__ cams, const int* __restrict__ radius,
                  const float2* __restrict__ g_xy, const float4* __restrict__ g_co,
                  const float4* __restrict__ g_rz, float* __restrict__ d_means,
                  float* __restrict__ d_scales, float4* __restrict__ d_quats,
                  float* __restrict__ d_opac, float* __restrict__ d_rgb, float* __restrict__ dxi,
                  const uint32_t* __restrict__ list, const uint32_t* __restrict__ list_count,
                  const unsigned long long* __restrict__ vmask, int t_begin, int t_end)
{
    __shared__ CamS s_cam[GEVO_MAX_VIEWS];
    __shared__ float s_dxi[GEVO_MAX_VIEWS][kDxiCopies][6];
    const int total = list_count ? (int)*list_count : t_end;
    if (t_begin + (int)(blockIdx.x * blockDim.x) >= total) return;   // whole block: before any barrier
    load_cams(L, cams, s_cam);
    for (int i = threadIdx.x; i < L.n_views * kDxiCopies * 6; i += blockDim.x) (&s_dxi[0][0][0])[i] = 0.f;
    __syncthreads();
    const int t = t_begin + blockIdx.x * blockDim.x + threadIdx.x;
    const int g = t < total ? (list ? (int)list[t] : t) : n;
    if (g < n) {
        const float mu[3] = {means[3 * g], means[3 * g + 1], means[3 * g + 2]};
        const float s[3] = {scales[3 * g], scales[3 * g + 1], scales[3 * g + 2]};
        float Rq[9], qn[4], qinv;
        quat_to_rot(__ldg(quats + g), Rq, qn, qinv);
        float N[9];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int k = 0; k < 3; k++) N[3 * i + k] = Rq[3 * i + k] * s[k];
        float dmu[3] = {0.f, 0.f, 0.f}, dN[9], dop = 0.f, drgb[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 9; i++) dN[i] = 0.f;
        unsigned long long vis = vmask ? vmask[t] : visible_views(L, n, g, radius);
        while (vis) {
            const int v = __ffsll((long long)vis) - 1;
            vis &= vis - 1;
            const CamS& cam = s_cam[v];
            const size_t idx = (size_t)v * n + g;
            const float2 gxy = g_xy[idx];
            const float4 gco = g_co[idx];
            const float4 grz = g_rz[idx];
            Geo G;
            geometry(cam, mu, N, G);
            dop += gco.w;
            if (HAS_RGB) { drgb[0] += grz.x; drgb[1] += grz.y; drgb[2] += grz.z; }
            const float idet = 1.f / G.det;
            const float ca = G.c * idet, cb = -G.b * idet, cc = G.a * idet;
            // dL/dSigma2 = -Q Gc Q with Gc = [[gA, gB/2], [gB/2, gC]]
            const float hb = 0.5f * gco.y;
            const float q00 = ca * gco.x + cb * hb, q01 = ca * hb + cb * gco.z;
            const float q10 = cb * gco.x + cc * hb, q11 = cb * hb + cc * gco.z;
            const float dA = -(q00 * ca + q01 * cb), dC = -(q10 * cb + q11 * cc);
            const float dB = -2.f * (q00 * cb + q01 * cc);
            // Sigma2 = T T^T + 0.3 I  ->  dT = 2 [[dA, dB/2], [dB/2, dC]] T
            float dT[6];
#pragma unroll
            for (int kk = 0; kk < 3; kk++) {
                dT[kk] = 2.f * dA * G.T[kk] + dB * G.T[3 + kk];
                dT[3 + kk] = dB * G.T[kk] + 2.f * dC * G.T[3 + kk];
            }
            float dM[6];   // T = M N
#pragma unroll
            for (int r = 0; r < 2; r++)
#pragma unroll
                for (int i = 0; i < 3; i++)
                    dM[3 * r + i] = dT[3 * r] * N[3 * i] + dT[3 * r + 1] * N[3 * i + 1] +
                                    dT[3 * r + 2] * N[3 * i + 2];
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int kk = 0; kk < 3; kk++) dN[3 * i + kk] += G.M[i] * dT[kk] + G.M[3 + i] * dT[3 + kk];
            // M = J W
            const float dJ00 = dM[0] * cam.R[0] + dM[1] * cam.R[1] + dM[2] * cam.R[2];
            const float dJ02 = dM[0] * cam.R[6] + dM[1] * cam.R[7] + dM[2] * cam.R[8];
            const float dJ11 = dM[3] * cam.R[3] + dM[4] * cam.R[4] + dM[5] * cam.R[5];
            const float dJ12 = dM[3] * cam.R[6] + dM[4] * cam.R[7] + dM[5] * cam.R[8];
            const float iz = G.iz, iz2 = iz * iz;
            float dp[3];
            dp[0] = gxy.x * cam.fx * iz;
            dp[1] = gxy.y * cam.fy * iz;
            dp[2] = -(gxy.x * cam.fx * G.p[0] + gxy.y * cam.fy * G.p[1]) * iz2 + grz.w;
            dp[2] += -(dJ00 * cam.fx + dJ11 * cam.fy) * iz2;
            if (!G.clx) {
                dp[0] += -dJ02 * cam.fx * iz2;
                dp[2] += 2.f * dJ02 * cam.fx * G.p[0] * iz2 * iz;
            } else {
                dp[2] += dJ02 * cam.fx * G.txz * iz2;
            }
            if (!G.cly) {
                dp[1] += -dJ12 * cam.fy * iz2;
                dp[2] += 2.f * dJ12 * cam.fy * G.p[1] * iz2 * iz;
            } else {
                dp[2] += dJ12 * cam.fy * G.tyz * iz2;
            }
#pragma unroll
            for (int j = 0; j < 3; j++)
                dmu[j] += cam.R[j] * dp[0] + cam.R[3 + j] * dp[1] + cam.R[6 + j] * dp[2];
            if (dxi) {
                float dW[9];  // dW[k][i] = sum_r J[r][k] dM[r][i]
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    dW[i] = G.J00 * dM[i];
                    dW[3 + i] = G.J11 * dM[3 + i];
                    dW[6 + i] = G.J02 * dM[i] + G.J12 * dM[3 + i];
                }
                float B[9];  // dW W^T
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int j = 0; j < 3; j++)
                        B[3 * i + j] = dW[3 * i] * cam.R[3 * j] + dW[3 * i + 1] * cam.R[3 * j + 1] +
                                       dW[3 * i + 2] * cam.R[3 * j + 2];
                float* o = s_dxi[v][threadIdx.x % kDxiCopies];
                atomicAdd(o + 0, dp[0]);
                atomicAdd(o + 1, dp[1]);
                atomicAdd(o + 2, dp[2]);
                atomicAdd(o + 3, G.p[1] * dp[2] - G.p[2] * dp[1] + B[7] - B[5]);
                atomicAdd(o + 4, G.p[2] * dp[0] - G.p[0] * dp[2] + B[2] - B[6]);
                atomicAdd(o + 5, G.p[0] * dp[1] - G.p[1] * dp[0] + B[3] - B[1]);
            }
        }
        // N = Rq diag(s)
        float dRq[9];
#pragma unroll
        for (int kk = 0; kk < 3; kk++) {
            d_scales[3 * g + kk] = dN[kk] * Rq[kk] + dN[3 + kk] * Rq[3 + kk] + dN[6 + kk] * Rq[6 + kk];
#pragma unroll
            for (int i = 0; i < 3; i++) dRq[3 * i + kk] = dN[3 * i + kk] * s[kk];
        }
        const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
        const float* Gq = dRq;
        float dq[4];
        dq[0] = 2.f * (-z * Gq[1] + y * Gq[2] + z * Gq[3] - x * Gq[5] - y * Gq[6] + x * Gq[7]);
        dq[1] = 2.f * (y * Gq[1] + z * Gq[2] + y * Gq[3] - 2.f * x * Gq[4] - w * Gq[5] + z * Gq[6] +
                       w * Gq[7] - 2.f * x * Gq[8]);
        dq[2] = 2.f * (-2.f * y * Gq[0] + x * Gq[1] + w * Gq[2] + x * Gq[3] + z * Gq[5] - w * Gq[6] +
                       z * Gq[7] - 2.f * y * Gq[8]);
        dq[3] = 2.f * (-2.f * z * Gq[0] - w * Gq[1] + x * Gq[2] + w * Gq[3] - 2.f * z * Gq[4] +
                       y * Gq[5] + x * Gq[6] + y * Gq[7]);
        const float dot = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
        d_quats[g] = make_float4((dq[0] - w * dot) * qinv, (dq[1] - x * dot) * qinv,
                                 (dq[2] - y * dot) * qinv, (dq[3] - z * dot) * qinv);
        if (ADD_MEANS) {   // onto the SH colour kernel's share
            d_means[3 * g] += dmu[0]; d_means[3 * g + 1] += dmu[1]; d_means[3 * g + 2] += dmu[2];
        } else {
            d_means[3 * g] = dmu[0]; d_means[3 * g + 1] = dmu[1]; d_means[3 * g + 2] = dmu[2];
        }
        d_opac[g] = dop;
        if (HAS_RGB) { d_rgb[3 * g] = drgb[0]; d_rgb[3 * g + 1] = drgb[1]; d_rgb[3 * g + 2] = drgb[2]; }
    }
    if (dxi) {
        __syncthreads();
        for (int i = threadIdx.x; i < L.n_views * 6; i += blockDim.x) {
            float r = 0.f;
#pragma unroll
            for (int c = 0; c < kDxiCopies; c++) r += s_dxi[i / 6][c][i % 6];
            if (r != 0.f) atomicAdd(dxi + i, r);
        }
    }
}

// SH colour part: colour = max(0, sum_k Y_k(d) k_k + 0.5), d the unit direction
// from the camera centre.  Writes dL/dSH and the direction's share of dL/dmean
// (k_project_bwd_geo, launched after it, adds the rest) and adds the camera
// centre's share to the translation part of the pose twist.  It runs first so
// that the SH gradients, most of the bytes, are final while the geometry part
// still runs.
template <int DEG>
__global__ void __launch_bounds__(128)
k_project_bwd_col(gevo_layout L, int n, const float* __restrict__ means,
                  const float* __restrict__ coef, const gevo_camera* __restrict__ cams,
                  const int* __restrict__ radius, const float4* __restrict__ g_rz,
                  float* __restrict__ d_means, float* __restrict__ d_coef, float* __restrict__ dxi,
                  const uint32_t* __restrict__ list, const uint32_t* __restrict__ list_count,
                  const unsigned long long* __restrict__ vmask, int t_begin, int t_end)
{
    constexpr int K = (DEG + 1) * (DEG + 1);
    __shared__ CamS s_cam[GEVO_MAX_VIEWS];
    __shared__ float s_dxi[GEVO_MAX_VIEWS][kDxiCopies][3];
    const int total = list_count ? (int)*list_count : t_end;
    if (t_begin + (int)(blockIdx.x * blockDim.x) >= total) return;   // whole block: before any barrier
    load_cams(L, cams, s_cam);
    for (int i = threadIdx.x; i < L.n_views * kDxiCopies * 3; i += blockDim.x) (&s_dxi[0][0][0])[i] = 0.f;
    __syncthreads();
    const int t = t_begin + blockIdx.x * blockDim.x + threadIdx.x;
    const int g = t < total ? (list ? (int)list[t] : t) : n;
    if (g < n) {
        const float mu[3] = {means[3 * g], means[3 * g + 1], means[3 * g + 2]};
        float k[16][3];
        load_colour<DEG, false>(coef, g, k);
        float dk[16][3];
#pragma unroll
        for (int i = 0; i < 16; i++) dk[i][0] = dk[i][1] = dk[i][2] = 0.f;
        float dmu[3] = {0.f, 0.f, 0.f};
        unsigned long long vis = vmask ? vmask[t] : visible_views(L, n, g, radius);
        while (vis) {
            const int v = __ffsll((long long)vis) - 1;
            vis &= vis - 1;
            const CamS& cam = s_cam[v];
            const float4 grz = g_rz[(size_t)v * n + g];
            const float ux = mu[0] - cam.c[0], uy = mu[1] - cam.c[1], uz = mu[2] - cam.c[2];
            const float inl = rsqrtf(ux * ux + uy * uy + uz * uz);
            const float dx = ux * inl, dy = uy * inl, dz = uz * inl;
            float Y[16];
            sh_eval<DEG>(dx, dy, dz, Y);
            float gm[3];
            const float gin[3] = {grz.x, grz.y, grz.z};
#pragma unroll
            for (int ch = 0; ch < 3; ch++) {
                float acc = 0.5f;
#pragma unroll
                for (int i = 0; i < K; i++) acc += Y[i] * k[i][ch];
                gm[ch] = acc < 0.f ? 0.f : gin[ch];
            }
            float w[16];
#pragma unroll
            for (int i = 0; i < K; i++) {
                dk[i][0] += gm[0] * Y[i]; dk[i][1] += gm[1] * Y[i]; dk[i][2] += gm[2] * Y[i];
                w[i] = gm[0] * k[i][0] + gm[1] * k[i][1] + gm[2] * k[i][2];
            }
            if (DEG > 0) {
                float gx, gy, gz;
                sh_grad_dir<DEG>(dx, dy, dz, w, gx, gy, gz);
                const float dd = dx * gx + dy * gy + dz * gz;
                const float ex = (gx - dx * dd) * inl, ey = (gy - dy * dd) * inl, ez = (gz - dz * dd) * inl;
                dmu[0] += ex; dmu[1] += ey; dmu[2] += ez;
                if (dxi) {
                    // camera centre c = -R^T (t + rho): dL/drho = -R dL/dc = R (dL/d(mu - c))
#pragma unroll
                    for (int i = 0; i < 3; i++)
                        atomicAdd(&s_dxi[v][threadIdx.x % kDxiCopies][i], cam.R[3 * i] * ex + cam.R[3 * i + 1] * ey +
                                                    cam.R[3 * i + 2] * ez);
                }
            }
        }
        d_means[3 * g] = dmu[0]; d_means[3 * g + 1] = dmu[1]; d_means[3 * g + 2] = dmu[2];
        if ((K * 3) % 4 == 0) {
            float4* p = reinterpret_cast<float4*>(d_coef + (size_t)g * K * 3);
            float tmp[K * 3];
#pragma unroll
            for (int i = 0; i < K; i++) { tmp[3 * i] = dk[i][0]; tmp[3 * i + 1] = dk[i][1]; tmp[3 * i + 2] = dk[i][2]; }
#pragma unroll
            for (int i = 0; i < K * 3 / 4; i++)
                p[i] = make_float4(tmp[4 * i], tmp[4 * i + 1], tmp[4 * i + 2], tmp[4 * i + 3]);
        } else {
#pragma unroll
            for (int i = 0; i < K; i++)
#pragma unroll
                for (int ch = 0; ch < 3; ch++) d_coef[((size_t)g * K + i) * 3 + ch] = dk[i][ch];
        }
    }
    if (dxi) {
        __syncthreads();
        for (int v = threadIdx.x; v < L.n_views; v += blockDim.x)
            for (int i = 0; i < 3; i++) {
                float r = 0.f;
#pragma unroll
                for (int c = 0; c < kDxiCopies; c++) r += s_dxi[v][c][i];
                if (r != 0.f) atomicAdd(dxi + 6 * v + i, r);
            }
    }
}

template <int DEG, bool RGB>
static void launch_fwd(const gevo_layout& L, const gevo_gaussians& g, const gevo_camera* cams,
                       const gevo_proj& o, int part, int g_begin, int g_end, uint32_t* err,
                       cudaStream_t st, const gevo_grad2d* zero = nullptr)
{
    float2* z_xy = zero ? reinterpret_cast<float2*>(zero->xy) : nullptr;
    float4* z_co = zero ? reinterpret_cast<float4*>(zero->conic_opacity) : nullptr;
    float4* z_rz = zero ? reinterpret_cast<float4*>(zero->rgb_depth) : nullptr;
    const int threads = 128;
    const int blocks = (g_end - g_begin + threads - 1) / threads;
    if (blocks == 0) return;
    const float* coef = RGB ? g.rgb : g.sh;
    if (part == GEVO_PART_ALL)
        k_project_fwd<DEG, RGB, true><<<blocks, threads, 0, st>>>(
            L, g.n, g.means, g.scales, reinterpret_cast<const float4*>(g.quats), g.opacities, coef,
            cams, reinterpret_cast<float2*>(o.xy), reinterpret_cast<float4*>(o.conic_opacity),
            reinterpret_cast<float4*>(o.rgb_depth), o.radius, o.tiles_touched, err, g_begin, g_end,
            z_xy, z_co, z_rz);
    else if (part == GEVO_PART_GEOMETRY)
        k_project_fwd<0, true, false><<<blocks, threads, 0, st>>>(
            L, g.n, g.means, g.scales, reinterpret_cast<const float4*>(g.quats), g.opacities,
            nullptr, cams, reinterpret_cast<float2*>(o.xy),
            reinterpret_cast<float4*>(o.conic_opacity), reinterpret_cast<float4*>(o.rgb_depth),
            o.radius, o.tiles_touched, err, g_begin, g_end, z_xy, z_co, z_rz);
    else
        k_project_colour<DEG, RGB><<<blocks, threads, 0, st>>>(
            L, g.n, g.means, coef, cams, o.radius, reinterpret_cast<float4*>(o.rgb_depth), g_begin,
            g_end);
}

// SH colour kernel first (it writes the means' gradient, the geometry kernel
// adds to it), then the geometry kernel; part selects one of the two.
template <int DEG, bool RGB>
static void launch_bwd(const gevo_layout& L, const gevo_gaussians& g, const gevo_camera* cams,
                       const gevo_proj& o, const gevo_grad2d& gr, const gevo_gaussian_grads& out,
                       float* dxi, int part, int t_begin, int t_end, cudaStream_t st,
                       const uint32_t* list, const uint32_t* list_count,
                       const unsigned long long* vmask)
{
    const int threads = 128;
    const int blocks = (t_end - t_begin + threads - 1) / threads;
    if (blocks == 0) return;
    if (!RGB && part != GEVO_PART_GEOMETRY)
        k_project_bwd_col<DEG><<<blocks, threads, 0, st>>>(
            L, g.n, g.means, g.sh, cams, o.radius, reinterpret_cast<const float4*>(gr.rgb_depth),
            out.means, out.sh, dxi, list, list_count, vmask, t_begin, t_end);
    if (part == GEVO_PART_COLOUR) return;
    const auto geo = RGB ? k_project_bwd_geo<true, false> : k_project_bwd_geo<false, true>;
    geo<<<blocks, threads, 0, st>>>(
        L, g.n, g.means, g.scales, reinterpret_cast<const float4*>(g.quats), cams, o.radius,
        reinterpret_cast<const float2*>(gr.xy), reinterpret_cast<const float4*>(gr.conic_opacity),
        reinterpret_cast<const float4*>(gr.rgb_depth), out.means, out.scales,
        reinterpret_cast<float4*>(out.quats), out.opacities, out.rgb, dxi, list, list_count,
        vmask, t_begin, t_end);
}

static bool valid_gaussians(const gevo_gaussians* g)
{
    if (!g || g->n < 0 || !g->means || !g->scales || !g->quats || !g->opacities) return false;
    if ((g->sh == nullptr) == (g->rgb == nullptr)) return false;
    if (g->sh && (g->sh_degree < 0 || g->sh_degree > 3)) return false;
    if (!gevo_aligned(g->quats, 16)) return false;
    if (g->sh && (g->sh_degree == 1 || g->sh_degree == 3) && !gevo_aligned(g->sh, 16)) return false;
    return true;
}

static bool valid_proj(const gevo_proj* p)
{
    return p && p->xy && p->conic_opacity && p->rgb_depth && p->radius && p->tiles_touched &&
           gevo_aligned(p->xy, 8) && gevo_aligned(p->conic_opacity, 16) &&
           gevo_aligned(p->rgb_depth, 16);
}

}  // namespace gevo

using namespace gevo;

static gevo_status project_fwd(const gevo_layout* layout, const gevo_gaussians* g,
                               const gevo_camera* cams, gevo_proj* out, int32_t part,
                               int32_t g_begin, int32_t g_end, void* workspace, void* stream,
                               const gevo_grad2d* zero)
{
    if (!layout || !gevo::layout_valid(*layout) || !valid_gaussians(g) || !cams || !valid_proj(out) ||
        !workspace || !gevo_aligned(workspace, 256) || part < GEVO_PART_ALL ||
        part > GEVO_PART_COLOUR || g_begin < 0 || g_begin > g_end || g_end > g->n)
        return GEVO_ERR_INVALID;
    if (zero && (part == GEVO_PART_COLOUR || !zero->xy || !zero->conic_opacity ||
                 !zero->rgb_depth || !gevo_aligned(zero->xy, 8) ||
                 !gevo_aligned(zero->conic_opacity, 16) || !gevo_aligned(zero->rgb_depth, 16)))
        return GEVO_ERR_INVALID;
    if (g_begin == g_end) return GEVO_OK;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* err = reinterpret_cast<uint32_t*>(workspace);
    if (g->rgb) {
        launch_fwd<0, true>(*layout, *g, cams, *out, part, g_begin, g_end, err, st, zero);
    } else {
        switch (g->sh_degree) {
        case 0: launch_fwd<0, false>(*layout, *g, cams, *out, part, g_begin, g_end, err, st, zero); break;
        case 1: launch_fwd<1, false>(*layout, *g, cams, *out, part, g_begin, g_end, err, st, zero); break;
        case 2: launch_fwd<2, false>(*layout, *g, cams, *out, part, g_begin, g_end, err, st, zero); break;
        default: launch_fwd<3, false>(*layout, *g, cams, *out, part, g_begin, g_end, err, st, zero); break;
        }
    }
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}

extern "C" gevo_status gevo_project_part(const gevo_layout* layout, const gevo_gaussians* g,
                                         const gevo_camera* cams, gevo_proj* out, int32_t part,
                                         int32_t g_begin, int32_t g_end, void* workspace,
                                         void* stream)
{
    return project_fwd(layout, g, cams, out, part, g_begin, g_end, workspace, stream, nullptr);
}

extern "C" gevo_status gevo_project_zero(const gevo_layout* layout, const gevo_gaussians* g,
                                         const gevo_camera* cams, gevo_proj* out,
                                         gevo_grad2d* grad2d, int32_t part, int32_t g_begin,
                                         int32_t g_end, void* workspace, void* stream)
{
    if (!grad2d) return GEVO_ERR_INVALID;
    return project_fwd(layout, g, cams, out, part, g_begin, g_end, workspace, stream, grad2d);
}

extern "C" gevo_status gevo_project(const gevo_layout* layout, const gevo_gaussians* g,
                                    const gevo_camera* cams, gevo_proj* out, void* workspace,
                                    void* stream)
{
    return gevo_project_part(layout, g, cams, out, GEVO_PART_ALL, 0, g ? g->n : 0, workspace,
                             stream);
}

static gevo_status project_bwd(const gevo_layout* layout, const gevo_gaussians* g,
                               const gevo_camera* cams, const gevo_proj* proj,
                               const gevo_grad2d* grad2d, gevo_gaussian_grads* out, float* dxi,
                               void* workspace, void* stream, const uint32_t* list,
                               const uint32_t* list_count, int part = GEVO_PART_ALL,
                               int t_begin = 0, int t_end = -1)
{
    if (part < GEVO_PART_ALL || part > GEVO_PART_COLOUR) return GEVO_ERR_INVALID;
    if (g && t_end < 0) t_end = g->n;
    // a range of the whole map: whole ranges of the walk order
    if (!g || t_begin < 0 || t_begin > t_end || t_end > g->n || t_begin % kPbwdRange != 0 ||
        (t_end % kPbwdRange != 0 && t_end != g->n) || (list && (t_begin != 0 || t_end != g->n)))
        return GEVO_ERR_INVALID;
    if (!layout || !gevo::layout_valid(*layout) || !valid_gaussians(g) || !cams || !proj || !proj->radius ||
        !grad2d || !grad2d->xy || !grad2d->conic_opacity || !grad2d->rgb_depth || !out ||
        !out->means || !out->scales || !out->quats || !out->opacities || !workspace ||
        !gevo_aligned(workspace, 256))
        return GEVO_ERR_INVALID;
    if ((g->sh != nullptr) != (out->sh != nullptr) || (g->rgb != nullptr) != (out->rgb != nullptr))
        return GEVO_ERR_INVALID;
    if (!gevo_aligned(out->quats, 16) || !gevo_aligned(grad2d->conic_opacity, 16) ||
        !gevo_aligned(grad2d->rgb_depth, 16) || !gevo_aligned(grad2d->xy, 8))
        return GEVO_ERR_INVALID;
    if (out->sh && (g->sh_degree == 1 || g->sh_degree == 3) && !gevo_aligned(out->sh, 16))
        return GEVO_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    // the colour part of the range starting at 0 (alone, or first of the two)
    // starts the pose twist at zero and builds the walk order
    const bool first = part != GEVO_PART_GEOMETRY && t_begin == 0;
    if (dxi && first &&
        cudaMemsetAsync(dxi, 0, sizeof(float) * 6 * layout->n_views, st) != cudaSuccess)
        return GEVO_ERR_CUDA;
    if (g->n == 0) return GEVO_OK;
    const gevo_layout& L = *layout;
    const unsigned long long* vmask = nullptr;
    if (!list) {   // the whole map: walk it in the stored order (built by the first part)
        const WsLayout w = ws_layout(L, g->n, 0);
        char* ws = reinterpret_cast<char*>(workspace);
        uint32_t* perm = reinterpret_cast<uint32_t*>(ws + w.pb_perm);
        auto* vm = reinterpret_cast<unsigned long long*>(ws + w.pb_mask);
        if (first) {
            k_pbwd_order<<<(g->n + kPbwdRange - 1) / kPbwdRange, kPbwdRange, 0, st>>>(
                L, g->n, proj->radius, perm, vm);
            GEVO_CHECK_LAUNCH();
        }
        list = perm;
        vmask = vm;
    }
    if (g->rgb) {
        launch_bwd<0, true>(L, *g, cams, *proj, *grad2d, *out, dxi, part, t_begin, t_end, st, list, list_count, vmask);
    } else {
        switch (g->sh_degree) {
        case 0: launch_bwd<0, false>(L, *g, cams, *proj, *grad2d, *out, dxi, part, t_begin, t_end, st, list, list_count, vmask); break;
        case 1: launch_bwd<1, false>(L, *g, cams, *proj, *grad2d, *out, dxi, part, t_begin, t_end, st, list, list_count, vmask); break;
        case 2: launch_bwd<2, false>(L, *g, cams, *proj, *grad2d, *out, dxi, part, t_begin, t_end, st, list, list_count, vmask); break;
        default: launch_bwd<3, false>(L, *g, cams, *proj, *grad2d, *out, dxi, part, t_begin, t_end, st, list, list_count, vmask); break;
        }
    }
    GEVO_CHECK_LAUNCH();
    return GEVO_OK;
}

extern "C" gevo_status gevo_project_bwd(const gevo_layout* layout, const gevo_gaussians* g,
                                        const gevo_camera* cams, const gevo_proj* proj,
                                        const gevo_grad2d* grad2d, gevo_gaussian_grads* out,
                                        float* dxi, void* workspace, void* stream)
{
    return project_bwd(layout, g, cams, proj, grad2d, out, dxi, workspace, stream, nullptr, nullptr);
}

extern "C" gevo_status gevo_project_bwd_part(const gevo_layout* layout, const gevo_gaussians* g,
                                             const gevo_camera* cams, const gevo_proj* proj,
                                             const gevo_grad2d* grad2d, gevo_gaussian_grads* out,
                                             float* dxi, int32_t part, int32_t g_begin,
                                             int32_t g_end, void* workspace, void* stream)
{
    return project_bwd(layout, g, cams, proj, grad2d, out, dxi, workspace, stream, nullptr, nullptr,
                       part, g_begin, g_end);
}

extern "C" gevo_status gevo_project_bwd_active(const gevo_layout* layout, const gevo_gaussians* g,
                                               const gevo_camera* cams, const gevo_proj* proj,
                                               const gevo_grad2d* grad2d,
                                               const uint32_t* active_list, const uint32_t* counts,
                                               gevo_gaussian_grads* out, float* dxi,
                                               void* workspace, void* stream)
{
    if (!active_list || !counts) return GEVO_ERR_INVALID;
    return project_bwd(layout, g, cams, proj, grad2d, out, dxi, workspace, stream, active_list,
                       counts);
}
