/*
 * gevo_oracle.c -- plain FP64 CPU oracle of the differentiable Gaussian-splatting
 * rasterizer R(M, T) that GEVO renders with (Section I, "GS" of the 3DGS paper it
 * cites; Section III-B, Eq. 2 and Eq. 3 optimise the map and the pose T_k through
 * it; Eq. 6 renders past keyframes with it instead of storing them).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  It shares no code, header,
 * table or constant with the CUDA library; the library never loads it.
 *
 * The paper defines the renderer only by citation, so every step below is the
 * plain definition of the 3DGS forward model (projection, binning, blending) and
 * its exact derivative, written out literally:
 *   - everything is double precision, except the tile binning, which is defined
 *     in binary32 on the binary32 projection outputs (reading R7 of the design
 *     notes) so that tile lists and sort keys can be compared bit for bit;
 *   - the per-tile lists are built by brute force and sorted with qsort on the
 *     (tile, depth bit pattern, id) tuple -- no radix sort, no scan;
 *   - each pixel walks its tile list one entry at a time;
 *   - the backward pass keeps every blended entry of a pixel in a small array and
 *     applies the chain rule entry by entry (no division to recover T).
 * Compile with -ffp-contract=off so that the binary32 binning rounds exactly as
 * written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Constants of the 3DGS formulation (readings R2-R9). */
#define ORC_NEAR_Z      0.2          /* cull if camera depth <= 0.2 m            */
#define ORC_DILATION    0.3          /* px^2 low-pass added to the 2-D covariance */
#define ORC_GUARD       1.3          /* EWA Jacobian guard band (x/z clamp)        */
#define ORC_ALPHA_MAX   0.99         /* alpha clamp                                */
#define ORC_ALPHA_MIN   (1.0 / 255.0)/* skip below                                 */
#define ORC_T_STOP      1e-4         /* stop before T falls below                  */
#define ORC_TILE        16           /* 16 x 16 pixel tiles                        */

/* Camera block: c[0..8] world->camera rotation (row-major), c[9..11] translation,
 * c[12..15] = fx, fy, cx, cy. */

/* ------------------------------------------------------------------------ */
/* Real spherical-harmonic basis up to degree 3 (the basis 3DGS colours with), */
/* constants from their closed forms.                                         */
/* ------------------------------------------------------------------------ */
static void sh_consts(double C[16])
{
    const double pi = 3.14159265358979323846;
    C[0] = 0.5 * sqrt(1.0 / pi);
    C[1] = -sqrt(3.0 / (4.0 * pi));  /* times y */
    C[2] = sqrt(3.0 / (4.0 * pi));   /* times z */
    C[3] = -sqrt(3.0 / (4.0 * pi));  /* times x */
    C[4] = 0.5 * sqrt(15.0 / pi);    /* xy */
    C[5] = -0.5 * sqrt(15.0 / pi);   /* yz */
    C[6] = 0.25 * sqrt(5.0 / pi);    /* 2z^2 - x^2 - y^2 */
    C[7] = -0.5 * sqrt(15.0 / pi);   /* xz */
    C[8] = 0.25 * sqrt(15.0 / pi);   /* x^2 - y^2 */
    C[9] = -0.25 * sqrt(35.0 / (2.0 * pi));  /* y(3x^2 - y^2) */
    C[10] = 0.5 * sqrt(105.0 / pi);          /* xyz */
    C[11] = -0.25 * sqrt(21.0 / (2.0 * pi)); /* y(4z^2 - x^2 - y^2) */
    C[12] = 0.25 * sqrt(7.0 / pi);           /* z(2z^2 - 3x^2 - 3y^2) */
    C[13] = -0.25 * sqrt(21.0 / (2.0 * pi)); /* x(4z^2 - x^2 - y^2) */
    C[14] = 0.25 * sqrt(105.0 / pi);         /* z(x^2 - y^2) */
    C[15] = -0.25 * sqrt(35.0 / (2.0 * pi)); /* x(x^2 - 3y^2) */
}

/* Y[k] and dY[k][0..2] = dY_k/d(x,y,z) at the (unit) direction (x,y,z). */
void orc_sh_basis(int deg, const double d[3], double Y[16], double dY[48])
{
    double C[16];
    sh_consts(C);
    const double x = d[0], y = d[1], z = d[2];
    const double xx = x * x, yy = y * y, zz = z * z;
    memset(Y, 0, 16 * sizeof(double));
    if (dY) memset(dY, 0, 48 * sizeof(double));
    Y[0] = C[0];
    if (deg < 1) return;
    Y[1] = C[1] * y; Y[2] = C[2] * z; Y[3] = C[3] * x;
    if (dY) { dY[1*3+1] = C[1]; dY[2*3+2] = C[2]; dY[3*3+0] = C[3]; }
    if (deg < 2) return;
    Y[4] = C[4] * x * y;
    Y[5] = C[5] * y * z;
    Y[6] = C[6] * (2.0 * zz - xx - yy);
    Y[7] = C[7] * x * z;
    Y[8] = C[8] * (xx - yy);
    if (dY) {
        dY[4*3+0] = C[4] * y;        dY[4*3+1] = C[4] * x;
        dY[5*3+1] = C[5] * z;        dY[5*3+2] = C[5] * y;
        dY[6*3+0] = -2.0 * C[6] * x; dY[6*3+1] = -2.0 * C[6] * y; dY[6*3+2] = 4.0 * C[6] * z;
        dY[7*3+0] = C[7] * z;        dY[7*3+2] = C[7] * x;
        dY[8*3+0] = 2.0 * C[8] * x;  dY[8*3+1] = -2.0 * C[8] * y;
    }
    if (deg < 3) return;
    Y[9]  = C[9]  * y * (3.0 * xx - yy);
    Y[10] = C[10] * x * y * z;
    Y[11] = C[11] * y * (4.0 * zz - xx - yy);
    Y[12] = C[12] * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
    Y[13] = C[13] * x * (4.0 * zz - xx - yy);
    Y[14] = C[14] * z * (xx - yy);
    Y[15] = C[15] * x * (xx - 3.0 * yy);
    if (dY) {
        dY[9*3+0] = C[9] * 6.0 * x * y;          dY[9*3+1] = C[9] * (3.0 * xx - 3.0 * yy);
        dY[10*3+0] = C[10] * y * z; dY[10*3+1] = C[10] * x * z; dY[10*3+2] = C[10] * x * y;
        dY[11*3+0] = C[11] * (-2.0 * x * y);
        dY[11*3+1] = C[11] * (4.0 * zz - xx - 3.0 * yy);
        dY[11*3+2] = C[11] * 8.0 * y * z;
        dY[12*3+0] = C[12] * (-6.0 * x * z);
        dY[12*3+1] = C[12] * (-6.0 * y * z);
        dY[12*3+2] = C[12] * (6.0 * zz - 3.0 * xx - 3.0 * yy);
        dY[13*3+0] = C[13] * (4.0 * zz - 3.0 * xx - yy);
        dY[13*3+1] = C[13] * (-2.0 * x * y);
        dY[13*3+2] = C[13] * 8.0 * x * z;
        dY[14*3+0] = C[14] * 2.0 * x * z; dY[14*3+1] = C[14] * (-2.0 * y * z);
        dY[14*3+2] = C[14] * (xx - yy);
        dY[15*3+0] = C[15] * (3.0 * xx - 3.0 * yy); dY[15*3+1] = C[15] * (-6.0 * x * y);
    }
}

/* ------------------------------------------------------------------------ */
/* Quaternion (w, x, y, z), normalised, to a rotation matrix, and the four    */
/* partial derivatives dR/dw, dR/dx, dR/dy, dR/dz (row-major 3x3 each).       */
/* ------------------------------------------------------------------------ */
static void quat_to_rot(const double qn[4], double R[9], double dR[4][9])
{
    const double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
    if (!dR) return;
    const double dw[9] = {0, -2*z, 2*y,  2*z, 0, -2*x,  -2*y, 2*x, 0};
    const double dx[9] = {0, 2*y, 2*z,  2*y, -4*x, -2*w,  2*z, 2*w, -4*x};
    const double dy[9] = {-4*y, 2*x, 2*w,  2*x, 0, 2*z,  -2*w, 2*z, -4*y};
    const double dz[9] = {-4*z, -2*w, 2*x,  2*w, -4*z, 2*y,  2*x, 2*y, 0};
    memcpy(dR[0], dw, sizeof dw); memcpy(dR[1], dx, sizeof dx);
    memcpy(dR[2], dy, sizeof dy); memcpy(dR[3], dz, sizeof dz);
}

/* Sigma3 = Rq diag(s)^2 Rq^T (row-major 3x3). */
void orc_cov3d(const double s[3], const double q[4], double S3[9])
{
    double nq = sqrt(q[0]*q[0] + q[1]*q[1] + q[2]*q[2] + q[3]*q[3]);
    double qn[4] = {q[0]/nq, q[1]/nq, q[2]/nq, q[3]/nq};
    double R[9];
    quat_to_rot(qn, R, NULL);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += R[i*3+k] * s[k] * s[k] * R[j*3+k];
            S3[i*3+j] = acc;
        }
}

/* Tile rectangle of one projected Gaussian, in binary32 as the binning step
 * defines it: [xmin, xmax) x [ymin, ymax) in tiles, clamped to the grid. */
static void rect_f32(float mx, float my, int32_t r, int32_t tiles_x, int32_t tiles_y, int32_t out[4])
{
    float rf = (float)r;
    float v[4];
    v[0] = floorf((mx - rf) / 16.0f);
    v[1] = floorf((my - rf) / 16.0f);
    v[2] = floorf(((mx + rf) + 15.0f) / 16.0f);
    v[3] = floorf(((my + rf) + 15.0f) / 16.0f);
    float lim[4] = {(float)tiles_x, (float)tiles_y, (float)tiles_x, (float)tiles_y};
    for (int k = 0; k < 4; k++) {
        float c = v[k] < 0.0f ? 0.0f : v[k];
        c = c > lim[k] ? lim[k] : c;
        out[k] = (int32_t)c;
    }
}

void orc_rect_f32(float mx, float my, int32_t r, int32_t tiles_x, int32_t tiles_y, int32_t* out)
{
    rect_f32(mx, my, r, tiles_x, tiles_y, out);
}

static int near_int(double v, double tol) { return fabs(v - floor(v + 0.5)) <= tol; }

/* ------------------------------------------------------------------------ */
/* Step 1: projection of one view (per Gaussian).                            */
/* ------------------------------------------------------------------------ */
/* Outputs (per Gaussian g):
 *   xy[2]      pixel-space mean (x = fx*X/Z + cx - 0.5; pixel i is sampled at i)
 *   conic[3]   (a, b, c) of the inverse 2-D covariance
 *   cov2d[3]   the 2-D covariance (after the 0.3 px^2 dilation)
 *   depth      camera-frame Z
 *   radius     ceil(3 sqrt(lambda_max)); 0 = culled
 *   rgb[3]     colour (given, or from SH with the max(0, .) clamp)
 *   clamped[3] 1 where the SH colour was clamped at 0
 *   fragile    1 when a discrete decision (near plane, guard band, radius ceil,
 *              tile-rect floor) lies within a small margin of its threshold, so a
 *              binary32 evaluation may legitimately decide the other way. */
void orc_project(int32_t n, const double* mean, const double* scale, const double* quat,
                 const double* opac, const double* sh, int32_t sh_deg, const double* rgb_in,
                 const double* cam, int32_t W, int32_t H,
                 double* xy, double* conic, double* cov2d, double* depth, int32_t* radius,
                 double* rgb, int32_t* clamped, int32_t* tiles_touched, int32_t* fragile)
{
    (void)opac;
    const double* Rw = cam;
    const double* tw = cam + 9;
    const double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    const int32_t tiles_x = (W + ORC_TILE - 1) / ORC_TILE, tiles_y = (H + ORC_TILE - 1) / ORC_TILE;
    const double limx = ORC_GUARD * (0.5 * W) / fx, limy = ORC_GUARD * (0.5 * H) / fy;
    /* camera centre c = -R^T t */
    double cc[3];
    for (int i = 0; i < 3; i++) cc[i] = -(Rw[0*3+i] * tw[0] + Rw[1*3+i] * tw[1] + Rw[2*3+i] * tw[2]);
    const int ncoef = (sh_deg + 1) * (sh_deg + 1);

    for (int32_t g = 0; g < n; g++) {
        radius[g] = 0; tiles_touched[g] = 0; fragile[g] = 0;
        xy[2*g] = xy[2*g+1] = 0.0; conic[3*g] = conic[3*g+1] = conic[3*g+2] = 0.0;
        cov2d[3*g] = cov2d[3*g+1] = cov2d[3*g+2] = 0.0; depth[g] = 0.0;
        rgb[3*g] = rgb[3*g+1] = rgb[3*g+2] = 0.0;
        clamped[3*g] = clamped[3*g+1] = clamped[3*g+2] = 0;

        const double* mu = mean + 3*g;
        double p[3];
        for (int i = 0; i < 3; i++) p[i] = Rw[i*3] * mu[0] + Rw[i*3+1] * mu[1] + Rw[i*3+2] * mu[2] + tw[i];
        depth[g] = p[2];
        if (fabs(p[2] - ORC_NEAR_Z) <= 1e-5) fragile[g] = 1;
        if (p[2] <= ORC_NEAR_Z) continue;

        double S3[9];
        orc_cov3d(scale + 3*g, quat + 4*g, S3);

        const double z = p[2];
        double txz = p[0] / z, tyz = p[1] / z;
        if (fabs(fabs(txz) - limx) <= 1e-6 * limx || fabs(fabs(tyz) - limy) <= 1e-6 * limy) fragile[g] = 1;
        if (txz > limx) txz = limx;
        if (txz < -limx) txz = -limx;
        if (tyz > limy) tyz = limy;
        if (tyz < -limy) tyz = -limy;
        double J[6] = { fx / z, 0.0, -fx * txz / z,
                        0.0, fy / z, -fy * tyz / z };
        double M[6]; /* M = J W, 2x3 */
        for (int r = 0; r < 2; r++)
            for (int i = 0; i < 3; i++)
                M[r*3+i] = J[r*3+0] * Rw[0*3+i] + J[r*3+1] * Rw[1*3+i] + J[r*3+2] * Rw[2*3+i];
        double S2[4] = {0, 0, 0, 0};
        for (int r = 0; r < 2; r++)
            for (int c2 = 0; c2 < 2; c2++) {
                double acc = 0.0;
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) acc += M[r*3+i] * S3[i*3+j] * M[c2*3+j];
                S2[r*2+c2] = acc;
            }
        const double a = S2[0] + ORC_DILATION, b = S2[1], c = S2[3] + ORC_DILATION;
        cov2d[3*g] = a; cov2d[3*g+1] = b; cov2d[3*g+2] = c;
        const double det = a * c - b * b;
        if (det <= 0.0) continue;
        conic[3*g] = c / det; conic[3*g+1] = -b / det; conic[3*g+2] = a / det;
        const double mid = 0.5 * (a + c);
        double disc = mid * mid - det;
        if (disc < 0.1) disc = 0.1;
        const double lmax = mid + sqrt(disc);
        const double r3 = 3.0 * sqrt(lmax);
        if (near_int(r3, 1e-4 * (r3 > 1.0 ? r3 : 1.0))) fragile[g] = 1;
        const int32_t r = (int32_t)ceil(r3);
        xy[2*g] = fx * p[0] / z + cx - 0.5;
        xy[2*g+1] = fy * p[1] / z + cy - 0.5;

        /* binning rectangle (binary32 definition) */
        int32_t rc[4];
        rect_f32((float)xy[2*g], (float)xy[2*g+1], r, tiles_x, tiles_y, rc);
        for (int k = 0; k < 2; k++) {
            double m = xy[2*g+k];
            if (near_int((m - r) / 16.0, 1e-3 / 16.0) || near_int((m + r + 15.0) / 16.0, 1e-3 / 16.0))
                fragile[g] = 1;
        }
        const int32_t area = (rc[2] - rc[0]) * (rc[3] - rc[1]);
        if (area == 0) continue;

        /* colour */
        if (rgb_in) {
            for (int ch = 0; ch < 3; ch++) rgb[3*g+ch] = rgb_in[3*g+ch];
        } else {
            double d[3] = {mu[0] - cc[0], mu[1] - cc[1], mu[2] - cc[2]};
            double nd = sqrt(d[0]*d[0] + d[1]*d[1] + d[2]*d[2]);
            d[0] /= nd; d[1] /= nd; d[2] /= nd;
            double Y[16];
            orc_sh_basis(sh_deg, d, Y, NULL);
            for (int ch = 0; ch < 3; ch++) {
                double v = 0.5;
                for (int k = 0; k < ncoef; k++) v += Y[k] * sh[((size_t)g * ncoef + k) * 3 + ch];
                if (fabs(v) <= 1e-6) fragile[g] = 1;
                if (v < 0.0) { clamped[3*g+ch] = 1; v = 0.0; }
                rgb[3*g+ch] = v;
            }
        }
        radius[g] = r;
        tiles_touched[g] = area;
    }
}

/* ------------------------------------------------------------------------ */
/* Steps 2-4: duplicate keys, sort, per-tile ranges (brute force).            */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t key; uint32_t val; } orc_pair;

static int cmp_pair(const void* A, const void* B)
{
    const orc_pair* a = (const orc_pair*)A;
    const orc_pair* b = (const orc_pair*)B;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->val != b->val) return a->val < b->val ? -1 : 1;
    return 0;
}

/* n_views views, n Gaussians, inputs [view][n].  Tiles are numbered view-major:
 * global tile = (tiles of all earlier views) + ty * tiles_x + tx.  The key is
 * (global tile << 32) | bit pattern of the binary32 depth; equal keys are ordered
 * by Gaussian id.  ranges[2*t] / [2*t+1] = [start, end) of tile t, (0, 0) when the
 * tile is empty.  Returns the true duplicate count D; if D > capacity, keys and
 * vals are left untouched and every range is (0, 0). */
int64_t orc_bin_f32(int32_t n_views, const int32_t* W, const int32_t* H, int32_t n,
                    const float* xy, const int32_t* radius, const float* depth,
                    int64_t capacity, uint64_t* keys, uint32_t* vals, uint32_t* ranges,
                    int32_t* tiles_touched)
{
    int64_t total_tiles = 0;
    for (int v = 0; v < n_views; v++)
        total_tiles += (int64_t)((W[v] + 15) / 16) * ((H[v] + 15) / 16);
    int64_t D = 0;
    int64_t tile_base = 0;
    for (int v = 0; v < n_views; v++) {
        int32_t tx = (W[v] + 15) / 16, ty = (H[v] + 15) / 16;
        for (int32_t g = 0; g < n; g++) {
            size_t i = (size_t)v * n + g;
            tiles_touched[i] = 0;
            if (radius[i] <= 0) continue;
            int32_t rc[4];
            rect_f32(xy[2*i], xy[2*i+1], radius[i], tx, ty, rc);
            tiles_touched[i] = (rc[2] - rc[0]) * (rc[3] - rc[1]);
            D += tiles_touched[i];
        }
        tile_base += (int64_t)tx * ty;
    }
    memset(ranges, 0, sizeof(uint32_t) * 2 * (size_t)total_tiles);
    if (D > capacity || D == 0) return D;

    orc_pair* P = (orc_pair*)malloc(sizeof(orc_pair) * (size_t)D);
    int64_t k = 0;
    tile_base = 0;
    for (int v = 0; v < n_views; v++) {
        int32_t tx = (W[v] + 15) / 16, ty = (H[v] + 15) / 16;
        for (int32_t g = 0; g < n; g++) {
            size_t i = (size_t)v * n + g;
            if (radius[i] <= 0) continue;
            int32_t rc[4];
            rect_f32(xy[2*i], xy[2*i+1], radius[i], tx, ty, rc);
            uint32_t dbits;
            memcpy(&dbits, &depth[i], 4);
            for (int32_t y = rc[1]; y < rc[3]; y++)
                for (int32_t x = rc[0]; x < rc[2]; x++) {
                    uint64_t tile = (uint64_t)(tile_base + (int64_t)y * tx + x);
                    P[k].key = (tile << 32) | (uint64_t)dbits;
                    P[k].val = (uint32_t)g;
                    k++;
                }
        }
        tile_base += (int64_t)tx * ty;
    }
    qsort(P, (size_t)D, sizeof(orc_pair), cmp_pair);
    for (int64_t i = 0; i < D; i++) {
        keys[i] = P[i].key;
        vals[i] = P[i].val;
        uint64_t t = P[i].key >> 32;
        if (i == 0 || (P[i-1].key >> 32) != t) ranges[2*t] = (uint32_t)i;
        if (i == D - 1 || (P[i+1].key >> 32) != t) ranges[2*t+1] = (uint32_t)(i + 1);
    }
    free(P);
    return D;
}

/* ------------------------------------------------------------------------ */
/* Step 5: front-to-back blending of one view.                                */
/* ------------------------------------------------------------------------ */
/* Per pixel (px, py) of the view, walk the list of its tile:
 *   power = -1/2 (a dx^2 + c dy^2) - b dx dy,  d = mean2D - pixel
 *   skip if power > 0; alpha = min(0.99, o exp(power)); skip if alpha < 1/255;
 *   stop (without blending) if T (1 - alpha) < 1e-4;
 *   C += alpha T c;  D += alpha T z;  T *= 1 - alpha.
 * Final C += T bg.  n_contrib = 1 + list position of the last blended entry.
 * n_eval = entries examined (including skips and the stopping entry).
 * wsum = sum of blend weights (for the partition-of-unity check).
 * fragile = 1 where some examined entry lies within a small margin of one of the
 * thresholds (power sign, alpha clamp, alpha skip, T stop).
 * sig = a hash of the event set (which entries blend, clamp, where it stops).
 * ranges: this view's tiles ([tiles][2], positions into vals). */
static uint64_t mix64(uint64_t h, uint64_t v)
{
    h ^= v + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2);
    h *= 0xbf58476d1ce4e5b9ULL;
    return h ^ (h >> 31);
}

void orc_render_fwd(int32_t W, int32_t H, const double* xy, const double* conic, const double* opac,
                    const double* rgb, const double* depth,
                    const uint32_t* vals, const uint32_t* ranges, const double* bg,
                    double* out_rgb, double* out_depth, double* out_T, int32_t* n_contrib,
                    int32_t* n_eval, double* wsum, int32_t* fragile, uint64_t* sig,
                    const double* pix_err, double* gauss_err,
                    const uint8_t* active, int32_t* act_last, double* act_T, double* act_rest,
                    int32_t* n_blend)
{
    /* pix_err / gauss_err (both NULL or both set): the per-Gaussian rendering
     * error of Section III-B2 (Eq. 5), E(g) += w(g, u) e(u) summed over the
     * pixels u, w(g, u) the blending weight alpha T of g at u and e(u) the
     * per-pixel error; gauss_err is indexed by Gaussian id.
     * active (NULL or one byte per Gaussian) with act_last / act_T / act_rest:
     * per pixel, 1 + the list position of the last blended entry of an active
     * Gaussian (0 if none), the transmittance right after it (1 if none), and
     * the colour (3 channels, plus T_final bg) and depth blended behind it
     * (act_rest[4 * pix + c]; 0 if none). */
    const int32_t tiles_x = (W + ORC_TILE - 1) / ORC_TILE;
    const size_t P = (size_t)W * H;
    for (int32_t py = 0; py < H; py++)
        for (int32_t px = 0; px < W; px++) {
            const size_t pix = (size_t)py * W + px;
            const int32_t tile = (py / ORC_TILE) * tiles_x + (px / ORC_TILE);
            const uint32_t s = ranges[2*tile], e = ranges[2*tile+1];
            double T = 1.0, C[3] = {0, 0, 0}, Dd = 0.0, ws = 0.0;
            int32_t last = 0, ne = 0, frag = 0, la = 0, nbl = 0;
            double Ta = 1.0, Ca[3] = {0, 0, 0}, Da = 0.0;   /* colour, depth through the last active entry */
            uint64_t h = 0x1234567ULL;
            for (uint32_t i = s; i < e; i++) {
                const uint32_t g = vals[i];
                ne++;
                const double dx = xy[2*g] - px, dy = xy[2*g+1] - py;
                const double a = conic[3*g], b = conic[3*g+1], c = conic[3*g+2];
                const double power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
                const double mag = 0.5 * (fabs(a) * dx * dx + fabs(c) * dy * dy) + fabs(b * dx * dy);
                if (fabs(power) <= 1e-5 * mag + 1e-12) frag = 1;
                if (power > 0.0) continue;
                const double og = opac[g] * exp(power);
                if (fabs(og - ORC_ALPHA_MAX) <= 1e-4 * ORC_ALPHA_MAX) frag = 1;
                const double alpha = og < ORC_ALPHA_MAX ? og : ORC_ALPHA_MAX;
                if (fabs(alpha - ORC_ALPHA_MIN) <= 1e-4 * ORC_ALPHA_MIN) frag = 1;
                if (alpha < ORC_ALPHA_MIN) continue;
                const double Tn = T * (1.0 - alpha);
                if (fabs(Tn - ORC_T_STOP) <= 1e-3 * ORC_T_STOP) frag = 1;
                if (Tn < ORC_T_STOP) { h = mix64(h, 0xFFFFFFFF00000000ULL | (i - s)); break; }
                const double w = alpha * T;
                if (gauss_err) gauss_err[g] += w * pix_err[pix];
                for (int ch = 0; ch < 3; ch++) C[ch] += w * rgb[3*g+ch];
                Dd += w * depth[g];
                ws += w;
                T = Tn;
                last = (int32_t)(i - s + 1);
                nbl++;
                if (active && active[g]) {
                    la = last;
                    Ta = T;
                    for (int ch = 0; ch < 3; ch++) Ca[ch] = C[ch];
                    Da = Dd;
                }
                h = mix64(h, ((uint64_t)(og > ORC_ALPHA_MAX) << 40) | ((uint64_t)g << 8) | 1u);
            }
            for (int ch = 0; ch < 3; ch++) out_rgb[ch * P + pix] = C[ch] + T * bg[ch];
            out_depth[pix] = Dd;
            out_T[pix] = T;
            n_contrib[pix] = last;
            if (n_eval) n_eval[pix] = ne;
            if (n_blend) n_blend[pix] = nbl;
            if (wsum) wsum[pix] = ws;
            if (fragile) fragile[pix] = frag;
            if (sig) sig[pix] = mix64(h, (uint64_t)last);
            if (active) {
                /* what lies behind the last active entry: the whole colour
                 * minus what was blended up to it (exact in the reals; the
                 * CUDA path sums the part behind on its own) */
                act_last[pix] = la;
                act_T[pix] = la ? Ta : 1.0;
                for (int ch = 0; ch < 3; ch++)
                    act_rest[4 * pix + ch] = la ? (C[ch] - Ca[ch]) + T * bg[ch] : 0.0;
                act_rest[4 * pix + 3] = la ? Dd - Da : 0.0;
            }
        }
}

/* ------------------------------------------------------------------------ */
/* Step 6: exact derivative of step 5 for one view.                          */
/* ------------------------------------------------------------------------ */
/* Accumulates (+=) per Gaussian: g_xy[2], g_conic[3] (w.r.t. a, b, c as they
 * appear in power), g_opac, g_rgb[3], g_depth.  dL_dT may be NULL.
 * Derivation, per pixel with blended entries i = 0..m-1 (weights w_i = alpha_i T_i):
 *   dC/dc_i = w_i,  dD/dz_i = w_i,
 *   dC/dalpha_i = T_i (c_i - S_i),  S_i = colour seen behind i per unit of T_{i+1}
 *                 (S_{m-1} = bg; S_{i-1} = alpha_i c_i + (1 - alpha_i) S_i),
 *   dD/dalpha_i = T_i (z_i - S^D_i)  (same recursion with bg = 0),
 *   dT_final/dalpha_i = -T_final / (1 - alpha_i).
 * alpha = o exp(power) below the clamp (no gradient where clamped). */
typedef struct { uint32_t g; double alpha, T, G, dx, dy; int clamped; } orc_blend;

void orc_render_bwd(int32_t W, int32_t H, const double* xy, const double* conic, const double* opac,
                    const double* rgb, const double* depth,
                    const uint32_t* vals, const uint32_t* ranges, const double* bg,
                    const double* dL_drgb, const double* dL_ddepth, const double* dL_dT,
                    double* g_xy, double* g_conic, double* g_opac, double* g_rgb, double* g_depth)
{
    const int32_t tiles_x = (W + ORC_TILE - 1) / ORC_TILE;
    const size_t P = (size_t)W * H;
    size_t cap = 64;
    orc_blend* L = (orc_blend*)malloc(sizeof(orc_blend) * cap);
    for (int32_t py = 0; py < H; py++)
        for (int32_t px = 0; px < W; px++) {
            const size_t pix = (size_t)py * W + px;
            const int32_t tile = (py / ORC_TILE) * tiles_x + (px / ORC_TILE);
            const uint32_t s = ranges[2*tile], e = ranges[2*tile+1];
            /* forward again, keeping the blended entries */
            size_t m = 0;
            double T = 1.0;
            for (uint32_t i = s; i < e; i++) {
                const uint32_t g = vals[i];
                const double dx = xy[2*g] - px, dy = xy[2*g+1] - py;
                const double a = conic[3*g], b = conic[3*g+1], c = conic[3*g+2];
                const double power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
                if (power > 0.0) continue;
                const double G = exp(power);
                const double og = opac[g] * G;
                const double alpha = og < ORC_ALPHA_MAX ? og : ORC_ALPHA_MAX;
                if (alpha < ORC_ALPHA_MIN) continue;
                const double Tn = T * (1.0 - alpha);
                if (Tn < ORC_T_STOP) break;
                if (m == cap) { cap *= 2; L = (orc_blend*)realloc(L, sizeof(orc_blend) * cap); }
                L[m].g = g; L[m].alpha = alpha; L[m].T = T; L[m].G = G;
                L[m].dx = dx; L[m].dy = dy; L[m].clamped = og > ORC_ALPHA_MAX;
                m++;
                T = Tn;
            }
            const double Tf = T;
            const double gC[3] = {dL_drgb[pix], dL_drgb[P + pix], dL_drgb[2*P + pix]};
            const double gD = dL_ddepth ? dL_ddepth[pix] : 0.0;
            const double gT = dL_dT ? dL_dT[pix] : 0.0;
            double S[3] = {bg[0], bg[1], bg[2]}, SD = 0.0;
            for (size_t k = m; k-- > 0;) {
                const orc_blend* B = &L[k];
                const uint32_t g = B->g;
                const double w = B->alpha * B->T;
                double dLda = 0.0;
                for (int ch = 0; ch < 3; ch++) {
                    g_rgb[3*g+ch] += gC[ch] * w;
                    dLda += gC[ch] * B->T * (rgb[3*g+ch] - S[ch]);
                }
                g_depth[g] += gD * w;
                dLda += gD * B->T * (depth[g] - SD);
                dLda += gT * (-Tf / (1.0 - B->alpha));
                for (int ch = 0; ch < 3; ch++) S[ch] = B->alpha * rgb[3*g+ch] + (1.0 - B->alpha) * S[ch];
                SD = B->alpha * depth[g] + (1.0 - B->alpha) * SD;
                if (B->clamped) continue;
                g_opac[g] += dLda * B->G;
                const double dLdp = dLda * B->alpha;          /* d alpha / d power = alpha */
                const double a = conic[3*g], b = conic[3*g+1], c = conic[3*g+2];
                g_conic[3*g]   += dLdp * (-0.5 * B->dx * B->dx);
                g_conic[3*g+1] += dLdp * (-B->dx * B->dy);
                g_conic[3*g+2] += dLdp * (-0.5 * B->dy * B->dy);
                g_xy[2*g]   += dLdp * (-(a * B->dx + b * B->dy));
                g_xy[2*g+1] += dLdp * (-(b * B->dx + c * B->dy));
            }
        }
    free(L);
}

/* ------------------------------------------------------------------------ */
/* Step 7: exact derivative of step 1 for one view, including the camera      */
/* pose.  Accumulates (+=).  The pose gradient is w.r.t. a left perturbation   */
/* xi = (rho, phi) of the world->camera transform, T <- Exp(xi) T, at xi = 0    */
/* (reading R10): p_c -> p_c + phi x p_c + rho, W -> (I + [phi]x) W,            */
/* camera centre -> c - R^T rho.                                               */
/* ------------------------------------------------------------------------ */
void orc_project_bwd(int32_t n, const double* mean, const double* scale, const double* quat,
                     const double* opac, const double* sh, int32_t sh_deg, const double* rgb_in,
                     const double* cam, int32_t W, int32_t H, const int32_t* radius,
                     const double* g_xy, const double* g_conic, const double* g_opac,
                     const double* g_rgb, const double* g_depth,
                     double* d_mean, double* d_scale, double* d_quat, double* d_opac,
                     double* d_sh, double* d_rgb, double* d_xi)
{
    (void)opac;
    const double* Rw = cam;
    const double* tw = cam + 9;
    const double fx = cam[12], fy = cam[13];
    const double limx = ORC_GUARD * (0.5 * W) / fx, limy = ORC_GUARD * (0.5 * H) / fy;
    double cc[3];
    for (int i = 0; i < 3; i++) cc[i] = -(Rw[0*3+i] * tw[0] + Rw[1*3+i] * tw[1] + Rw[2*3+i] * tw[2]);
    const int ncoef = (sh_deg + 1) * (sh_deg + 1);

    for (int32_t g = 0; g < n; g++) {
        if (radius[g] <= 0) continue;
        const double* mu = mean + 3*g;
        const double* s = scale + 3*g;
        const double* q = quat + 4*g;
        double p[3];
        for (int i = 0; i < 3; i++) p[i] = Rw[i*3] * mu[0] + Rw[i*3+1] * mu[1] + Rw[i*3+2] * mu[2] + tw[i];
        const double z = p[2];
        double dLdp[3] = {0, 0, 0};   /* gradient w.r.t. the camera-frame mean */
        double dLdW[9];               /* gradient w.r.t. W through the covariance path */
        memset(dLdW, 0, sizeof dLdW);
        double dLdmu[3] = {0, 0, 0};
        double dLdcc[3] = {0, 0, 0};  /* gradient w.r.t. the camera centre */

        d_opac[g] += g_opac[g];

        /* --- mean2D and depth --- */
        dLdp[0] += g_xy[2*g] * fx / z;
        dLdp[1] += g_xy[2*g+1] * fy / z;
        dLdp[2] += g_xy[2*g] * (-fx * p[0] / (z * z)) + g_xy[2*g+1] * (-fy * p[1] / (z * z));
        dLdp[2] += g_depth[g];

        /* --- covariance path --- */
        double nq = sqrt(q[0]*q[0] + q[1]*q[1] + q[2]*q[2] + q[3]*q[3]);
        double qn[4] = {q[0]/nq, q[1]/nq, q[2]/nq, q[3]/nq};
        double Rq[9], dRq[4][9];
        quat_to_rot(qn, Rq, dRq);
        double S3[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double acc = 0.0;
                for (int k = 0; k < 3; k++) acc += Rq[i*3+k] * s[k] * s[k] * Rq[j*3+k];
                S3[i*3+j] = acc;
            }
        double txz = p[0] / z, tyz = p[1] / z;
        const int clx = (txz > limx) || (txz < -limx);
        const int cly = (tyz > limy) || (tyz < -limy);
        if (txz > limx) txz = limx;
        if (txz < -limx) txz = -limx;
        if (tyz > limy) tyz = limy;
        if (tyz < -limy) tyz = -limy;
        double J[6] = { fx / z, 0.0, -fx * txz / z,  0.0, fy / z, -fy * tyz / z };
        double M[6];
        for (int r = 0; r < 2; r++)
            for (int i = 0; i < 3; i++)
                M[r*3+i] = J[r*3+0] * Rw[0*3+i] + J[r*3+1] * Rw[1*3+i] + J[r*3+2] * Rw[2*3+i];
        double S2[4] = {0, 0, 0, 0};
        for (int r = 0; r < 2; r++)
            for (int c2 = 0; c2 < 2; c2++) {
                double acc = 0.0;
                for (int i = 0; i < 3; i++)
                    for (int j = 0; j < 3; j++) acc += M[r*3+i] * S3[i*3+j] * M[c2*3+j];
                S2[r*2+c2] = acc;
            }
        const double a = S2[0] + ORC_DILATION, b = S2[1], c = S2[3] + ORC_DILATION;
        const double Dt = a * c - b * b, D2 = Dt * Dt;
        /* conic (ca, cb, cc) = (c, -b, a) / Dt; partials w.r.t. (a, b, c) */
        const double gA = g_conic[3*g], gB = g_conic[3*g+1], gC = g_conic[3*g+2];
        const double dca_da = -c * c / D2, dca_db = 2.0 * b * c / D2, dca_dc = 1.0 / Dt - c * a / D2;
        const double dcb_da = b * c / D2, dcb_db = -1.0 / Dt - 2.0 * b * b / D2, dcb_dc = b * a / D2;
        const double dcc_da = 1.0 / Dt - a * c / D2, dcc_db = 2.0 * a * b / D2, dcc_dc = -a * a / D2;
        const double dLda = gA * dca_da + gB * dcb_da + gC * dcc_da;
        const double dLdb = gA * dca_db + gB * dcb_db + gC * dcc_db;
        const double dLdc = gA * dca_dc + gB * dcb_dc + gC * dcc_dc;
        /* a = M0 S3 M0^T + 0.3, b = M0 S3 M1^T, c = M1 S3 M1^T + 0.3 */
        double S3M0[3], S3M1[3];
        for (int i = 0; i < 3; i++) {
            S3M0[i] = S3[i*3] * M[0] + S3[i*3+1] * M[1] + S3[i*3+2] * M[2];
            S3M1[i] = S3[i*3] * M[3] + S3[i*3+1] * M[4] + S3[i*3+2] * M[5];
        }
        double dLdM[6];
        for (int i = 0; i < 3; i++) {
            dLdM[i]     = 2.0 * dLda * S3M0[i] + dLdb * S3M1[i];
            dLdM[3 + i] = dLdb * S3M0[i] + 2.0 * dLdc * S3M1[i];
        }
        double dLdS3[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++)
                dLdS3[i*3+j] = dLda * M[i] * M[j] + dLdb * M[i] * M[3+j] + dLdc * M[3+i] * M[3+j];
        /* M = J W */
        double dLdJ[6];
        for (int r = 0; r < 2; r++)
            for (int k = 0; k < 3; k++) {
                double acc = 0.0;
                for (int i = 0; i < 3; i++) acc += dLdM[r*3+i] * Rw[k*3+i];
                dLdJ[r*3+k] = acc;
            }
        for (int k = 0; k < 3; k++)
            for (int i = 0; i < 3; i++)
                dLdW[k*3+i] += J[0*3+k] * dLdM[0*3+i] + J[1*3+k] * dLdM[1*3+i];
        /* J entries as functions of p */
        dLdp[2] += dLdJ[0] * (-fx / (z * z)) + dLdJ[4] * (-fy / (z * z));
        if (!clx) {
            dLdp[0] += dLdJ[2] * (-fx / (z * z));
            dLdp[2] += dLdJ[2] * (2.0 * fx * p[0] / (z * z * z));
        } else {
            dLdp[2] += dLdJ[2] * (fx * txz / (z * z));
        }
        if (!cly) {
            dLdp[1] += dLdJ[5] * (-fy / (z * z));
            dLdp[2] += dLdJ[5] * (2.0 * fy * p[1] / (z * z * z));
        } else {
            dLdp[2] += dLdJ[5] * (fy * tyz / (z * z));
        }
        /* Sigma3 = Rq diag(s^2) Rq^T */
        for (int k = 0; k < 3; k++) {
            double acc = 0.0;
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) acc += dLdS3[i*3+j] * 2.0 * s[k] * Rq[i*3+k] * Rq[j*3+k];
            d_scale[3*g+k] += acc;
        }
        double dLdRq[9];
        for (int i = 0; i < 3; i++)
            for (int k = 0; k < 3; k++) {
                double acc = 0.0;
                for (int j = 0; j < 3; j++) acc += (dLdS3[i*3+j] + dLdS3[j*3+i]) * s[k] * s[k] * Rq[j*3+k];
                dLdRq[i*3+k] = acc;
            }
        double dLdqn[4];
        for (int u = 0; u < 4; u++) {
            double acc = 0.0;
            for (int e = 0; e < 9; e++) acc += dLdRq[e] * dRq[u][e];
            dLdqn[u] = acc;
        }
        double dot = 0.0;
        for (int u = 0; u < 4; u++) dot += qn[u] * dLdqn[u];
        for (int u = 0; u < 4; u++) d_quat[4*g+u] += (dLdqn[u] - qn[u] * dot) / nq;

        /* --- colour --- */
        if (rgb_in) {
            for (int ch = 0; ch < 3; ch++) d_rgb[3*g+ch] += g_rgb[3*g+ch];
        } else {
            double dr[3] = {mu[0] - cc[0], mu[1] - cc[1], mu[2] - cc[2]};
            double nd = sqrt(dr[0]*dr[0] + dr[1]*dr[1] + dr[2]*dr[2]);
            double d[3] = {dr[0]/nd, dr[1]/nd, dr[2]/nd};
            double Y[16], dY[48];
            orc_sh_basis(sh_deg, d, Y, dY);
            double gm[3];
            for (int ch = 0; ch < 3; ch++) {
                double v = 0.5;
                for (int k = 0; k < ncoef; k++) v += Y[k] * sh[((size_t)g * ncoef + k) * 3 + ch];
                gm[ch] = v < 0.0 ? 0.0 : g_rgb[3*g+ch];
            }
            double dLdd[3] = {0, 0, 0};
            for (int k = 0; k < ncoef; k++)
                for (int ch = 0; ch < 3; ch++) {
                    d_sh[((size_t)g * ncoef + k) * 3 + ch] += gm[ch] * Y[k];
                    for (int u = 0; u < 3; u++)
                        dLdd[u] += gm[ch] * sh[((size_t)g * ncoef + k) * 3 + ch] * dY[k*3+u];
                }
            double dd = d[0]*dLdd[0] + d[1]*dLdd[1] + d[2]*dLdd[2];
            for (int u = 0; u < 3; u++) {
                double gr = (dLdd[u] - d[u] * dd) / nd;  /* w.r.t. mu - c */
                dLdmu[u] += gr;
                dLdcc[u] -= gr;
            }
        }

        /* --- camera-frame mean to world mean --- */
        for (int j = 0; j < 3; j++)
            dLdmu[j] += Rw[0*3+j] * dLdp[0] + Rw[1*3+j] * dLdp[1] + Rw[2*3+j] * dLdp[2];
        for (int j = 0; j < 3; j++) d_mean[3*g+j] += dLdmu[j];

        if (d_xi) {
            /* rho: p_c += rho; camera centre c -= R^T rho */
            for (int i = 0; i < 3; i++) {
                double fromc = Rw[i*3] * dLdcc[0] + Rw[i*3+1] * dLdcc[1] + Rw[i*3+2] * dLdcc[2];
                d_xi[i] += dLdp[i] - fromc;
            }
            /* phi: p_c += phi x p_c  ->  p_c x dL/dp_c */
            d_xi[3] += p[1] * dLdp[2] - p[2] * dLdp[1];
            d_xi[4] += p[2] * dLdp[0] - p[0] * dLdp[2];
            d_xi[5] += p[0] * dLdp[1] - p[1] * dLdp[0];
            /* phi: W -> (I + [phi]x) W ; B = dL/dW W^T */
            double B[9];
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; k++) acc += dLdW[i*3+k] * Rw[j*3+k];
                    B[i*3+j] = acc;
                }
            d_xi[3] += B[2*3+1] - B[1*3+2];
            d_xi[4] += B[0*3+2] - B[2*3+0];
            d_xi[5] += B[1*3+0] - B[0*3+1];
        }
    }
}
