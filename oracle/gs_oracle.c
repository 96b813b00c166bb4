/*
 * gs_oracle.c -- plain, slow FP64 CPU oracle of the differentiable 3D Gaussian
 * splatting mapping step: projection, binning, front-to-back compositing, the
 * photometric loss, the analytic backward, Adam and the lifecycle scores.
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this library; the product path never does.  It shares
 * no code with the CUDA sources.
 *
 * What the paper fixes, and where:
 *   - compositing of sorted Gaussians along the ray with the transmittance
 *     T_j = prod_{m<j} (1 - alpha_m)  (Supp. D.2, depth volume rendering);
 *   - L_photo = 0.8 ||I - I^||_1 + 0.2 (1 - SSIM(I, I^))  (Supp. D.4);
 *   - the error mask M_v, kappa_v and S_d  (Supp. E.1), gamma_v, the
 *     log transform and min-max normalisation of S_p  (Supp. E.2), the OR
 *     and max aggregation over chunks  (Sec. 3.3.2), tau_err = 0.1,
 *     tau_d = 5, tau_p = 0.99  (Supp. F).
 * What the paper leaves open is taken as the standard EWA splatting of the
 * cited 3D Gaussian splatting work, written here from the mathematics:
 *   R1 camera: x_c = R x_w + t, x right, y down, z forward; u = fx x/z + cx;
 *      pixel (i, j) samples (i + 0.5, j + 0.5).
 *   R2 cull z <= near (0.2), empty tile rectangles and opacity below alpha_min
 *      (FP32 logit below the FP32 logit of alpha_min: such a Gaussian never blends).
 *   R3 Sigma = R(q) S S^T R(q)^T, S = diag(exp(log_scale)); EWA
 *      Sigma' = J W Sigma W^T J^T + 0.3 I with J evaluated at x/z, y/z clamped
 *      to 1.3 tan(fov/2); the clamp has zero derivative on the clamped side.
 *   R4 radius = ceil(3 sqrt(lambda_max)), lambda_max = mid + sqrt(max(0.1, mid^2 - det)).
 *   R5 tile rectangle = the tiles overlapped by [u - r, u + r] x [v - r, v + r]:
 *      xmin = floor((u - r)/tw), xmax = floor((u + r)/tw) + 1, clamped to the grid.
 *   R6 colour = max(0, sum_k sh_k Y_k(dir) + 0.5), dir = normalise(mean - camera centre),
 *      real spherical harmonics with the Condon-Shortley phase.
 *   R7 pairs ordered by (tile, depth, Gaussian index).
 *   R8 per pixel: power = -(a dx^2 + c dy^2)/2 - b dx dy (skip if > 0);
 *      alpha = min(0.99, o e^power); skip alpha < 1/255; stop before blending
 *      when T (1 - alpha) < 1e-4; C += c alpha T; T *= (1 - alpha); C += T bg.
 *   R9 SSIM: 11x11 Gaussian window, sigma 1.5, zero padding, C1 = 0.01^2,
 *      C2 = 0.03^2, mean over channels and pixels.
 *   R10 Adam (Kingma & Ba) with bias correction, dense over all parameters.
 *   R11 Omega_v(i) = pixels where Gaussian i is blended under R8.
 *   R12 ||.||_1 in M_v sums the three colour channels.
 *   R13 S_p is 0 for Gaussians with empty footprint in the chunk and for a
 *       chunk whose active scores are all equal.
 * Probabilistic initialisation (Sec. 3.3.1: DoG, normalised depth gradient,
 * P, P_kf, 3x3 NMS, voxel quantisation; Supp. D.5: dynamic map expansion
 * through a voxel hash; Supp. F: lambda = 0.9, m = 5 levels) reads:
 *   R19 DoG on Y = (R + G + B) / 3 taken in 8-bit intensity units (255 Y;
 *       on [0, 1] intensities the clamp at 1 could never act: the DoG of a
 *       unit step peaks near 0.11); G_s sampled on integer offsets within
 *       ceil(3 s), normalised to sum 1; replicated borders; s1 = 1, s2 = 1.6.
 *   R20 ||grad D|| by central differences in depth units per pixel with
 *       replicated borders; min-max over the keyframe, a flat map gives 0.
 *   R21 P^ is the same formula applied to the rendered I^, D^ (own
 *       min-max); the first keyframe has P^ = 0.
 *   R22 selection: (P_kf, -raster index) is the lexicographic maximum of
 *       the 3x3 window, P_kf > 0, a caller's uniform draw U < P_kf (the
 *       paper samples from P_kf and names no sampler), depth > near (0.2).
 *   R23 level = first l with ||x_c|| < max_dist_l (10, 25, 100, 500, inf m);
 *       voxel sizes (0.1, 0.25, 1, 5, 25), the printed third size 0.1 read
 *       as 1 (the printed sequence is otherwise increasing).
 *   R24 voxel idx = floor(x / eps_l), anchor p = idx eps_l (the paper's
 *       formula); one anchor per (l, idx); new anchors numbered in raster
 *       order of the first pixel reaching their voxel.
 * Scaffold-GS anchors (Supp. D.1 decoding, Supp. D.3 LoD mask) read:
 *   R25 one decoder for the K = 10 Gaussians of an anchor: input (f, dir,
 *       log(1 + d)) (32 + 3 + 1), hidden layer of 64 with ReLU, 14 K linear
 *       outputs, per Gaussian (colour 3, opacity 1, rotation 4, scale 3,
 *       offset 3).
 *   R26 colour = sigmoid, opacity = tanh (Gaussians with opacity <= 0 are
 *       dropped, as in Scaffold-GS), rotation = (1, 0, 0, 0) + output
 *       (normalised by the rasteriser), scale factor = sigmoid, offset raw.
 *   R27 mu = p + (O_k + dO_k) * l, s = l * ds_k (l = exp of the stored
 *       log-scale), opacity masked by the LoD band of the anchor's level:
 *       [max_dist[l-1], max_dist[l]) (0 below the first level, R23 bands).
 *   R28 decoded Gaussians enter the rasteriser as SH-degree-0 Gaussians:
 *       sh0 = (c - 1/2) / Y00, opacity logit = log(a / (1 - a)); dropped ones
 *       get logit -30 and are culled (R2).
 *   R29 anchor positions stay fixed; f, the log-scale, the offsets and the
 *       decoder's weights are optimised.
 * Parity pins for each function are in the tests; every function below is
 * pinned (closed forms, brute force, library routines, finite differences).
 */
#include "gs_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics, from the associated-Legendre definition          */
/* ------------------------------------------------------------------------ */

#define OR_MAX_SH_DEG 8

static double factorial(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return f;
}

/* Coefficients of the Legendre polynomial P_l(z) (Bonnet recursion). */
static void legendre_coeffs(int l, double *c /* l+1 entries, c[k] of z^k */) {
    double p0[OR_MAX_SH_DEG + 2] = {0}, p1[OR_MAX_SH_DEG + 2] = {0}, p2[OR_MAX_SH_DEG + 2];
    p0[0] = 1.0;            /* P_0 = 1 */
    p1[1] = 1.0;            /* P_1 = z */
    if (l == 0) { c[0] = 1.0; return; }
    for (int n = 1; n < l; ++n) {
        /* (n+1) P_{n+1} = (2n+1) z P_n - n P_{n-1} */
        for (int k = 0; k <= n + 1; ++k) {
            double zp = (k >= 1) ? p1[k - 1] : 0.0;
            p2[k] = ((2.0 * n + 1.0) * zp - n * p0[k]) / (n + 1.0);
        }
        memcpy(p0, p1, sizeof(p0));
        memcpy(p1, p2, sizeof(p1));
    }
    for (int k = 0; k <= l; ++k) c[k] = p1[k];
}

/* Value at z of the d-th derivative of the polynomial with coefficients c[0..l]. */
static double poly_deriv_eval(const double *c, int l, int d, double z) {
    double s = 0.0;
    for (int k = l; k >= d; --k) {
        double fk = 1.0;
        for (int j = 0; j < d; ++j) fk *= (double)(k - j);
        s = s * z + c[k] * fk;
    }
    /* Horner above multiplies by z once per step from k=l down to k=d; the
       highest surviving power is z^(l-d). */
    return s;
}

void or_sh_eval(int32_t D, const double d[3], double *Y, double *dY) {
    const double x = d[0], y = d[1], z = d[2];
    /* A_m + i B_m = (x + i y)^m */
    double A[OR_MAX_SH_DEG + 1], B[OR_MAX_SH_DEG + 1];
    A[0] = 1.0; B[0] = 0.0;
    for (int m = 1; m <= D; ++m) {
        A[m] = x * A[m - 1] - y * B[m - 1];
        B[m] = x * B[m - 1] + y * A[m - 1];
    }
    for (int l = 0; l <= D; ++l) {
        double c[OR_MAX_SH_DEG + 1];
        legendre_coeffs(l, c);
        for (int m = 0; m <= l; ++m) {
            double K = sqrt((2.0 * l + 1.0) / (4.0 * OR_PI) * factorial(l - m) / factorial(l + m));
            double Pm = poly_deriv_eval(c, l, m, z);          /* d^m P_l / dz^m */
            double Pm1 = (m + 1 <= l) ? poly_deriv_eval(c, l, m + 1, z) : 0.0;
            if (m == 0) {
                int k = l * l + l;
                Y[k] = K * Pm;
                if (dY) { dY[3 * k + 0] = 0.0; dY[3 * k + 1] = 0.0; dY[3 * k + 2] = K * Pm1; }
            } else {
                double s = sqrt(2.0) * K * ((m & 1) ? -1.0 : 1.0);
                int kp = l * l + l + m, kn = l * l + l - m;
                Y[kp] = s * Pm * A[m];
                Y[kn] = s * Pm * B[m];
                if (dY) {
                    /* d(x+iy)^m/dx = m (x+iy)^(m-1); d/dy = i m (x+iy)^(m-1) */
                    dY[3 * kp + 0] = s * Pm * (m * A[m - 1]);
                    dY[3 * kp + 1] = s * Pm * (-m * B[m - 1]);
                    dY[3 * kp + 2] = s * Pm1 * A[m];
                    dY[3 * kn + 0] = s * Pm * (m * B[m - 1]);
                    dY[3 * kn + 1] = s * Pm * (m * A[m - 1]);
                    dY[3 * kn + 2] = s * Pm1 * B[m];
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Rotations                                                                  */
/* ------------------------------------------------------------------------ */

static void quat_rot_unit(double w, double x, double y, double z, double R[9]) {
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

void or_quat_to_rot(const double q[4], double R[9]) {
    double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    quat_rot_unit(q[0] / nq, q[1] / nq, q[2] / nq, q[3] / nq, R);
}

/* Partial derivatives of the nine entries of R with respect to (w, x, y, z). */
static void quat_rot_partials(double w, double x, double y, double z, double dR[4][9]) {
    const double dw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    const double dx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    const double dy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    const double dz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    memcpy(dR[0], dw, sizeof(dw));
    memcpy(dR[1], dx, sizeof(dx));
    memcpy(dR[2], dy, sizeof(dy));
    memcpy(dR[3], dz, sizeof(dz));
}

/* ------------------------------------------------------------------------ */
/* Projection                                                                 */
/* ------------------------------------------------------------------------ */

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static int32_t sh_coeffs(int32_t D) { return (D + 1) * (D + 1); }

/* Camera centre in world coordinates: c = -R^T t. */
static void camera_centre(const or_camera *cam, double c[3]) {
    for (int k = 0; k < 3; ++k)
        c[k] = -(cam->R[0 * 3 + k] * cam->t[0] + cam->R[1 * 3 + k] * cam->t[1] + cam->R[2 * 3 + k] * cam->t[2]);
}

void or_project(const or_params *p, const or_camera *cam, const or_cfg *cfg, or_projected *out) {
    const int64_t n = p->n;
    const int32_t D = p->sh_degree, K = sh_coeffs(D);
    const int GW = (cam->width + cfg->tile_w - 1) / cfg->tile_w;
    const int GH = (cam->height + cfg->tile_h - 1) / cfg->tile_h;
    double cc[3];
    camera_centre(cam, cc);

#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const double *mu = p->means + 3 * i;
        out->radius[i] = 0;
        out->tiles_touched[i] = 0;
        for (int k = 0; k < 4; ++k) out->rect[4 * i + k] = 0;

        /* FP32 evaluation order of the camera-frame point and pixel position:
           every product, sum and quotient rounds to float, left to right. */
        float mf[3] = {(float)mu[0], (float)mu[1], (float)mu[2]};
        float Rf[9], tf[3];
        for (int k = 0; k < 9; ++k) Rf[k] = (float)cam->R[k];
        for (int k = 0; k < 3; ++k) tf[k] = (float)cam->t[k];
        float xc32 = Rf[0] * mf[0] + Rf[1] * mf[1] + Rf[2] * mf[2] + tf[0];
        float yc32 = Rf[3] * mf[0] + Rf[4] * mf[1] + Rf[5] * mf[2] + tf[1];
        float zc32 = Rf[6] * mf[0] + Rf[7] * mf[1] + Rf[8] * mf[2] + tf[2];
        float u32 = ((float)cam->fx * xc32) / zc32 + (float)cam->cx;
        float v32 = ((float)cam->fy * yc32) / zc32 + (float)cam->cy;
        out->u32[i] = u32; out->v32[i] = v32; out->z32[i] = zc32;

        /* FP64 camera-frame point */
        double pc[3];
        for (int r = 0; r < 3; ++r)
            pc[r] = cam->R[3 * r + 0] * mu[0] + cam->R[3 * r + 1] * mu[1] + cam->R[3 * r + 2] * mu[2] + cam->t[r];
        const double x = pc[0], y = pc[1], z = pc[2];

        int culled = cfg->fp32_positions ? (zc32 <= (float)cfg->near_z) : (z <= cfg->near_z);
        /* R2: a Gaussian whose opacity is below alpha_min can never blend under R8; the
           test is on the FP32 logit against the FP32 logit of alpha_min */
        {
            const double am = (double)(float)cfg->alpha_min;  /* the device receives alpha_min in FP32 */
            culled |= (float)p->opacity_logits[i] < (float)log(am / (1.0 - am));
        }
        if (culled) continue;

        /* 3D covariance */
        double Rq[9];
        or_quat_to_rot(p->quats + 4 * i, Rq);
        double s[3];
        for (int k = 0; k < 3; ++k) s[k] = exp(p->log_scales[3 * i + k]);
        double M[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) M[3 * r + c] = Rq[3 * r + c] * s[c];
        double Sig[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += M[3 * r + k] * M[3 * c + k];
                Sig[3 * r + c] = acc;
            }

        /* EWA */
        const double limx = cfg->tan_clamp * cam->width / (2.0 * cam->fx);
        const double limy = cfg->tan_clamp * cam->height / (2.0 * cam->fy);
        double rx = x / z, ry = y / z;
        double tx = z * (rx < -limx ? -limx : (rx > limx ? limx : rx));
        double ty = z * (ry < -limy ? -limy : (ry > limy ? limy : ry));
        double J[6] = {cam->fx / z, 0.0, -cam->fx * tx / (z * z),
                       0.0, cam->fy / z, -cam->fy * ty / (z * z)};
        double T[6];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c)
                T[3 * r + c] = J[3 * r + 0] * cam->R[0 * 3 + c] + J[3 * r + 1] * cam->R[1 * 3 + c] +
                               J[3 * r + 2] * cam->R[2 * 3 + c];
        double cov[3] = {0, 0, 0}; /* A = S'00, B = S'01, C = S'11 */
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) {
                cov[0] += T[k] * Sig[3 * k + l] * T[l];
                cov[1] += T[k] * Sig[3 * k + l] * T[3 + l];
                cov[2] += T[3 + k] * Sig[3 * k + l] * T[3 + l];
            }
        cov[0] += cfg->dilation;
        cov[2] += cfg->dilation;
        double det = cov[0] * cov[2] - cov[1] * cov[1];
        if (!(det > 0.0)) continue;
        out->cov2d[3 * i + 0] = cov[0];
        out->cov2d[3 * i + 1] = cov[1];
        out->cov2d[3 * i + 2] = cov[2];
        out->conic[3 * i + 0] = cov[2] / det;
        out->conic[3 * i + 1] = -cov[1] / det;
        out->conic[3 * i + 2] = cov[0] / det;

        double mid = 0.5 * (cov[0] + cov[2]);
        double disc = mid * mid - det;
        double lam = mid + sqrt(disc > 0.1 ? disc : 0.1);
        double rex = 3.0 * sqrt(lam);
        int radius = (int)ceil(rex);
        out->radius_exact[i] = rex;

        double u64 = cam->fx * x / z + cam->cx;
        double v64 = cam->fy * y / z + cam->cy;
        int xmin, xmax, ymin, ymax;
        if (cfg->fp32_positions) {
            float rf = (float)radius;
            float twf = (float)cfg->tile_w, thf = (float)cfg->tile_h;
            float fxmin = floorf((u32 - rf) / twf), fxmax = floorf((u32 + rf) / twf) + 1.0f;
            float fymin = floorf((v32 - rf) / thf), fymax = floorf((v32 + rf) / thf) + 1.0f;
            fxmin = fminf(fmaxf(fxmin, 0.0f), (float)GW); fxmax = fminf(fmaxf(fxmax, 0.0f), (float)GW);
            fymin = fminf(fmaxf(fymin, 0.0f), (float)GH); fymax = fminf(fmaxf(fymax, 0.0f), (float)GH);
            xmin = (int)fxmin; xmax = (int)fxmax; ymin = (int)fymin; ymax = (int)fymax;
            out->u[i] = (double)u32; out->v[i] = (double)v32; out->z[i] = (double)zc32;
        } else {
            double fxmin = floor((u64 - radius) / cfg->tile_w), fxmax = floor((u64 + radius) / cfg->tile_w) + 1.0;
            double fymin = floor((v64 - radius) / cfg->tile_h), fymax = floor((v64 + radius) / cfg->tile_h) + 1.0;
            xmin = (int)fmin(fmax(fxmin, 0.0), GW); xmax = (int)fmin(fmax(fxmax, 0.0), GW);
            ymin = (int)fmin(fmax(fymin, 0.0), GH); ymax = (int)fmin(fmax(fymax, 0.0), GH);
            out->u[i] = u64; out->v[i] = v64; out->z[i] = z;
        }
        xmin = clampi(xmin, 0, GW); xmax = clampi(xmax, 0, GW);
        ymin = clampi(ymin, 0, GH); ymax = clampi(ymax, 0, GH);
        int touched = (xmax - xmin) * (ymax - ymin);
        if (touched <= 0) continue;

        /* colour */
        double dir[3] = {mu[0] - cc[0], mu[1] - cc[1], mu[2] - cc[2]};
        double nd = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
        for (int k = 0; k < 3; ++k) dir[k] /= nd;
        double Y[(OR_MAX_SH_DEG + 1) * (OR_MAX_SH_DEG + 1)];
        or_sh_eval(D, dir, Y, NULL);
        for (int ch = 0; ch < 3; ++ch) {
            double c = 0.5;
            for (int k = 0; k < K; ++k) c += p->sh[(i * K + k) * 3 + ch] * Y[k];
            out->rgb_raw[3 * i + ch] = c;
            out->rgb_clamped[3 * i + ch] = c < 0.0;
            out->rgb[3 * i + ch] = c < 0.0 ? 0.0 : c;
        }
        out->opacity[i] = 1.0 / (1.0 + exp(-p->opacity_logits[i]));
        out->radius[i] = radius;
        out->rect[4 * i + 0] = xmin; out->rect[4 * i + 1] = ymin;
        out->rect[4 * i + 2] = xmax; out->rect[4 * i + 3] = ymax;
        out->tiles_touched[i] = touched;
    }
}

/* ------------------------------------------------------------------------ */
/* Binning                                                                    */
/* ------------------------------------------------------------------------ */

typedef struct { int64_t tile; double z; int64_t g; } bin_entry;

static int bin_cmp(const void *a, const void *b) {
    const bin_entry *x = (const bin_entry *)a, *y = (const bin_entry *)b;
    if (x->tile != y->tile) return x->tile < y->tile ? -1 : 1;
    if (x->z != y->z) return x->z < y->z ? -1 : 1;
    if (x->g != y->g) return x->g < y->g ? -1 : 1;
    return 0;
}

int64_t or_bin(const or_projected *pr, int64_t n, const or_camera *cam, const or_cfg *cfg,
               int64_t capacity, uint64_t *keys, int32_t *vals, int64_t *ranges) {
    const int GW = (cam->width + cfg->tile_w - 1) / cfg->tile_w;
    const int GH = (cam->height + cfg->tile_h - 1) / cfg->tile_h;
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) total += pr->radius[i] > 0 ? pr->tiles_touched[i] : 0;
    if (total > capacity || keys == NULL) return total;
    bin_entry *e = (bin_entry *)malloc(sizeof(bin_entry) * (size_t)(total > 0 ? total : 1));
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (pr->radius[i] <= 0) continue;
        const int32_t *r = pr->rect + 4 * i;
        for (int ty = r[1]; ty < r[3]; ++ty)
            for (int tx = r[0]; tx < r[2]; ++tx) {
                e[k].tile = (int64_t)ty * GW + tx;
                e[k].z = pr->z[i];
                e[k].g = i;
                ++k;
            }
    }
    qsort(e, (size_t)total, sizeof(bin_entry), bin_cmp);
    for (int64_t t = 0; t < (int64_t)GW * GH; ++t) { ranges[2 * t] = 0; ranges[2 * t + 1] = 0; }
    for (int64_t j = 0; j < total; ++j) {
        float zf = (float)e[j].z;
        uint32_t zb;
        memcpy(&zb, &zf, sizeof(zb));
        keys[j] = ((uint64_t)e[j].tile << 32) | (uint64_t)zb;
        vals[j] = (int32_t)e[j].g;
        if (j == 0 || e[j - 1].tile != e[j].tile) ranges[2 * e[j].tile] = j;
        ranges[2 * e[j].tile + 1] = j + 1;
    }
    free(e);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Compositing                                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t g, pos;
    double alpha, T, G, dx, dy;
    int clamped;
} contrib;

/* Front-to-back compositing of one pixel.  Returns the number of blended
 * Gaussians; fills buf (up to cap) with their records. */
static int64_t composite_pixel(const or_projected *pr, const int32_t *vals, int64_t start, int64_t end,
                               const or_cfg *cfg, double px, double py, contrib *buf, int64_t cap,
                               double C[3], double *Dp, double *Tout, int64_t *last, int32_t *flags) {
    double T = 1.0;
    double acc[3] = {0, 0, 0}, dacc = 0.0;
    int64_t nb = 0;
    *last = -1;
    *flags = 0;
    for (int64_t j = start; j < end; ++j) {
        int64_t g = vals[j];
        double dx = px - pr->u[g], dy = py - pr->v[g];
        const double *q = pr->conic + 3 * g;
        double power = -0.5 * (q[0] * dx * dx + q[2] * dy * dy) - q[1] * dx * dy;
        if (power > 0.0) continue;
        double G = exp(power);
        double a_raw = pr->opacity[g] * G;
        if (fabs(a_raw - cfg->alpha_min) < 1e-6) *flags |= OR_FLAG_NEAR_ALPHA_MIN;
        if (fabs(a_raw - cfg->alpha_max) < 1e-6) *flags |= OR_FLAG_NEAR_ALPHA_MAX;
        int clamped = a_raw > cfg->alpha_max;
        double alpha = clamped ? cfg->alpha_max : a_raw;
        if (alpha < cfg->alpha_min) continue;
        double Tn = T * (1.0 - alpha);
        if (fabs(Tn - cfg->t_min) < 1e-3 * cfg->t_min) *flags |= OR_FLAG_NEAR_T_CUT;
        if (Tn < cfg->t_min) break;
        for (int ch = 0; ch < 3; ++ch) acc[ch] += pr->rgb[3 * g + ch] * alpha * T;
        dacc += pr->z[g] * alpha * T;
        if (buf && nb < cap) {
            buf[nb].g = g; buf[nb].pos = j; buf[nb].alpha = alpha; buf[nb].T = T;
            buf[nb].G = G; buf[nb].dx = dx; buf[nb].dy = dy; buf[nb].clamped = clamped;
        }
        ++nb;
        *last = j;
        T = Tn;
    }
    for (int ch = 0; ch < 3; ++ch) C[ch] = acc[ch] + T * cfg->bg[ch];
    *Dp = dacc;
    *Tout = T;
    return nb;
}

void or_render(const or_projected *pr, const int32_t *vals, const int64_t *ranges,
               const or_camera *cam, const or_cfg *cfg,
               double *img, double *depth, double *T_final, int32_t *n_contrib,
               int64_t *last_pos, int32_t *flags) {
    const int W = cam->width, H = cam->height;
    const int GW = (W + cfg->tile_w - 1) / cfg->tile_w;
    const int64_t npx = (int64_t)W * H;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < npx; ++p) {
        int i = (int)(p % W), j = (int)(p / W);
        int64_t tile = (int64_t)(j / cfg->tile_h) * GW + (i / cfg->tile_w);
        double C[3], Dp, T;
        int64_t last;
        int32_t fl;
        int64_t nb = composite_pixel(pr, vals, ranges[2 * tile], ranges[2 * tile + 1], cfg,
                                     i + 0.5, j + 0.5, NULL, 0, C, &Dp, &T, &last, &fl);
        for (int ch = 0; ch < 3; ++ch) img[ch * npx + p] = C[ch];
        if (depth) depth[p] = Dp;
        if (T_final) T_final[p] = T;
        if (n_contrib) n_contrib[p] = (int32_t)nb;
        if (last_pos) last_pos[p] = last;
        if (flags) flags[p] = fl;
    }
}

/* ------------------------------------------------------------------------ */
/* Photometric loss                                                           */
/* ------------------------------------------------------------------------ */

#define SSIM_R 5
static void ssim_window(double w[2 * SSIM_R + 1]) {
    double s = 0.0;
    for (int k = -SSIM_R; k <= SSIM_R; ++k) {
        w[k + SSIM_R] = exp(-(double)(k * k) / (2.0 * 1.5 * 1.5));
        s += w[k + SSIM_R];
    }
    for (int k = 0; k < 2 * SSIM_R + 1; ++k) w[k] /= s;
}

static const double SSIM_C1 = 0.01 * 0.01, SSIM_C2 = 0.03 * 0.03;

/* Local statistics at every pixel of one channel by direct 2D windowed sums
 * with zero padding. */
static void ssim_stats(const double *x, const double *y, int H, int W, const double *w,
                       double *mx, double *my, double *sxx, double *syy, double *sxy) {
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < (int64_t)H * W; ++p) {
        int i = (int)(p % W), j = (int)(p / W);
        double a = 0, b = 0, aa = 0, bb = 0, ab = 0;
        for (int dj = -SSIM_R; dj <= SSIM_R; ++dj) {
            int jj = j + dj;
            if (jj < 0 || jj >= H) continue;
            for (int di = -SSIM_R; di <= SSIM_R; ++di) {
                int ii = i + di;
                if (ii < 0 || ii >= W) continue;
                double wt = w[dj + SSIM_R] * w[di + SSIM_R];
                double xv = x[(int64_t)jj * W + ii], yv = y[(int64_t)jj * W + ii];
                a += wt * xv; b += wt * yv; aa += wt * xv * xv; bb += wt * yv * yv; ab += wt * xv * yv;
            }
        }
        mx[p] = a; my[p] = b;
        sxx[p] = aa - a * a; syy[p] = bb - b * b; sxy[p] = ab - a * b;
    }
}

void or_ssim_map(const double *x, const double *y, int32_t C, int32_t H, int32_t W, double *map) {
    double w[2 * SSIM_R + 1];
    ssim_window(w);
    const int64_t npx = (int64_t)H * W;
    double *buf = (double *)malloc(sizeof(double) * 5 * npx);
    for (int ch = 0; ch < C; ++ch) {
        double *mx = buf, *my = buf + npx, *sxx = buf + 2 * npx, *syy = buf + 3 * npx, *sxy = buf + 4 * npx;
        ssim_stats(x + ch * npx, y + ch * npx, H, W, w, mx, my, sxx, syy, sxy);
        for (int64_t p = 0; p < npx; ++p)
            map[ch * npx + p] = ((2 * mx[p] * my[p] + SSIM_C1) * (2 * sxy[p] + SSIM_C2)) /
                                ((mx[p] * mx[p] + my[p] * my[p] + SSIM_C1) * (sxx[p] + syy[p] + SSIM_C2));
    }
    free(buf);
}

double or_loss(const double *img, const double *target, int32_t C, int32_t H, int32_t W,
               double lambda_dssim, double *dL_dimg, double *ssim_mean) {
    const int64_t npx = (int64_t)H * W, ntot = npx * C;
    double l1 = 0.0;
    for (int64_t k = 0; k < ntot; ++k) l1 += fabs(img[k] - target[k]);
    l1 /= (double)ntot;
    if (dL_dimg)
        for (int64_t k = 0; k < ntot; ++k) {
            double d = img[k] - target[k];
            dL_dimg[k] = (1.0 - lambda_dssim) * (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / (double)ntot;
        }

    double w[2 * SSIM_R + 1];
    ssim_window(w);
    double *buf = (double *)malloc(sizeof(double) * 8 * npx);
    double ssum = 0.0;
    for (int ch = 0; ch < C; ++ch) {
        const double *x = img + ch * npx, *y = target + ch * npx;
        double *mx = buf, *my = buf + npx, *sxx = buf + 2 * npx, *syy = buf + 3 * npx, *sxy = buf + 4 * npx;
        double *dmu = buf + 5 * npx, *dsxx = buf + 6 * npx, *dsxy = buf + 7 * npx;
        ssim_stats(x, y, H, W, w, mx, my, sxx, syy, sxy);
        for (int64_t p = 0; p < npx; ++p) {
            double A1 = 2 * mx[p] * my[p] + SSIM_C1, A2 = 2 * sxy[p] + SSIM_C2;
            double B1 = mx[p] * mx[p] + my[p] * my[p] + SSIM_C1, B2 = sxx[p] + syy[p] + SSIM_C2;
            double s = (A1 * A2) / (B1 * B2);
            ssum += s;
            /* partial derivatives of s with respect to mu_x, sigma_xx, sigma_xy */
            dmu[p] = (2 * my[p] * A2) / (B1 * B2) - s * 2 * mx[p] / B1;
            dsxx[p] = -s / B2;
            dsxy[p] = 2 * A1 / (B1 * B2);
        }
        if (dL_dimg) {
            /* dSSIM_mean/dx(q) = (1/ntot) sum_p w(q-p) [ ds/dmu_x(p)
                 + ds/dsxx(p) (2 x(q) - 2 mu_x(p)) + ds/dsxy(p) (y(q) - mu_y(p)) ] */
#pragma omp parallel for schedule(static)
            for (int64_t q = 0; q < npx; ++q) {
                int i = (int)(q % W), j = (int)(q / W);
                double g = 0.0;
                for (int dj = -SSIM_R; dj <= SSIM_R; ++dj) {
                    int jj = j + dj;
                    if (jj < 0 || jj >= H) continue;
                    for (int di = -SSIM_R; di <= SSIM_R; ++di) {
                        int ii = i + di;
                        if (ii < 0 || ii >= W) continue;
                        int64_t pp = (int64_t)jj * W + ii;
                        double wt = w[dj + SSIM_R] * w[di + SSIM_R];
                        g += wt * (dmu[pp] + dsxx[pp] * (2 * x[q] - 2 * mx[pp]) + dsxy[pp] * (y[q] - my[pp]));
                    }
                }
                dL_dimg[ch * npx + q] -= lambda_dssim * g / (double)ntot;
            }
        }
    }
    free(buf);
    double ssim = ssum / (double)ntot;
    if (ssim_mean) *ssim_mean = ssim;
    return (1.0 - lambda_dssim) * l1 + lambda_dssim * (1.0 - ssim);
}

/* ------------------------------------------------------------------------ */
/* Backward of the compositing                                                */
/* ------------------------------------------------------------------------ */

static void atomic_add(double *a, double v) {
#pragma omp atomic
    *a += v;
}

static void atomic_max(double *a, double v) {
#pragma omp critical(or_max)
    {
        if (v > *a) *a = v;
    }
}

void or_render_backward(const or_projected *pr, int64_t n, const int32_t *vals, const int64_t *ranges,
                        const or_camera *cam, const or_cfg *cfg,
                        const double *dL_dimg, const double *dL_ddepth,
                        const double *img, const double *target, double tau_err, double loss_v,
                        double mask_tol, double *grad2d, double *stats, double *kappa_amb) {
    const int W = cam->width, H = cam->height;
    const int GW = (W + cfg->tile_w - 1) / cfg->tile_w;
    const int64_t npx = (int64_t)W * H;
    /* this view's footprint size and screen-space gradient per Gaussian, for
       the ||dL/d(u,v)|| and view-count statistics */
    double *view_omega = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *view_duv = (double *)calloc((size_t)(2 * (n > 0 ? n : 1)), sizeof(double));
    int64_t nmax = 0;
    for (int64_t t = 0; t < (int64_t)GW * ((H + cfg->tile_h - 1) / cfg->tile_h); ++t) {
        int64_t len = ranges[2 * t + 1] - ranges[2 * t];
        if (len > nmax) nmax = len;
    }
#pragma omp parallel
    {
        contrib *buf = (contrib *)malloc(sizeof(contrib) * (size_t)(nmax > 0 ? nmax : 1));
#pragma omp for schedule(dynamic, 64)
        for (int64_t p = 0; p < npx; ++p) {
            int i = (int)(p % W), j = (int)(p / W);
            int64_t tile = (int64_t)(j / cfg->tile_h) * GW + (i / cfg->tile_w);
            double C[3], Dp, Tf;
            int64_t last;
            int32_t fl;
            int64_t nb = composite_pixel(pr, vals, ranges[2 * tile], ranges[2 * tile + 1], cfg,
                                         i + 0.5, j + 0.5, buf, nmax, C, &Dp, &Tf, &last, &fl);
            double gC[3] = {dL_dimg[p], dL_dimg[npx + p], dL_dimg[2 * npx + p]};
            double gD = dL_ddepth ? dL_ddepth[p] : 0.0;
            /* error mask of this pixel */
            int mask = 0, amb = 0;
            if (stats) {
                double e = 0.0;
                for (int ch = 0; ch < 3; ++ch) e += fabs(target[ch * npx + p] - img[ch * npx + p]);
                mask = e > tau_err;
                amb = fabs(e - tau_err) < mask_tol;
            }
            /* colour (and depth) behind each blended Gaussian, as suffix sums
               of the blended terms plus the background weighted by T_final */
            double behind[3] = {Tf * cfg->bg[0], Tf * cfg->bg[1], Tf * cfg->bg[2]};
            double behind_d = 0.0;
            for (int64_t k = nb - 1; k >= 0; --k) {
                const contrib *c = buf + k;
                const int64_t g = c->g;
                const double *rgb = pr->rgb + 3 * g;
                const double w = c->alpha * c->T;
                double *gg = grad2d + 10 * g;
                /* dC/dc_j = alpha_j T_j */
                for (int ch = 0; ch < 3; ++ch) atomic_add(&gg[6 + ch], gC[ch] * w);
                atomic_add(&gg[9], gD * w);
                /* dC/dalpha_j = T_j c_j - behind_j / (1 - alpha_j) */
                double dL_dalpha = 0.0;
                for (int ch = 0; ch < 3; ++ch)
                    dL_dalpha += gC[ch] * (c->T * rgb[ch] - behind[ch] / (1.0 - c->alpha));
                dL_dalpha += gD * (c->T * pr->z[g] - behind_d / (1.0 - c->alpha));
                for (int ch = 0; ch < 3; ++ch) behind[ch] += rgb[ch] * w;
                behind_d += pr->z[g] * w;
                if (!c->clamped) {
                    /* alpha = o G, G = exp(power) */
                    atomic_add(&gg[5], dL_dalpha * c->G);
                    double dL_dpow = dL_dalpha * pr->opacity[g] * c->G;
                    const double *q = pr->conic + 3 * g;
                    /* power = -(a dx^2 + c dy^2)/2 - b dx dy, dx = px - u, dy = py - v */
                    double du = dL_dpow * (q[0] * c->dx + q[1] * c->dy);
                    double dv = dL_dpow * (q[2] * c->dy + q[1] * c->dx);
                    atomic_add(&gg[0], du);
                    atomic_add(&gg[1], dv);
                    atomic_add(&view_duv[2 * g], du);
                    atomic_add(&view_duv[2 * g + 1], dv);
                    atomic_add(&gg[2], dL_dpow * (-0.5 * c->dx * c->dx));
                    atomic_add(&gg[3], dL_dpow * (-c->dx * c->dy));
                    atomic_add(&gg[4], dL_dpow * (-0.5 * c->dy * c->dy));
                }
                atomic_add(&view_omega[g], 1.0);
                if (stats) {
                    double *st = stats + 6 * g;
                    atomic_add(&st[0], 1.0);
                    atomic_add(&st[1], (double)mask);
                    atomic_add(&st[2], loss_v);
                    atomic_max(&st[3], w);
                    if (kappa_amb) atomic_add(&kappa_amb[g], (double)amb);
                }
            }
        }
        free(buf);
    }
    if (stats)
        for (int64_t g = 0; g < n; ++g) {
            double du = view_duv[2 * g], dv = view_duv[2 * g + 1];
            stats[6 * g + 4] += sqrt(du * du + dv * dv);
            stats[6 * g + 5] += view_omega[g] > 0.0 ? 1.0 : 0.0;
        }
    free(view_omega);
    free(view_duv);
}

/* ------------------------------------------------------------------------ */
/* Backward of the projection                                                 */
/* ------------------------------------------------------------------------ */

void or_project_backward(const or_params *p, const or_camera *cam, const or_cfg *cfg,
                         const or_projected *pr, const double *grad2d,
                         double *g_means, double *g_log_scales, double *g_quats,
                         double *g_opacity_logits, double *g_sh) {
    const int64_t n = p->n;
    const int32_t D = p->sh_degree, K = sh_coeffs(D);
    double cc[3];
    camera_centre(cam, cc);
    const double *Wc = cam->R;

#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (pr->radius[i] <= 0) continue;
        const double *g2 = grad2d + 10 * i;
        const double *mu = p->means + 3 * i;
        double dmu[3] = {0, 0, 0};

        /* opacity = sigmoid(logit) */
        double o = pr->opacity[i];
        g_opacity_logits[i] += g2[5] * o * (1.0 - o);

        /* colour = max(0, sum_k sh_k Y_k(dir) + 0.5), dir = (mu - c)/|mu - c| */
        double dvec[3] = {mu[0] - cc[0], mu[1] - cc[1], mu[2] - cc[2]};
        double nd = sqrt(dvec[0] * dvec[0] + dvec[1] * dvec[1] + dvec[2] * dvec[2]);
        double dir[3] = {dvec[0] / nd, dvec[1] / nd, dvec[2] / nd};
        double Y[(OR_MAX_SH_DEG + 1) * (OR_MAX_SH_DEG + 1)], dY[3 * (OR_MAX_SH_DEG + 1) * (OR_MAX_SH_DEG + 1)];
        or_sh_eval(D, dir, Y, dY);
        double ddir[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ++ch) {
            if (pr->rgb_clamped[3 * i + ch]) continue;
            double gc = g2[6 + ch];
            for (int k = 0; k < K; ++k) {
                double shk = p->sh[(i * K + k) * 3 + ch];
                g_sh[(i * K + k) * 3 + ch] += gc * Y[k];
                for (int a = 0; a < 3; ++a) ddir[a] += gc * shk * dY[3 * k + a];
            }
        }
        double dd = dir[0] * ddir[0] + dir[1] * ddir[1] + dir[2] * ddir[2];
        for (int a = 0; a < 3; ++a) dmu[a] += (ddir[a] - dir[a] * dd) / nd;

        /* conic (a, b, c) = (C, -B, A)/det of the dilated covariance (A, B, C) */
        const double A = pr->cov2d[3 * i + 0], B = pr->cov2d[3 * i + 1], C = pr->cov2d[3 * i + 2];
        const double det = A * C - B * B, det2 = det * det;
        const double ga = g2[2], gb = g2[3], gcn = g2[4];
        double dA = ga * (-C * C / det2) + gb * (B * C / det2) + gcn * (1.0 / det - A * C / det2);
        double dC = ga * (1.0 / det - C * A / det2) + gb * (B * A / det2) + gcn * (-A * A / det2);
        double dB = ga * (2.0 * B * C / det2) + gb * (-1.0 / det - 2.0 * B * B / det2) + gcn * (2.0 * A * B / det2);

        /* recompute the forward quantities */
        double pc[3];
        for (int r = 0; r < 3; ++r)
            pc[r] = Wc[3 * r + 0] * mu[0] + Wc[3 * r + 1] * mu[1] + Wc[3 * r + 2] * mu[2] + cam->t[r];
        const double x = pc[0], y = pc[1], z = pc[2];
        double qv[4] = {p->quats[4 * i], p->quats[4 * i + 1], p->quats[4 * i + 2], p->quats[4 * i + 3]};
        double nq = sqrt(qv[0] * qv[0] + qv[1] * qv[1] + qv[2] * qv[2] + qv[3] * qv[3]);
        double qh[4] = {qv[0] / nq, qv[1] / nq, qv[2] / nq, qv[3] / nq};
        double Rq[9];
        quat_rot_unit(qh[0], qh[1], qh[2], qh[3], Rq);
        double s[3];
        for (int k = 0; k < 3; ++k) s[k] = exp(p->log_scales[3 * i + k]);
        double M[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) M[3 * r + c] = Rq[3 * r + c] * s[c];
        double Sig[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += M[3 * r + k] * M[3 * c + k];
                Sig[3 * r + c] = acc;
            }
        const double limx = cfg->tan_clamp * cam->width / (2.0 * cam->fx);
        const double limy = cfg->tan_clamp * cam->height / (2.0 * cam->fy);
        double rx = x / z, ry = y / z;
        int cx_lo = rx < -limx, cx_hi = rx > limx, cy_lo = ry < -limy, cy_hi = ry > limy;
        double tx = z * (cx_lo ? -limx : (cx_hi ? limx : rx));
        double ty = z * (cy_lo ? -limy : (cy_hi ? limy : ry));
        double dtx_dx = (cx_lo || cx_hi) ? 0.0 : 1.0, dtx_dz = cx_lo ? -limx : (cx_hi ? limx : 0.0);
        double dty_dy = (cy_lo || cy_hi) ? 0.0 : 1.0, dty_dz = cy_lo ? -limy : (cy_hi ? limy : 0.0);
        const double fx = cam->fx, fy = cam->fy;
        double J[6] = {fx / z, 0.0, -fx * tx / (z * z), 0.0, fy / z, -fy * ty / (z * z)};
        double T[6];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c)
                T[3 * r + c] = J[3 * r + 0] * Wc[0 * 3 + c] + J[3 * r + 1] * Wc[1 * 3 + c] + J[3 * r + 2] * Wc[2 * 3 + c];

        /* A = T0 Sig T0^T, B = T0 Sig T1^T, C = T1 Sig T1^T */
        double dSig[9];
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l)
                dSig[3 * k + l] = dA * T[k] * T[l] + dC * T[3 + k] * T[3 + l] + dB * T[k] * T[3 + l];
        double ST0[3], ST1[3];
        for (int k = 0; k < 3; ++k) {
            ST0[k] = Sig[3 * k + 0] * T[0] + Sig[3 * k + 1] * T[1] + Sig[3 * k + 2] * T[2];
            ST1[k] = Sig[3 * k + 0] * T[3] + Sig[3 * k + 1] * T[4] + Sig[3 * k + 2] * T[5];
        }
        double dT[6];
        for (int k = 0; k < 3; ++k) {
            dT[k] = 2.0 * dA * ST0[k] + dB * ST1[k];
            dT[3 + k] = 2.0 * dC * ST1[k] + dB * ST0[k];
        }
        /* T = J W: dJ_rk = sum_c dT_rc W_kc */
        double dJ[6];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k)
                dJ[3 * r + k] = dT[3 * r + 0] * Wc[3 * k + 0] + dT[3 * r + 1] * Wc[3 * k + 1] + dT[3 * r + 2] * Wc[3 * k + 2];
        double dpc[3] = {0, 0, 0};
        const double z2 = z * z, z3 = z2 * z;
        dpc[2] += dJ[0] * (-fx / z2) + dJ[4] * (-fy / z2);
        dpc[2] += dJ[2] * (-fx * dtx_dz / z2 + 2.0 * fx * tx / z3);
        dpc[2] += dJ[5] * (-fy * dty_dz / z2 + 2.0 * fy * ty / z3);
        dpc[0] += dJ[2] * (-fx / z2) * dtx_dx;
        dpc[1] += dJ[5] * (-fy / z2) * dty_dy;
        /* u = fx x/z + cx, v = fy y/z + cy, depth z */
        dpc[0] += g2[0] * fx / z;
        dpc[2] += g2[0] * (-fx * x / z2);
        dpc[1] += g2[1] * fy / z;
        dpc[2] += g2[1] * (-fy * y / z2);
        dpc[2] += g2[9];
        for (int a = 0; a < 3; ++a) dmu[a] += Wc[0 * 3 + a] * dpc[0] + Wc[1 * 3 + a] * dpc[1] + Wc[2 * 3 + a] * dpc[2];

        /* Sig = M M^T, M = Rq diag(s) */
        double dM[9];
        for (int k = 0; k < 3; ++k)
            for (int m = 0; m < 3; ++m) {
                double acc = 0.0;
                for (int l = 0; l < 3; ++l) acc += (dSig[3 * k + l] + dSig[3 * l + k]) * M[3 * l + m];
                dM[3 * k + m] = acc;
            }
        double dRq[9];
        for (int m = 0; m < 3; ++m) {
            double ds = 0.0;
            for (int k = 0; k < 3; ++k) {
                ds += dM[3 * k + m] * Rq[3 * k + m];
                dRq[3 * k + m] = dM[3 * k + m] * s[m];
            }
            g_log_scales[3 * i + m] += ds * s[m];
        }
        double dR[4][9];
        quat_rot_partials(qh[0], qh[1], qh[2], qh[3], dR);
        double dqh[4];
        for (int a = 0; a < 4; ++a) {
            double acc = 0.0;
            for (int e = 0; e < 9; ++e) acc += dRq[e] * dR[a][e];
            dqh[a] = acc;
        }
        double qd = qh[0] * dqh[0] + qh[1] * dqh[1] + qh[2] * dqh[2] + qh[3] * dqh[3];
        for (int a = 0; a < 4; ++a) g_quats[4 * i + a] += (dqh[a] - qh[a] * qd) / nq;
        for (int a = 0; a < 3; ++a) g_means[3 * i + a] += dmu[a];
    }
}

/* ------------------------------------------------------------------------ */
/* Adam                                                                       */
/* ------------------------------------------------------------------------ */

void or_adam(int64_t n, double *p, const double *g, double *m, double *v, const double *lr,
             double beta1, double beta2, double eps, int64_t step) {
    const double bc1 = 1.0 - pow(beta1, (double)step), bc2 = 1.0 - pow(beta2, (double)step);
    for (int64_t k = 0; k < n; ++k) {
        m[k] = beta1 * m[k] + (1.0 - beta1) * g[k];
        v[k] = beta2 * v[k] + (1.0 - beta2) * g[k] * g[k];
        double mhat = m[k] / bc1, vhat = v[k] / bc2;
        p[k] -= lr[k] * mhat / (sqrt(vhat) + eps);
    }
}

/* ------------------------------------------------------------------------ */
/* Lifecycle scores (Supp. E.1, E.2; Sec. 3.3.2)                              */
/* ------------------------------------------------------------------------ */

void or_prune_finalize(int64_t n, const double *omega, const double *kappa, const double *gamma,
                       int32_t n_views, double tau_d, double tau_p,
                       double *S_d, double *S_p, uint8_t *densify, double *prune_max,
                       uint8_t *prune) {
    double lmin = INFINITY, lmax = -INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        /* S_d = mean over the sampled views of kappa_v */
        S_d[i] = kappa[i] / (double)n_views;
        if (S_d[i] > tau_d) densify[i] = 1;
        if (omega[i] > 0.0) {
            double L = log(1.0 + gamma[i]);
            if (L < lmin) lmin = L;
            if (L > lmax) lmax = L;
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        double sp = 0.0;
        if (omega[i] > 0.0 && lmax > lmin) sp = (log(1.0 + gamma[i]) - lmin) / (lmax - lmin);
        S_p[i] = sp;
        if (sp > prune_max[i]) prune_max[i] = sp;
        prune[i] = prune_max[i] > tau_p;
    }
}

/* ------------------------------------------------------------------------ */
/* Geometric and isotropic terms of L_total (Supp. D.4)                       */
/* ------------------------------------------------------------------------ */

/* L_geo = mean over the npx pixels of [prior > 0] |prior - depth|; returns it
 * and writes dL/ddepth (nullable).  Reading: the printed L1 norm taken as a
 * mean over pixels like L_photo, pixels without a prior (prior <= 0) adding 0. */
double or_geo_loss(const double *depth, const double *prior, int64_t npx, double *dL_ddepth) {
    double s = 0.0;
    for (int64_t p = 0; p < npx; ++p) {
        double g = 0.0;
        if (prior[p] > 0.0) {
            double d = depth[p] - prior[p];
            s += fabs(d);
            g = (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / (double)npx;
        }
        if (dL_ddepth) dL_ddepth[p] = g;
    }
    return s / (double)npx;
}

/* L_iso = mean over the n Gaussians of sum_k |s_k - mean(s)|, s = exp(log-scale);
 * returns it and adds dL/dlog-scale into g_log_scales (nullable).  Reading:
 * the printed sum over Gaussians normalised by n as in the cited MonoGS. */
double or_iso_loss(int64_t n, const double *log_scales, double *g_log_scales) {
    double L = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double s[3], mean = 0.0;
        for (int k = 0; k < 3; ++k) { s[k] = exp(log_scales[3 * i + k]); mean += s[k] / 3.0; }
        double e[3], esum = 0.0;
        for (int k = 0; k < 3; ++k) {
            double d = s[k] - mean;
            L += fabs(d);
            e[k] = d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0);
            esum += e[k];
        }
        if (g_log_scales)
            for (int k = 0; k < 3; ++k)  /* d|s_k - m|/ds_j = e_k (delta_kj - 1/3) */
                g_log_scales[3 * i + k] += (e[k] - esum / 3.0) * s[k] / (double)n;
    }
    return L / (double)n;
}

/* ------------------------------------------------------------------------ */
/* Learned prune / densify predictor (a later row of the build; the paper     */
/* decides with the plain criterion of Supp. E): MLP 16 -> 64 -> 64 -> 2       */
/* with ReLU hidden layers and sigmoid outputs (densify, prune).              */
/* ------------------------------------------------------------------------ */

/* Weights in one array: W1[64][16], b1[64], W2[64][64], b2[64], W3[2][64], b3[2]. */
#define OR_MLP_IN 16
#define OR_MLP_H 64
#define OR_MLP_OUT 2
#define OR_MLP_W1 0
#define OR_MLP_B1 (OR_MLP_W1 + OR_MLP_H * OR_MLP_IN)
#define OR_MLP_W2 (OR_MLP_B1 + OR_MLP_H)
#define OR_MLP_B2 (OR_MLP_W2 + OR_MLP_H * OR_MLP_H)
#define OR_MLP_W3 (OR_MLP_B2 + OR_MLP_H)
#define OR_MLP_B3 (OR_MLP_W3 + OR_MLP_OUT * OR_MLP_H)
#define OR_MLP_NW (OR_MLP_B3 + OR_MLP_OUT)

/* Round to the nearest bfloat16 (ties to even) through float, as a tensor-core
 * operand is rounded. */
static double bf16_round(double v) {
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (double)f;  /* inf / nan unchanged */
    u += 0x7fffu + ((u >> 16) & 1u);
    u &= 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

int32_t or_mlp_num_weights(void) { return OR_MLP_NW; }

/* Forward of n rows of features x[n][16]; writes p[n][2] (nullable), and the
 * hidden activations h1[n][64], h2[n][64] (nullable).  bf16 != 0 rounds the
 * tensor-core operands (x, W1, W2, h1) to bfloat16 as the kernels do. */
void or_mlp_forward(int64_t n, const double *x, const double *w, int32_t bf16, double *p, double *h1o, double *h2o) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double xi[OR_MLP_IN], h1[OR_MLP_H], h2[OR_MLP_H];
        for (int c = 0; c < OR_MLP_IN; ++c) xi[c] = bf16 ? bf16_round(x[i * OR_MLP_IN + c]) : x[i * OR_MLP_IN + c];
        for (int o = 0; o < OR_MLP_H; ++o) {
            double s = 0.0;
            for (int c = 0; c < OR_MLP_IN; ++c) {
                double wv = w[OR_MLP_W1 + o * OR_MLP_IN + c];
                s += (bf16 ? bf16_round(wv) : wv) * xi[c];
            }
            s += w[OR_MLP_B1 + o];
            h1[o] = s > 0.0 ? s : 0.0;
        }
        for (int o = 0; o < OR_MLP_H; ++o) {
            double s = 0.0;
            for (int c = 0; c < OR_MLP_H; ++c) {
                double wv = w[OR_MLP_W2 + o * OR_MLP_H + c];
                s += (bf16 ? bf16_round(wv) : wv) * (bf16 ? bf16_round(h1[c]) : h1[c]);
            }
            s += w[OR_MLP_B2 + o];
            h2[o] = s > 0.0 ? s : 0.0;
        }
        for (int k = 0; k < OR_MLP_OUT; ++k) {
            double z = w[OR_MLP_B3 + k];
            for (int c = 0; c < OR_MLP_H; ++c) z += w[OR_MLP_W3 + k * OR_MLP_H + c] * h2[c];
            if (p) p[i * OR_MLP_OUT + k] = 1.0 / (1.0 + exp(-z));
        }
        if (h1o) memcpy(h1o + i * OR_MLP_H, h1, sizeof(h1));
        if (h2o) memcpy(h2o + i * OR_MLP_H, h2, sizeof(h2));
    }
}

/* Mean binary cross-entropy over the n rows and both outputs of the labels
 * y[n][2] in {0, 1}; writes dL/dw (accumulated into g) and returns L.
 * bf16 as in or_mlp_forward: the forward's hidden-layer operands (x, W1, W2,
 * h1) are rounded to bfloat16, which is all the BF16 reading fixes.  The
 * backward is the plain FP64 chain rule of that forward, the rounding taken
 * as the identity (a rounded operand's gradient is the gradient of the value
 * it stands for): no quantity of the backward is rounded.
 * dh2o, dh1o (nullable, [n][64]): the per-row gradients with respect to the
 * layer-2 and layer-1 pre-activations (after the ReLU masks), for tests that
 * bound how far a kernel's own roundings of them may move the weight sums. */
double or_mlp_bce_grad(int64_t n, const double *x, const double *y, const double *w, int32_t bf16, double *g,
                       double *dh2o, double *dh1o) {
    double L = 0.0;
    const double scale = 1.0 / (double)(n * OR_MLP_OUT);
    for (int64_t i = 0; i < n; ++i) {
        double xi[OR_MLP_IN], h1[OR_MLP_H], h2[OR_MLP_H], p[OR_MLP_OUT];
        or_mlp_forward(1, x + i * OR_MLP_IN, w, bf16, p, h1, h2);
        for (int c = 0; c < OR_MLP_IN; ++c) xi[c] = bf16 ? bf16_round(x[i * OR_MLP_IN + c]) : x[i * OR_MLP_IN + c];
        double dz[OR_MLP_OUT];
        for (int k = 0; k < OR_MLP_OUT; ++k) {
            const double yk = y[i * OR_MLP_OUT + k];
            const double pk = p[k] < 1e-300 ? 1e-300 : (p[k] > 1.0 - 1e-16 ? 1.0 - 1e-16 : p[k]);
            L -= yk * log(pk) + (1.0 - yk) * log(1.0 - pk);
            dz[k] = (p[k] - yk) * scale;  /* dBCE/dz = p - y */
            g[OR_MLP_B3 + k] += dz[k];
            for (int c = 0; c < OR_MLP_H; ++c) g[OR_MLP_W3 + k * OR_MLP_H + c] += dz[k] * h2[c];
        }
        double dh2[OR_MLP_H];
        for (int c = 0; c < OR_MLP_H; ++c) {
            double s = 0.0;
            for (int k = 0; k < OR_MLP_OUT; ++k) s += dz[k] * w[OR_MLP_W3 + k * OR_MLP_H + c];
            dh2[c] = h2[c] > 0.0 ? s : 0.0;
        }
        /* layer 2: z2 = W2 h1' + b2 with h1' = bf16(h1) in bf16 mode */
        for (int o = 0; o < OR_MLP_H; ++o) {
            g[OR_MLP_B2 + o] += dh2[o];
            for (int c = 0; c < OR_MLP_H; ++c) g[OR_MLP_W2 + o * OR_MLP_H + c] += dh2[o] * (bf16 ? bf16_round(h1[c]) : h1[c]);
        }
        /* through layer 2 to h1, with the weights the forward multiplied by */
        double dh1[OR_MLP_H];
        for (int c = 0; c < OR_MLP_H; ++c) {
            double s = 0.0;
            for (int o = 0; o < OR_MLP_H; ++o) {
                const double wv = w[OR_MLP_W2 + o * OR_MLP_H + c];
                s += dh2[o] * (bf16 ? bf16_round(wv) : wv);
            }
            dh1[c] = h1[c] > 0.0 ? s : 0.0;
        }
        /* layer 1: z1 = W1 x' + b1 with x' = bf16(x) in bf16 mode */
        for (int o = 0; o < OR_MLP_H; ++o) {
            g[OR_MLP_B1 + o] += dh1[o];
            for (int c = 0; c < OR_MLP_IN; ++c) g[OR_MLP_W1 + o * OR_MLP_IN + c] += dh1[o] * xi[c];
        }
        if (dh2o) memcpy(dh2o + i * OR_MLP_H, dh2, sizeof(dh2));
        if (dh1o) memcpy(dh1o + i * OR_MLP_H, dh1, sizeof(dh1));
    }
    return L * scale;
}

/* ------------------------------------------------------------------------ */
/* Predictor inputs and the densify / prune actions                          */
/* ------------------------------------------------------------------------ */

void or_mlp_features(int64_t n, const double *means, const double *log_scales, const double *opacity_logits,
                     const double *stats, const double *ring, int32_t head, const double cam[3], double *feat) {
    for (int64_t i = 0; i < n; ++i) {
        double *f = feat + i * OR_MLP_IN;
        const double *st = stats + i * 6;
        const double views = st[5];
        f[0] = 1.0 / (1.0 + exp(-opacity_logits[i]));
        for (int k = 0; k < 3; ++k) f[1 + k] = log_scales[3 * i + k];
        f[4] = log(1.0 + views);
        f[5] = log(1.0 + 1e4 * st[4]);
        for (int j = 0; j < 8; ++j) f[6 + j] = ring[(int64_t)(((head - j) % 8 + 8) % 8) * n + i];
        double d2 = 0.0;
        for (int k = 0; k < 3; ++k) d2 += (means[3 * i + k] - cam[k]) * (means[3 * i + k] - cam[k]);
        f[14] = log(1.0 + sqrt(d2));
        f[15] = log(1.0 + st[0] / (views > 1.0 ? views : 1.0));
    }
}

int64_t or_densify_prune(int64_t n, int32_t K_row, const double *P, const double *m, const double *v,
                         const uint8_t *densify, const uint8_t *prune, const double *noise,
                         double split_log_scale, double split_factor, int64_t cap, double *P_out,
                         double *m_out, double *v_out) {
    int64_t o = 0;
    for (int64_t i = 0; i < n; ++i) {
        const double *src = P + i * K_row;
        if (prune[i]) continue;
        double rows[2][64 * 3];
        int emit = 1, moments_first = 1;
        memcpy(rows[0], src, sizeof(double) * K_row);
        if (densify[i]) {
            emit = 2;
            memcpy(rows[1], src, sizeof(double) * K_row);
            double lmax = src[3];
            if (src[4] > lmax) lmax = src[4];
            if (src[5] > lmax) lmax = src[5];
            if (lmax > split_log_scale) {  /* split into two samples of N(mu, Sigma) */
                double R[9];
                or_quat_to_rot(src + 6, R);
                for (int j = 0; j < 2; ++j) {
                    const double *xi = noise + i * 6 + 3 * j;
                    for (int r = 0; r < 3; ++r) {
                        double d = 0.0;
                        for (int c = 0; c < 3; ++c) d += R[3 * r + c] * exp(src[3 + c]) * xi[c];
                        rows[j][r] = src[r] + d;
                    }
                    for (int c = 0; c < 3; ++c) rows[j][3 + c] = src[3 + c] - log(split_factor);
                }
                moments_first = 0;
            }
        }
        for (int j = 0; j < emit; ++j, ++o) {
            if (o >= cap) continue;
            memcpy(P_out + o * K_row, rows[j], sizeof(double) * K_row);
            const int keep = j == 0 && moments_first;
            for (int k = 0; k < K_row; ++k) {
                if (m_out) m_out[o * K_row + k] = keep && m ? m[i * K_row + k] : 0.0;
                if (v_out) v_out[o * K_row + k] = keep && v ? v[i * K_row + k] : 0.0;
            }
        }
    }
    return o;
}

/* ------------------------------------------------------------------------ */
/* Probabilistic initialisation (Sec. 3.3.1, Supp. D.5)                        */
/* ------------------------------------------------------------------------ */

static double px_at(const double *a, int H, int W, int y, int x) {
    return a[(int64_t)clampi(y, 0, H - 1) * W + clampi(x, 0, W - 1)];
}

/* Y * G_s at every pixel: the direct 2D sum over the window (R19). */
static void gauss_blur_2d(const double *Y, int H, int W, double s, double *out) {
    const int r = (int)ceil(3.0 * s);
    double norm = 0.0;
    for (int dy = -r; dy <= r; ++dy)
        for (int dx = -r; dx <= r; ++dx) norm += exp(-(double)(dx * dx + dy * dy) / (2.0 * s * s));
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double acc = 0.0;
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx)
                    acc += exp(-(double)(dx * dx + dy * dy) / (2.0 * s * s)) / norm * px_at(Y, H, W, y + dy, x + dx);
            out[(int64_t)y * W + x] = acc;
        }
}

void or_init_saliency(int32_t H, int32_t W, const double *img, const double *depth, double sigma1,
                      double sigma2, double scale, double *dog, double *grad) {
    const int64_t npx = (int64_t)H * W;
    double *Y = (double *)malloc(sizeof(double) * npx);
    double *b1 = (double *)malloc(sizeof(double) * npx);
    double *b2 = (double *)malloc(sizeof(double) * npx);
    for (int64_t i = 0; i < npx; ++i) Y[i] = (img[i] + img[npx + i] + img[2 * npx + i]) / 3.0;
    gauss_blur_2d(Y, H, W, sigma1, b1);
    gauss_blur_2d(Y, H, W, sigma2, b2);
    for (int64_t i = 0; i < npx; ++i) dog[i] = fmin(scale * fabs(b1[i] - b2[i]), 1.0);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const double gx = (px_at(depth, H, W, y, x + 1) - px_at(depth, H, W, y, x - 1)) / 2.0;
            const double gy = (px_at(depth, H, W, y + 1, x) - px_at(depth, H, W, y - 1, x)) / 2.0;
            grad[(int64_t)y * W + x] = sqrt(gx * gx + gy * gy);
        }
    free(Y);
    free(b1);
    free(b2);
}

/* P = min(lambda DoG + (1 - lambda) minmax(||grad D||), 1) (Sec. 3.3.1, R20). */
static void init_p(int32_t H, int32_t W, const double *img, const double *depth, double s1, double s2,
                   double scale, double lambda, double *P) {
    const int64_t npx = (int64_t)H * W;
    double *dog = (double *)malloc(sizeof(double) * npx);
    double *g = (double *)malloc(sizeof(double) * npx);
    or_init_saliency(H, W, img, depth, s1, s2, scale, dog, g);
    double lo = g[0], hi = g[0];
    for (int64_t i = 1; i < npx; ++i) {
        lo = fmin(lo, g[i]);
        hi = fmax(hi, g[i]);
    }
    for (int64_t i = 0; i < npx; ++i) {
        const double gn = hi > lo ? (g[i] - lo) / (hi - lo) : 0.0;
        P[i] = fmin(lambda * dog[i] + (1.0 - lambda) * gn, 1.0);
    }
    free(dog);
    free(g);
}

void or_init_probability(int32_t H, int32_t W, const double *img, const double *depth, const double *img_r,
                         const double *depth_r, double sigma1, double sigma2, double scale, double lambda,
                         double *prob) {
    const int64_t npx = (int64_t)H * W;
    init_p(H, W, img, depth, sigma1, sigma2, scale, lambda, prob);
    if (!img_r) return;
    double *Pr = (double *)malloc(sizeof(double) * npx);
    init_p(H, W, img_r, depth_r, sigma1, sigma2, scale, lambda, Pr);
    for (int64_t i = 0; i < npx; ++i) prob[i] = fmax(prob[i] - Pr[i], 0.0); /* P_kf */
    free(Pr);
}

int64_t or_init_select(int32_t H, int32_t W, const double *prob, const double *uniform, const double *depth,
                       const or_camera *cam, double near_z, int32_t levels, const double *voxel,
                       const double *max_dist, int64_t n_old, const int64_t *old_keys, int64_t cap,
                       int64_t *new_keys, double *pos, int32_t *level, int32_t *pixel, uint8_t *selected,
                       uint8_t *uncertain, double tol, double tol_rel) {
    const int64_t npx = (int64_t)H * W;
    /* every occupied voxel, old ones first; grows as voxels are met */
    int64_t n_keys = n_old, key_cap = n_old + 1024, n_new = 0;
    int64_t *keys = (int64_t *)malloc(sizeof(int64_t) * 4 * (size_t)key_cap);
    if (n_old) memcpy(keys, old_keys, sizeof(int64_t) * 4 * (size_t)n_old);
    if (selected) memset(selected, 0, (size_t)npx);
    if (uncertain) memset(uncertain, 0, (size_t)npx);
    const double tabs = fabs(cam->t[0]) + fabs(cam->t[1]) + fabs(cam->t[2]);
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const int64_t p = (int64_t)y * W + x;
            const double P = prob[p];
            int unsure = 0, is_max = P > 0.0, dominated = 0, close = 0;
            /* 3x3 non-maximum suppression; equal values go to the lower raster index */
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int yy = y + dy, xx = x + dx;
                    if ((dx == 0 && dy == 0) || yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                    const int64_t q = (int64_t)yy * W + xx;
                    const double Q = prob[q];
                    if (Q > P || (Q == P && q < p)) is_max = 0;
                    if (Q > P + tol) dominated = 1;
                    else if (Q != P && fabs(Q - P) <= tol) close = 1;
                }
            /* a pixel beaten by more than tol stays suppressed; otherwise a near tie may flip */
            if (P > 0.0 && !dominated && (close || P <= tol)) unsure = 1;
            const double d = depth[p];
            if (is_max && (fabs(uniform[p] - P) <= tol || fabs(d - near_z) <= tol_rel * near_z)) unsure = 1;
            int l = -1, in_range = 1;
            int64_t idx[3] = {0, 0, 0};
            if (is_max && uniform[p] < P && d > near_z) {
                /* the pixel centre at its depth (R1), back to the world frame */
                const double xc[3] = {d * ((x + 0.5 - cam->cx) / cam->fx), d * ((y + 0.5 - cam->cy) / cam->fy), d};
                double xw[3];
                for (int i = 0; i < 3; ++i)
                    xw[i] = cam->R[0 + i] * (xc[0] - cam->t[0]) + cam->R[3 + i] * (xc[1] - cam->t[1]) +
                            cam->R[6 + i] * (xc[2] - cam->t[2]);
                const double dist = sqrt(xc[0] * xc[0] + xc[1] * xc[1] + xc[2] * xc[2]);
                for (int k = 0; k < levels && l < 0; ++k) {
                    if (fabs(dist - max_dist[k]) <= tol_rel * dist) unsure = 1;
                    if (dist < max_dist[k]) l = k;
                }
                if (l >= 0) {
                    const double xabs = fabs(xc[0]) + fabs(xc[1]) + fabs(xc[2]);
                    for (int i = 0; i < 3; ++i) {
                        const double q = xw[i] / voxel[l];
                        /* the device's FP32 point carries an error that scales with |x_c| + |t| */
                        if (fabs(q - floor(q + 0.5)) <= tol_rel * (1.0 + fabs(q) + (xabs + tabs) / voxel[l]))
                            unsure = 1;
                        idx[i] = (int64_t)floor(q);
                        if (idx[i] >= (1 << 19) || idx[i] < -(1 << 19)) in_range = 0;
                    }
                }
            }
            if (uncertain) uncertain[p] = (uint8_t)unsure;
            if (l < 0 || !in_range) continue;
            if (selected) selected[p] = 1;
            int seen = 0;
            for (int64_t k = 0; k < n_keys && !seen; ++k)
                seen = keys[4 * k] == l && keys[4 * k + 1] == idx[0] && keys[4 * k + 2] == idx[1] &&
                       keys[4 * k + 3] == idx[2];
            if (seen) continue;
            if (n_keys == key_cap) {
                key_cap *= 2;
                keys = (int64_t *)realloc(keys, sizeof(int64_t) * 4 * (size_t)key_cap);
            }
            int64_t *kk = keys + 4 * n_keys++;
            kk[0] = l;
            kk[1] = idx[0];
            kk[2] = idx[1];
            kk[3] = idx[2];
            if (n_new < cap) {
                memcpy(new_keys + 4 * n_new, kk, sizeof(int64_t) * 4);
                for (int i = 0; i < 3; ++i) pos[3 * n_new + i] = (double)idx[i] * voxel[l];
                level[n_new] = l;
                pixel[n_new] = (int32_t)p;
            }
            ++n_new;
        }
    free(keys);
    return n_new;
}

/* ------------------------------------------------------------------------ */
/* Scaffold-GS anchor decoding (Supp. D.1, D.3; readings R25-R29)            */
/* ------------------------------------------------------------------------ */

#define OR_ANC_K 10
#define OR_ANC_F 32
#define OR_ANC_IN 36
#define OR_ANC_H 64
#define OR_ANC_OUT (14 * OR_ANC_K)
#define OR_ANC_W1 0
#define OR_ANC_B1 (OR_ANC_W1 + OR_ANC_H * OR_ANC_IN)
#define OR_ANC_W2 (OR_ANC_B1 + OR_ANC_H)
#define OR_ANC_B2 (OR_ANC_W2 + OR_ANC_OUT * OR_ANC_H)
#define OR_ANC_NW (OR_ANC_B2 + OR_ANC_OUT)
#define OR_Y00 0.28209479177387814 /* 1 / (2 sqrt(pi)) */

int32_t or_anchor_num_weights(void) { return OR_ANC_NW; }

static double sigm(double z) { return 1.0 / (1.0 + exp(-z)); }

/* Decoder input, hidden pre-activations and the 14 K outputs of anchor i.
 * bf16 != 0 (reading R30) rounds the hidden layers' operands to bfloat16 as
 * the tensor cores take them: the input x (returned rounded), W1, the hidden
 * activation relu(pre) and W2; the sums and the biases stay FP64. */
static void anchor_mlp(const double *pos, const double *feat, const double *w, const double cc[3], double *x,
                       double *pre, double *z, double *dist, int bf16) {
    double v[3];
    for (int a = 0; a < 3; ++a) v[a] = pos[a] - cc[a];
    const double d = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int c = 0; c < OR_ANC_F; ++c) x[c] = feat[c];
    for (int a = 0; a < 3; ++a) x[OR_ANC_F + a] = v[a] / d;
    x[OR_ANC_F + 3] = log1p(d);
    if (bf16)
        for (int c = 0; c < OR_ANC_IN; ++c) x[c] = bf16_round(x[c]);
    for (int o = 0; o < OR_ANC_H; ++o) {
        double s = w[OR_ANC_B1 + o];
        for (int c = 0; c < OR_ANC_IN; ++c) {
            const double wv = w[OR_ANC_W1 + o * OR_ANC_IN + c];
            s += (bf16 ? bf16_round(wv) : wv) * x[c];
        }
        pre[o] = s;
    }
    for (int o = 0; o < OR_ANC_OUT; ++o) {
        double s = w[OR_ANC_B2 + o];
        for (int c = 0; c < OR_ANC_H; ++c) {
            const double wv = w[OR_ANC_W2 + o * OR_ANC_H + c], h = pre[c] > 0.0 ? pre[c] : 0.0;
            s += (bf16 ? bf16_round(wv) : wv) * (bf16 ? bf16_round(h) : h);
        }
        z[o] = s;
    }
    *dist = d;
}

void or_anchor_hidden(int64_t n, const double *pos, const double *feat, const double *w, const double cam_c[3],
                      int32_t bf16, double *x_raw, double *pre) {
    for (int64_t i = 0; i < n; ++i) {
        double x[OR_ANC_IN], p[OR_ANC_H], z[OR_ANC_OUT], d;
        if (x_raw) {
            anchor_mlp(pos + 3 * i, feat + OR_ANC_F * i, w, cam_c, x, p, z, &d, 0);
            for (int c = 0; c < OR_ANC_IN; ++c) x_raw[OR_ANC_IN * i + c] = x[c];
        }
        if (pre) {
            anchor_mlp(pos + 3 * i, feat + OR_ANC_F * i, w, cam_c, x, p, z, &d, bf16);
            for (int c = 0; c < OR_ANC_H; ++c) pre[OR_ANC_H * i + c] = p[c];
        }
    }
}

static int lod_active(int32_t level, double d, const double *max_dist) {
    const double lo = level > 0 ? max_dist[level - 1] : 0.0;
    return d >= lo && d < max_dist[level];
}

void or_anchor_decode(int64_t n, const double *pos, const int32_t *level, const double *feat, const double *log_l,
                      const double *offs, const double *w, const double cam_c[3], const double *max_dist,
                      double *rows, uint8_t *keep, uint8_t *unsure, double tol, int32_t bf16) {
    for (int64_t i = 0; i < n; ++i) {
        double x[OR_ANC_IN], pre[OR_ANC_H], z[OR_ANC_OUT], d;
        anchor_mlp(pos + 3 * i, feat + OR_ANC_F * i, w, cam_c, x, pre, z, &d, bf16);
        const int M = lod_active(level[i], d, max_dist);
        const double lo = level[i] > 0 ? max_dist[level[i] - 1] : 0.0;
        int near_band = fabs(d - lo) <= tol * d || fabs(d - max_dist[level[i]]) <= tol * d;
        const double *L = log_l + 3 * i;
        for (int k = 0; k < OR_ANC_K; ++k) {
            const double *zk = z + 14 * k;
            double *r = rows + 14 * (k * n + i);
            const double a = tanh(zk[3]);
            const int kp = M && a > 0.0;
            if (keep) keep[k * n + i] = (uint8_t)kp;
            if (unsure) unsure[k * n + i] = (uint8_t)(near_band || fabs(zk[3]) <= tol);
            if (!kp) {  /* dropped: a culled placeholder at the anchor */
                for (int c = 0; c < 3; ++c) r[c] = pos[3 * i + c];
                for (int c = 0; c < 3; ++c) r[3 + c] = L[c];
                r[6] = 1.0; r[7] = r[8] = r[9] = 0.0;
                r[10] = -30.0;
                r[11] = r[12] = r[13] = 0.0;
                continue;
            }
            for (int c = 0; c < 3; ++c) {
                const double l = exp(L[c]);
                r[c] = pos[3 * i + c] + (offs[(OR_ANC_K * i + k) * 3 + c] + zk[11 + c]) * l;  /* mean */
                r[3 + c] = L[c] + log(sigm(zk[8 + c]));                                       /* log(l ds) */
            }
            r[6] = 1.0 + zk[4];
            r[7] = zk[5];
            r[8] = zk[6];
            r[9] = zk[7];
            r[10] = log(a / (1.0 - a));
            for (int c = 0; c < 3; ++c) r[11 + c] = (sigm(zk[c]) - 0.5) / OR_Y00;
        }
    }
}

void or_anchor_decode_backward(int64_t n, const double *pos, const int32_t *level, const double *feat,
                               const double *log_l, const double *offs, const double *w, const double cam_c[3],
                               const double *max_dist, const double *g_rows, double *g_feat, double *g_log_l,
                               double *g_offs, double *g_w, int32_t bf16, double *dz_out, double *dp_out) {
    /* bf16: the plain FP64 chain rule of the bf16 forward (a rounded operand's
     * product differentiated with the rounded factor, nothing rounded here) */
    for (int64_t i = 0; i < n; ++i) {
        double x[OR_ANC_IN], pre[OR_ANC_H], z[OR_ANC_OUT], d, dz[OR_ANC_OUT];
        anchor_mlp(pos + 3 * i, feat + OR_ANC_F * i, w, cam_c, x, pre, z, &d, bf16);
        const int M = lod_active(level[i], d, max_dist);
        const double *L = log_l + 3 * i;
        for (int o = 0; o < OR_ANC_OUT; ++o) dz[o] = 0.0;
        for (int k = 0; k < OR_ANC_K; ++k) {
            const double *zk = z + 14 * k;
            const double a = tanh(zk[3]);
            if (!(M && a > 0.0)) continue;  /* dropped Gaussians pass no gradient */
            const double *g = g_rows + 14 * (k * n + i);
            double *dk = dz + 14 * k;
            for (int c = 0; c < 3; ++c) {
                const double l = exp(L[c]);
                const double O = offs[(OR_ANC_K * i + k) * 3 + c] + zk[11 + c];
                dk[11 + c] = g[c] * l;                                  /* offset */
                g_offs[(OR_ANC_K * i + k) * 3 + c] += g[c] * l;
                g_log_l[3 * i + c] += g[c] * O * l + g[3 + c];          /* mean and log-scale */
                dk[8 + c] = g[3 + c] * (1.0 - sigm(zk[8 + c]));         /* d log(sigmoid) */
                const double sc = sigm(zk[c]);
                dk[c] = g[11 + c] * sc * (1.0 - sc) / OR_Y00;           /* colour */
            }
            for (int c = 0; c < 4; ++c) dk[4 + c] = g[6 + c];           /* rotation */
            dk[3] = g[10] * (1.0 + a) / a;  /* d logit(tanh z) / dz = (1 - a^2) / (a (1 - a)) */
        }
        if (dz_out)
            for (int o = 0; o < OR_ANC_OUT; ++o) dz_out[OR_ANC_OUT * i + o] = dz[o];
        double dh[OR_ANC_H];
        for (int c = 0; c < OR_ANC_H; ++c) dh[c] = 0.0;
        for (int o = 0; o < OR_ANC_OUT; ++o) {
            if (dz[o] == 0.0) continue;
            g_w[OR_ANC_B2 + o] += dz[o];
            for (int c = 0; c < OR_ANC_H; ++c) {
                const double h = pre[c] > 0.0 ? pre[c] : 0.0, wv = w[OR_ANC_W2 + o * OR_ANC_H + c];
                g_w[OR_ANC_W2 + o * OR_ANC_H + c] += dz[o] * (bf16 ? bf16_round(h) : h);
                dh[c] += dz[o] * (bf16 ? bf16_round(wv) : wv);
            }
        }
        for (int c = 0; c < OR_ANC_H; ++c) {
            const double dp = pre[c] > 0.0 ? dh[c] : 0.0;
            if (dp_out) dp_out[OR_ANC_H * i + c] = dp;
            if (dp == 0.0) continue;
            g_w[OR_ANC_B1 + c] += dp;
            for (int m = 0; m < OR_ANC_IN; ++m) {
                const double wv = w[OR_ANC_W1 + c * OR_ANC_IN + m];
                g_w[OR_ANC_W1 + c * OR_ANC_IN + m] += dp * x[m];  /* x rounded in bf16 mode */
                if (m < OR_ANC_F) g_feat[OR_ANC_F * i + m] += dp * (bf16 ? bf16_round(wv) : wv);
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Spatial order of the rows (a memory layout, not a step of the method)      */
/* ------------------------------------------------------------------------ */

/* The Morton (Z-) order of the means as the library defines it, written with
 * plain loops: the bounding box, one scale 1024 / (largest extent), 1024
 * cells per axis, the cell indices' bits interleaved with x lowest, then a
 * sort by code with ties in row order.  FP32, because the library takes the
 * cell decision in FP32 (each operation rounded once, as here). */
typedef struct {
    uint32_t code;
    int64_t row;
} or_code_row;

static int cmp_code_row(const void *a, const void *b) {
    const or_code_row *x = (const or_code_row *)a, *y = (const or_code_row *)b;
    if (x->code != y->code) return x->code < y->code ? -1 : 1;
    return x->row < y->row ? -1 : (x->row > y->row);
}

void or_morton_order(int64_t n, const float *means, uint32_t *codes, int32_t *perm) {
    if (n <= 0) return;
    float lo[3], hi[3];
    for (int a = 0; a < 3; ++a) lo[a] = hi[a] = means[a];
    for (int64_t i = 1; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            const float m = means[3 * i + a];
            if (m < lo[a]) lo[a] = m;
            if (m > hi[a]) hi[a] = m;
        }
    float ext = 0.0f;
    for (int a = 0; a < 3; ++a) {
        const float e = hi[a] - lo[a];
        if (e > ext) ext = e;
    }
    const float scale = (ext > 0.0f && ext <= FLT_MAX) ? 1024.0f / ext : 0.0f;
    or_code_row *cr = (or_code_row *)malloc(sizeof(or_code_row) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t code = 0;
        for (int a = 0; a < 3; ++a) {
            const float t = (means[3 * i + a] - lo[a]) * scale;
            const int q = t >= 1023.0f ? 1023 : (t > 0.0f ? (int)t : 0);
            for (int b = 0; b < 10; ++b) code |= (uint32_t)((q >> b) & 1) << (3 * b + a);
        }
        cr[i].code = code;
        cr[i].row = i;
        if (codes) codes[i] = code;
    }
    qsort(cr, (size_t)n, sizeof(or_code_row), cmp_code_row);
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)cr[i].row;
    free(cr);
}
