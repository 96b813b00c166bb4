/*
 * gs_oracle.h -- interface of the FP64 CPU oracle of the differentiable
 * 3D Gaussian splatting mapping step.
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle is loaded by the test-suite, by the
 * package's smoke check and by the benchmark's CPU-baseline leg.  Nothing on the
 * product path links, imports or calls it, and it shares no code with the CUDA
 * sources: every formula below is written out again from the mathematics.
 *
 * Conventions (the readings the paper leaves open; see the header of
 * gs_oracle.c for the list):
 *   - parameters are array-of-structures FP64: means n*3, log_scales n*3,
 *     quats n*4 (w,x,y,z, unnormalised), opacity_logits n, sh n*(D+1)^2*3
 *     (coefficient-major, RGB-minor);
 *   - the camera maps world to camera frame, x right, y down, z forward;
 *     pixel (i, j) samples the continuous image point (i + 0.5, j + 0.5);
 *   - images are planar [3][H][W].
 */
#ifndef GS_ORACLE_H
#define GS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double R[9];            /* world -> camera rotation, row-major */
    double t[3];            /* world -> camera translation */
    double fx, fy, cx, cy;  /* pinhole intrinsics in pixels */
    int32_t width, height;
} or_camera;

typedef struct {
    int32_t tile_w, tile_h;
    double near_z;          /* cull z <= near_z */
    double dilation;        /* added to the diagonal of the 2D covariance */
    double alpha_min;       /* skip alpha < alpha_min */
    double alpha_max;       /* clamp alpha to alpha_max */
    double t_min;           /* stop before blending when T*(1-alpha) < t_min */
    double tan_clamp;       /* EWA Jacobian evaluated at x/z clamped to tan_clamp * W/(2 fx) */
    double bg[3];           /* background colour */
    int32_t fp32_positions; /* 1: u, v, z and the tile rectangle follow the FP32
                               evaluation order (bit-identical on every IEEE
                               implementation); 0: plain FP64 throughout */
} or_cfg;

typedef struct {
    int64_t n;
    int32_t sh_degree;
    const double *means, *log_scales, *quats, *opacity_logits, *sh;
} or_params;

/* Per-Gaussian projection record (caller-allocated arrays of n entries). */
typedef struct {
    double *u, *v, *z;       /* pixel position and camera depth used for rendering */
    double *conic;           /* n*3: (a, b, c), inverse of the dilated 2D covariance */
    double *cov2d;           /* n*3: (A, B, C), the dilated 2D covariance */
    double *rgb;             /* n*3: colour after the clamp at 0 */
    int32_t *rgb_clamped;    /* n*3: 1 where the clamp at 0 was active */
    double *rgb_raw;         /* n*3: colour before the clamp */
    double *opacity;         /* n */
    int32_t *radius;         /* n: integer pixel radius, 0 = culled */
    double *radius_exact;    /* n: 3*sqrt(lambda_max) before the ceiling */
    int32_t *rect;           /* n*4: tile rectangle xmin, ymin, xmax, ymax (max exclusive) */
    int32_t *tiles_touched;  /* n */
    float *u32, *v32, *z32;  /* n: the FP32 evaluation of u, v and camera depth */
} or_projected;

/* Real spherical harmonics of degree <= D at unit direction d; Y gets (D+1)^2
 * values, dY (nullable) the (D+1)^2 x 3 partial derivatives with respect to the
 * three Cartesian components of d. */
void or_sh_eval(int32_t D, const double d[3], double *Y, double *dY);

/* Quaternion (w,x,y,z), normalised inside, to a row-major rotation matrix. */
void or_quat_to_rot(const double q[4], double R[9]);

void or_project(const or_params *p, const or_camera *cam, const or_cfg *cfg, or_projected *out);

/* Pair list: one (key, Gaussian) entry per overlapped tile, ordered by
 * (tile, depth, Gaussian index).  Returns the number of pairs; arrays are
 * written only if capacity suffices.  ranges gets [tiles][2] = start, end. */
int64_t or_bin(const or_projected *pr, int64_t n, const or_camera *cam, const or_cfg *cfg,
               int64_t capacity, uint64_t *keys, int32_t *vals, int64_t *ranges);

/* Pixel flags returned by or_render. */
#define OR_FLAG_NEAR_ALPHA_MIN 1
#define OR_FLAG_NEAR_T_CUT     2
#define OR_FLAG_NEAR_ALPHA_MAX 4

void or_render(const or_projected *pr, const int32_t *vals, const int64_t *ranges,
               const or_camera *cam, const or_cfg *cfg,
               double *img, double *depth, double *T_final, int32_t *n_contrib,
               int64_t *last_pos, int32_t *flags);

/* Photometric loss (1-lambda)*L1 + lambda*(1-SSIM); returns the loss, writes
 * dL/dimg (nullable) and the mean SSIM (nullable). */
double or_loss(const double *img, const double *target, int32_t C, int32_t H, int32_t W,
               double lambda_dssim, double *dL_dimg, double *ssim_mean);

/* SSIM map (nullable outputs) of two planar images. */
void or_ssim_map(const double *x, const double *y, int32_t C, int32_t H, int32_t W, double *map);

/* Backward of the compositing for one view.  grad2d gets n*10 values per
 * Gaussian: dL/d(u, v, conic a, b, c, opacity, r, g, b, z) (accumulated).
 * stats (nullable) gets n*6 accumulators: |Omega|, kappa, gamma, max T*alpha,
 * ||dL/d(u,v)|| of this view, view count; kappa_amb (nullable) counts, per
 * Gaussian, footprint pixels whose error-mask decision lies within
 * mask_tol of tau_err. */
void or_render_backward(const or_projected *pr, int64_t n, const int32_t *vals, const int64_t *ranges,
                        const or_camera *cam, const or_cfg *cfg,
                        const double *dL_dimg, const double *dL_ddepth,
                        const double *img, const double *target, double tau_err, double loss_v,
                        double mask_tol, double *grad2d, double *stats, double *kappa_amb);

/* Chain rule from grad2d to the parameters (accumulated into grads, same
 * layout as the parameters). */
void or_project_backward(const or_params *p, const or_camera *cam, const or_cfg *cfg,
                         const or_projected *pr, const double *grad2d,
                         double *g_means, double *g_log_scales, double *g_quats,
                         double *g_opacity_logits, double *g_sh);

/* Bias-corrected Adam, element-wise with a per-element learning rate. */
void or_adam(int64_t n, double *p, const double *g, double *m, double *v, const double *lr,
             double beta1, double beta2, double eps, int64_t step);

/* Chunk scores and global decisions.  densify and prune_max are updated in
 * place (OR and max over chunks); prune is recomputed from prune_max. */
void or_prune_finalize(int64_t n, const double *omega, const double *kappa, const double *gamma,
                       int32_t n_views, double tau_d, double tau_p,
                       double *S_d, double *S_p, uint8_t *densify, double *prune_max,
                       uint8_t *prune);

/* Geometric term: mean over pixels of [prior > 0] |prior - depth| (Supp. D.4). */
double or_geo_loss(const double *depth, const double *prior, int64_t npx, double *dL_ddepth);

/* Isotropic term: mean over Gaussians of sum_k |s_k - mean(s)|, s = exp(log-scale)
 * (Supp. D.4); gradient added into g_log_scales (nullable). */
double or_iso_loss(int64_t n, const double *log_scales, double *g_log_scales);

/* Learned prune / densify MLP 16 -> 64 -> 64 -> 2 (ReLU, sigmoid outputs);
 * weights W1[64][16], b1[64], W2[64][64], b2[64], W3[2][64], b3[2] in one array. */
int32_t or_mlp_num_weights(void);
void or_mlp_forward(int64_t n, const double *x, const double *w, int32_t bf16, double *p, double *h1, double *h2);
double or_mlp_bce_grad(int64_t n, const double *x, const double *y, const double *w, int32_t bf16, double *g,
                       double *dh2, double *dh1);

/* The predictor's 16 inputs per Gaussian (a reading: the inputs are named in
 * the workload definition, not in the paper): sigmoid(opacity logit), the
 * three log-scales, log(1 + views seen), log(1 + 1e4 * accumulated
 * ||dL/d(u,v)||), the max blend weight T*alpha of the last 8 views (ring
 * slots head, head-1, ... mod 8), log(1 + ||mu - c||) for the camera centre
 * c, log(1 + mean |Omega_v| over the views seen).  stats[n][6] in the order
 * of or_render_backward; ring[8][n]; feat[n][16]. */
void or_mlp_features(int64_t n, const double *means, const double *log_scales, const double *opacity_logits,
                     const double *stats, const double *ring, int32_t head, const double cam[3], double *feat);

/* Densify / prune actions on explicit Gaussians (Sec. 3.3.2 decisions
 * applied per Gaussian; the clone / split rule is a reading, the paper
 * spawns anchors).  Rows are [means 3, log-scales 3, quaternion 4, opacity
 * logit 1, SH 3K] (K_row values each).  Gaussian i emits, in source order:
 * nothing if prune[i]; itself if not densify[i]; else, when its largest
 * log-scale exceeds split_log_scale, two children mu + R S xi_j (xi_j =
 * noise[i][3j..3j+2], R S the covariance factor) with log-scales reduced by
 * log(split_factor), otherwise itself and an identical clone.  Moments m, v
 * (nullable, same rows) follow the survivor; clones and split children start
 * at zero.  Writes at most cap rows and returns the rows needed. */
int64_t or_densify_prune(int64_t n, int32_t K_row, const double *P, const double *m, const double *v,
                         const uint8_t *densify, const uint8_t *prune, const double *noise,
                         double split_log_scale, double split_factor, int64_t cap, double *P_out,
                         double *m_out, double *v_out);

/* Probabilistic initialisation of new anchors at a keyframe (Sec. 3.3.1,
 * Supp. D.5), readings R19-R24 of gs_oracle.c.
 *
 * or_init_saliency: dog[H][W] = min(scale |(G_s1 - G_s2) * Y|, 1) with Y the
 * mean of the three planes of img[3][H][W] (scale 255: 8-bit intensity
 * units for [0, 1] images) and G_s the sampled 2D Gaussian of
 * radius ceil(3 s) normalised to sum 1, borders replicated; grad[H][W] =
 * ||grad D|| by central differences, borders replicated. */
void or_init_saliency(int32_t H, int32_t W, const double *img, const double *depth, double sigma1,
                      double sigma2, double scale, double *dog, double *grad);

/* prob[H][W] = max(P - P_r, 0) with P = min(lambda dog + (1 - lambda)
 * minmax(grad), 1) of (img, depth) and P_r the same of (img_r, depth_r);
 * img_r / depth_r null together: P_r = 0. */
void or_init_probability(int32_t H, int32_t W, const double *img, const double *depth, const double *img_r,
                         const double *depth_r, double sigma1, double sigma2, double scale, double lambda,
                         double *prob);

/* Selection, unprojection and voxel insertion over the pixels in raster
 * order.  Pixel p is selected when prob[p] > 0 is the (value, -index)
 * lexicographic maximum of its 3x3 window, uniform[p] < prob[p] and
 * depth[p] > near_z; its point x_w = R^T (d ((u+0.5-cx)/fx, (v+0.5-cy)/fy, 1)
 * - t) goes to level l = first l with ||x_c|| < max_dist[l] (none: skipped),
 * voxel idx = floor(x_w / voxel[l]) (skipped unless -2^19 <= idx < 2^19).
 * Voxels are keyed (l, ix, iy, iz); old_keys [n_old][4] are occupied
 * already.  Each new voxel becomes an anchor in the order its first pixel is
 * met: the first cap of them get new_keys [cap][4], pos [cap][3] = idx *
 * voxel[l], level and pixel (v W + u).  Returns the number of new voxels
 * (may exceed cap).  selected[H][W] (nullable): 1 for selected pixels whose
 * point got a voxel.  uncertain[H][W] (nullable): 1 where a decision of the
 * pixel lies within tol of flipping (a neighbour within tol and none above
 * by more; the draw) or within tol_rel, relative, of a threshold (depth,
 * distance band, voxel boundary). */
int64_t or_init_select(int32_t H, int32_t W, const double *prob, const double *uniform, const double *depth,
                       const or_camera *cam, double near_z, int32_t levels, const double *voxel,
                       const double *max_dist, int64_t n_old, const int64_t *old_keys, int64_t cap,
                       int64_t *new_keys, double *pos, int32_t *level, int32_t *pixel, uint8_t *selected,
                       uint8_t *uncertain, double tol, double tol_rel);

/* Scaffold-GS anchor decoding (Supp. D.1, D.3), readings R25-R29 of
 * gs_oracle.c.  Anchors: pos[n][3] (fixed), level[n], feat[n][32],
 * log_l[n][3], offs[n][10][3]; decoder weights W1[64][36], b1[64],
 * W2[140][64], b2[140] in one array (or_anchor_num_weights()).  The
 * Gaussian k of anchor i is row k n + i of rows[10 n][14] = [mean 3,
 * log-scale 3, quaternion 4, opacity logit 1, sh0 3]; keep[10 n] (nullable)
 * marks the Gaussians not dropped (LoD band and opacity > 0); unsure[10 n]
 * (nullable) marks those whose keep decision is within tol (relative
 * distance to a band edge, |opacity pre-activation|). */
int32_t or_anchor_num_weights(void);
void or_anchor_decode(int64_t n, const double *pos, const int32_t *level, const double *feat, const double *log_l,
                      const double *offs, const double *w, const double cam_c[3], const double *max_dist,
                      double *rows, uint8_t *keep, uint8_t *unsure, double tol, int32_t bf16);
/* Accumulates into g_feat, g_log_l, g_offs and g_w the gradient of a loss
 * whose gradient with respect to rows is g_rows (same layout).  bf16 != 0
 * rounds the decoder's hidden-layer operands (input, W1, hidden activation,
 * W2) to bfloat16 in the forward; the backward is its plain FP64 chain rule.
 * dz_out[n][140] and dp_out[n][64] (nullable) receive each anchor's gradient
 * with respect to the decoder's outputs and hidden pre-activations. */
void or_anchor_decode_backward(int64_t n, const double *pos, const int32_t *level, const double *feat,
                               const double *log_l, const double *offs, const double *w, const double cam_c[3],
                               const double *max_dist, const double *g_rows, double *g_feat, double *g_log_l,
                               double *g_offs, double *g_w, int32_t bf16, double *dz_out, double *dp_out);
/* The decoder's input x_raw[n][36] before any rounding and its hidden
 * pre-activations pre[n][64] (bf16 as in or_anchor_decode); either
 * nullable.  Used to find the anchors whose bfloat16 roundings sit next to a
 * rounding midpoint. */
void or_anchor_hidden(int64_t n, const double *pos, const double *feat, const double *w, const double cam_c[3],
                      int32_t bf16, double *x_raw, double *pre);

/* Spatial order of the rows (a memory layout of the library, not a step of
 * the method): means[n][3] FP32; codes[n] (nullable) receive the 30-bit Morton
 * codes, perm[n] the rows in increasing code order, ties in row order.  Box
 * lo/hi per axis; scale = 1024 / max extent (0 if that is 0 or not finite);
 * q = 1023 if t >= 1023, (int) t if t > 0, else 0 with t = (m - lo) * scale;
 * bit b of q_x, q_y, q_z at 3b, 3b + 1, 3b + 2.  All arithmetic FP32. */
void or_morton_order(int64_t n, const float *means, uint32_t *codes, int32_t *perm);

#ifdef __cplusplus
}
#endif
#endif
