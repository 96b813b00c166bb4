/*
 * gs.h -- C ABI of the B300 (sm_103a) differentiable 3D Gaussian splatting
 * mapping step: projection, binning and depth sort, front-to-back
 * compositing, the photometric loss, the back-to-front backward, Adam and the
 * lifecycle (densify / prune) scores.
 *
 * Paper: KiloGS-SLAM, "Robust and Efficient Monocular 3D Gaussian SLAM for
 * Kilometer-Scale Outdoor Scenes".  The mapping step optimises the map inside
 * a sliding window with L_total = L_photo + ... (Sec. 3.2.3); the colour is
 * composited front to back over depth-sorted Gaussians with transmittance
 * T_j = prod_{m<j}(1 - alpha_m) (Supp. D.2); L_photo = 0.8 L1 + 0.2 (1 - SSIM)
 * (Supp. D.4); the per-Gaussian footprint statistics, the densification
 * score S_d and the pruning score S_p follow Supp. E.1 and E.2, aggregated
 * over chunks by OR and max (Sec. 3.3.2).
 *
 * General conventions
 *   - Every pointer in the structs and arguments below is a DEVICE pointer
 *     unless marked "host".  The caller owns every buffer; the library never
 *     allocates device memory and keeps no state between calls other than
 *     cached device properties.
 *   - All work is enqueued on the caller's stream; no call synchronises the
 *     host, so the sequence can be captured into a CUDA graph.  Counts that
 *     are only known on the device (visible records, pairs) stay on the device.
 *   - Synchronous argument errors return a gs_status and enqueue nothing.
 *     Asynchronous conditions (pair-buffer overflow, non-finite values) are
 *     OR-ed as bit (1 << status) into the caller's device int32 status word,
 *     read by the caller after the stream completes.
 *   - Float buffers must be 16-byte aligned (GS_ERR_INVALID otherwise).
 *   - Images are planar [3][H][W] FP32 per view; views are packed back to back
 *     in the order of the camera array ("frame layout").
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID = 1,   /* bad argument: null, misaligned, out of range */
    GS_ERR_CUDA = 2,      /* a CUDA launch or copy failed */
    GS_ERR_CAPACITY = 3,  /* device: more (Gaussian, tile) pairs than max_pairs */
    GS_ERR_TIMEOUT = 4,   /* device: a bounded wait gave up */
    GS_ERR_NUMERIC = 5    /* device: a non-finite projection was culled */
} gs_status;

#define GS_MAX_VIEWS 64

/* Pinhole camera (host struct).  x_c = R x_w + t, x right, y down, z forward;
 * u = fx x_c/z_c + cx, v = fy y_c/z_c + cy; pixel (i, j) samples (i+0.5, j+0.5). */
typedef struct {
    float R[9];     /* world -> camera rotation, row-major */
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
} gs_camera;

/* Rasteriser constants (host struct).  The paper does not print them; these
 * are the standard EWA-splatting values of the 3DGS work it builds on. */
typedef struct {
    int32_t tile_w, tile_h; /* 16x16, 8x32 or 32x8 (tile_w * tile_h == 256) */
    float near_z;           /* cull camera depth <= near_z (0.2) */
    float dilation;         /* added to the 2D covariance diagonal (0.3) */
    float alpha_min;        /* skip alpha < alpha_min (1/255) */
    float alpha_max;        /* clamp alpha to alpha_max (0.99) */
    float t_min;            /* stop before blending when T (1 - alpha) < t_min (1e-4) */
    float tan_clamp;        /* EWA Jacobian taken at x/z clamped to tan_clamp * W/(2 fx) (1.3) */
    float bg[3];            /* background colour */
    int32_t batch;          /* pairs a warp scans per step in the compositing
                               kernels: 128, 256 or 512 (0 selects 512); a
                               tuning knob only, results do not depend on it */
    int32_t segment;        /* 0, or a power of two 32..65536: the pair list of a
                               tile longer than `segment` pairs is composited in
                               segments of that many pairs, one warp per segment
                               and 8x4 block: the forward composites each segment
                               from T = 1, chains the segments (T_start = product
                               of the earlier segments' T, C += T_start C_s) and
                               composites again, from the chained state, the one
                               segment where a pixel stops; the backward walks
                               each segment from the state recorded at its end.
                               Needs gs_frame.seg_ws.  Results equal the unsplit
                               traversal up to FP32 rounding */
} gs_raster_cfg;

/* Gaussian parameters: ONE device buffer of K planes of ld floats
 * (plane-major, so every attribute component streams contiguously):
 *   planes 0-2   mean x, y, z (world)
 *   planes 3-5   log-scale x, y, z
 *   planes 6-9   rotation quaternion w, x, y, z (need not be normalised)
 *   plane  10    opacity logit
 *   plane  11 + 3k + c   SH coefficient k in 0..(D+1)^2-1 of colour channel c
 * K = 11 + 3 (D+1)^2, D = sh_degree in 0..3, ld >= n and a multiple of 4.
 * Gradients and Adam moments use the same layout. */
typedef struct {
    float *data;
    int64_t n;
    int64_t ld;
    int32_t sh_degree;
} gs_params;

#define GS_PLANES(D) (11 + 3 * ((D) + 1) * ((D) + 1))

/* Per-view projection records, [n_views][ld] each (record index = view*ld + g). */
typedef struct {
    float *xy;            /* 2 floats: pixel position u, v */
    float *conic_opacity; /* 4 floats: conic a, b, c (inverse 2D covariance), opacity */
    float *rgb_depth;     /* 4 floats: colour r, g, b, camera depth z */
    int32_t *radius;      /* pixel radius, 0 = culled */
    int32_t *tiles_touched;
    int64_t ld;
    /* Optional (NULL = not kept), used only when sh_degree >= 1: 12 floats per
     * record, 16-byte aligned, per colour channel c at [12*rec + 4c]: the
     * gradient of that channel's unclamped SH colour (Eq. 1's view-dependent
     * colour) with respect to the mean through the view direction, then 1 if
     * the channel was kept by the clamp at 0 and 0 if clamped.  gs_project
     * writes it for every record with radius > 0; a backward given it reads
     * it instead of the SH coefficients, so it must come from the gs_project
     * call on the same parameters. */
    float *color_jac;
} gs_projected;

/* Pair list and tile ranges of all views.  Tiles of all views form one
 * global index space: view v's tile (tx, ty) is tile_offset[v] + ty*GW_v + tx
 * with tile_offset the running sum of GW*GH over the previous views. */
typedef struct {
    int32_t *gauss_ids;    /* [max_pairs] record index per pair, ordered by
                              (tile, depth, Gaussian index) */
    int32_t *tile_ranges;  /* [total_tiles][2] = first pair, one past the last */
    int32_t *counts;       /* device int32[4]: visible records, pairs written,
                              pairs needed, records covering more than 128 tiles */
    uint8_t *block_mask;   /* [gs_block_mask_size(max_pairs) bytes], 16-byte aligned:
                              per pair, bit b set when the Gaussian's alpha >=
                              alpha_min ellipse can reach the tile's 8x4 pixel
                              block b (blocks row-major, tile_w/8 per row); a
                              clear bit proves alpha < alpha_min on that block */
    int32_t *tile_order;   /* [total_tiles] the tiles ordered by decreasing pair
                              count (power-of-two classes): the order in which the
                              compositing kernels start them */
    int64_t max_pairs;
} gs_binning;

/* Rendered frame of all views (frame layout). */
typedef struct {
    float *img;       /* [sum_v 3 H_v W_v] colour */
    float *T_final;   /* [sum_v H_v W_v] transmittance left after the last blended Gaussian */
    int32_t *last;    /* [sum_v H_v W_v] pairs of the tile consumed up to and including
                         the last blended one (0 = none) */
    float *depth;     /* nullable: [sum_v H_v W_v] D^ = sum_j T_j alpha_j z_j (Supp. D.2) */
    void *seg_ws;     /* split workspace, gs_segment_workspace_size bytes (256-byte
                         aligned, sized for binning->max_pairs); written by
                         gs_render_fwd, read by gs_render_bwd; required when
                         cfg->segment > 0, else ignored */
    size_t seg_ws_bytes;
} gs_frame;

/* Per-Gaussian lifecycle accumulators, planes of ld floats, accumulated over
 * views and calls until the caller zeroes them (once per chunk):
 *   0 |Omega| summed over views   1 kappa summed over views
 *   2 gamma = sum_v L_photo^(v) |Omega_v|   3 max over views of max T*alpha
 *   4 sum over views of ||dL/d(u,v)||       5 views with |Omega_v| > 0 */
typedef struct {
    float *acc;
    int64_t ld;
} gs_stats;

/* Chunk outputs of gs_prune_stats (planes of n). */
typedef struct {
    float *S_d;          /* densification score of this chunk (Supp. E.1) */
    float *S_p;          /* pruning score of this chunk (Supp. E.2) */
    float *prune_max;    /* running max of S_p over chunks (in/out) */
    uint8_t *densify;    /* running OR over chunks of S_d > tau_d (in/out) */
    uint8_t *prune;      /* prune_max > tau_p */
} gs_chunk_scores;

typedef void *gs_stream; /* a cudaStream_t; NULL = legacy default stream */

const char *gs_status_string(gs_status s);

/* Library version and the device architecture it was built for (e.g. 1030). */
int32_t gs_version(void);

/* Total tiles of all views and, per view (host outputs, nullable), the tile
 * offset, the pixel offset of the view in the frame layout, GW and GH. */
gs_status gs_view_layout(const gs_camera *cams, int32_t n_views, const gs_raster_cfg *cfg,
                         int64_t *total_tiles, int64_t *total_pixels, int64_t *tile_offset,
                         int64_t *pixel_offset);

/* Workspace bytes of gs_sort for n_records = n_views * ld records and
 * max_pairs pairs. */
gs_status gs_sort_workspace_size(int64_t n_records, int64_t max_pairs, size_t *bytes);

/* Bytes of gs_binning.block_mask for max_pairs pairs. */
gs_status gs_block_mask_size(int64_t max_pairs, size_t *bytes);

/* Workspace bytes of gs_loss for a view of h x w pixels (the largest view). */
gs_status gs_loss_workspace_size(int32_t h, int32_t w, size_t *bytes);

/* Bytes of gs_frame.seg_ws.  A long tile (more than `segment` pairs) needs
 * 8 x S segment items (S = its segments), each about 1.45 KB (the forward's
 * local state, a re-run slot and the backward's checkpoint).  The capacities
 * follow from the bytes given: gs_segment_workspace_size covers the worst case
 * for max_pairs (every pair in a long tile), gs_segment_workspace_size_items a
 * measured item count.  When a launch needs more items than fit, the split is
 * off for that launch (every block walks its whole list: same results,
 * slower) and the item count it needed is left in the workspace's int32 at
 * byte offset 20 (the int32 at offset 16 is 1), for the caller to resize. */
gs_status gs_segment_workspace_size(int64_t max_pairs, int32_t segment, size_t *bytes);
gs_status gs_segment_workspace_size_items(int64_t items, size_t *bytes);

/* Workspace bytes of gs_render_bwd for n_records records. */
gs_status gs_bwd_workspace_size(int64_t n_records, size_t *bytes);

/* Workspace bytes of gs_prune_stats. */
gs_status gs_prune_workspace_size(int64_t n, size_t *bytes);

/*
 * Projection of every Gaussian into every view (EWA splatting; the paper
 * relies on the cited 3DGS rasteriser for it, Sec. 3.2 / Supp. D.2):
 * camera point, near cull, Sigma = R(q) S S^T R(q)^T, Sigma' = J W Sigma W^T
 * J^T + dilation I, conic, radius = ceil(3 sqrt(lambda_max)), tile rectangle,
 * SH colour max(0, sum_k sh_k Y_k(dir) + 0.5) and sigmoid opacity.  u, v and
 * the camera depth are evaluated in FP32 with each product, sum and quotient
 * rounded left to right (no contraction), which makes the binning exactly
 * reproducible.  cams is a HOST array of n_views <= GS_MAX_VIEWS cameras.
 * status (nullable device int32) gets bit 1<<GS_ERR_NUMERIC when a
 * non-finite projection was culled.
 */
gs_status gs_project(const gs_params *params, const gs_camera *cams, int32_t n_views,
                     const gs_raster_cfg *cfg, const gs_projected *out, int32_t *status,
                     gs_stream stream);

/*
 * Binning: one pair per (visible record, overlapped tile), ordered by
 * (global tile, camera depth, Gaussian index) -- the "sorted Gaussians along
 * the ray" of Supp. D.2 -- and the per-tile ranges.  Writes
 * binning->counts, gauss_ids[0..pairs), block_mask[0..pairs), tile_ranges
 * and tile_order (cfg->alpha_min sets the masks).  When the pairs
 * exceed max_pairs, no pair is written, counts[1] = 0, counts[2] = pairs
 * needed and status gets bit 1<<GS_ERR_CAPACITY.  ws: gs_sort_workspace_size
 * bytes (256-byte aligned).
 */
gs_status gs_sort(const gs_projected *proj, const gs_camera *cams, int32_t n_views,
                  const gs_raster_cfg *cfg, const gs_binning *binning, void *ws, size_t ws_bytes,
                  int32_t *status, gs_stream stream);

/*
 * Front-to-back alpha compositing of every pixel of every view (Supp. D.2):
 * C = sum_j c_j alpha_j T_j + T_final bg, T_j = prod_{m<j} (1 - alpha_m),
 * alpha_j = min(alpha_max, o_j exp(power_j)); Gaussians with alpha < alpha_min
 * are skipped and the pixel stops before the Gaussian that would take T below
 * t_min.  Writes the frame (depth only if frame->depth is set).
 */
gs_status gs_render_fwd(const gs_projected *proj, const gs_binning *binning, const gs_camera *cams,
                        int32_t n_views, const gs_raster_cfg *cfg, const gs_frame *frame,
                        gs_stream stream);

/*
 * Photometric loss per view (Supp. D.4):
 *   L_v = (1 - lambda) mean|I^ - I| + lambda (1 - mean SSIM(I^, I)),
 * lambda = lambda_dssim (0.2 in the paper), SSIM with an 11x11 Gaussian window
 * (sigma 1.5), zero padding, C1 = 0.01^2, C2 = 0.03^2, mean over the three
 * channels and all pixels.  img, target and dL_dimg are in frame layout;
 * loss_per_view gets n_views floats; dL_dimg gets dL_v/dI^.  ws:
 * gs_loss_workspace_size of the largest view.
 */
gs_status gs_loss(const float *img, const float *target, const gs_camera *cams, int32_t n_views,
                  float lambda_dssim, float *loss_per_view, float *dL_dimg, void *ws,
                  size_t ws_bytes, gs_stream stream);

/* Workspace bytes of gs_geo_loss and gs_iso_loss. */
gs_status gs_reg_workspace_size(size_t *bytes);

/*
 * Geometric term of L_total (Sec. 3.2.3; Supp. D.4 L_geo = ||D - D^||_1)
 * per view: weight * mean over the view's pixels of [D > 0] |D - D^|, D the
 * metric-depth prior (0 marks a pixel without one), D^ the rendered depth
 * (gs_frame.depth).  Writes weight * L_geo into loss_per_view[v] and
 * weight * dL_geo/dD^ into dL_ddepth (nullable), both in frame layout; pass
 * dL_ddepth to gs_render_bwd.  weight is lambda_g (0.01, Supp. F).
 */
gs_status gs_geo_loss(const float *depth, const float *prior, const gs_camera *cams, int32_t n_views,
                      float weight, float *loss_per_view, float *dL_ddepth, void *ws, size_t ws_bytes,
                      gs_stream stream);

/*
 * Isotropic term of L_total (Supp. D.4 L_iso = sum_i ||s_i - mean(s_i) 1||_1,
 * taken as a mean over the n Gaussians, s = exp(log-scale)): writes
 * weight * L_iso into *loss and ADDS weight * dL_iso/dlog-scale into the
 * log-scale planes of grads (nullable).  weight is lambda_iso (10, Supp. F).
 */
gs_status gs_iso_loss(const gs_params *params, float weight, float *loss, const gs_params *grads, void *ws,
                      size_t ws_bytes, gs_stream stream);

/*
 * gs_loss without a caller workspace.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory where
 * they need the loss -- code running while its allocator is unavailable
 * (a host callback, a memory-capped process whose budget another component
 * owns) or a plain C host that only receives the image and gradient pointers
 * from its framework.  Same arguments, arithmetic and outputs as gs_loss; the
 * scratch is a file-scope device array of the library (about 33 MB, held by
 * every GPU that loads the library until the process exits), which bounds
 * each view to at most 1280*720 pixels with width and height <= 2048;
 * larger views return GS_ERR_INVALID before anything is enqueued.  The first
 * call in a device's context looks up the array's device address (with that
 * device current) and caches it under the context, so make that first call
 * before any stream capture; a new context on the device (after a reset of
 * the primary context) gets its own lookup on its first call.  Every call
 * shares the device's copy of the array and leaves its last contents there;
 * calls that overlap on the same device (other streams, other threads) race
 * on it.  It never calls cudaMalloc, cudaFree or an allocating library routine.
 */
gs_status gs_loss_static(const float *img, const float *target, const gs_camera *cams, int32_t n_views,
                         float lambda_dssim, float *loss_per_view, float *dL_dimg, gs_stream stream);

/*
 * Backward of compositing and projection: traverses each tile back to front
 * from the pixel's last blended pair, recovers T_j = T_{j+1} / (1 - alpha_j),
 * and accumulates dL/d(u, v, conic, opacity, colour, depth) per record into
 * the workspace; then chains through the projection to every parameter plane
 * (as gs_project_bwd).  grads (same layout as params) is overwritten, or
 * accumulated into when accumulate != 0; with grads = NULL only the
 * compositing half runs and the per-record gradients stay in ws, record
 * major: record r's value p at float index r * 16 + p, values dL/du, dL/dv,
 * dL/da, dL/db, dL/dc, dL/dopacity, dL/dr, dL/dg, dL/db, dL/dz, |Omega_v|,
 * kappa_v, max T*alpha (p = 0..12; 13..15 unused).
 * dL_ddepth is nullable.  stats (nullable) receives the lifecycle
 * accumulators (Supp. E.1, E.2): per pixel the error mask
 * M_v = [sum_c |I - I^| > tau_err] (tau_err = 0.1, Supp. F) with the
 * rendered frame->img and target, and gamma uses loss_per_view.
 * ws: gs_bwd_workspace_size bytes.
 */
gs_status gs_render_bwd(const gs_params *params, const gs_camera *cams, int32_t n_views,
                        const gs_raster_cfg *cfg, const gs_projected *proj,
                        const gs_binning *binning, const gs_frame *frame, const float *dL_dimg,
                        const float *dL_ddepth, const float *target, const float *loss_per_view,
                        float tau_err, const gs_params *grads, int32_t accumulate,
                        const gs_stats *stats, void *ws, size_t ws_bytes, gs_stream stream);

/*
 * Stored per-pixel lists, the alternative to recomputing the blending in the
 * backward (the backward of the compositing sum of Supp. D.2 either way).
 * gs_render_fwd_lists renders exactly as gs_render_fwd without the split of
 * long tile lists (frame->seg_ws is not used) and records, per pixel of the
 * frame layout (views back to back), the record id and alpha of every
 * Gaussian the pixel blends, front to back: list_offsets [total_pixels + 1]
 * int64 (device, 8-byte aligned) gets each pixel's first slot and, at
 * [total_pixels], the number of blend events; list_ids (int32) and
 * list_alpha (float) [list_capacity] get the events.  When the events exceed
 * list_capacity, status gets bit 1<<GS_ERR_CAPACITY, only the slots below the
 * capacity are written, and the count at list_offsets[total_pixels] tells
 * the caller what to allocate.  ws: gs_list_workspace_size bytes (256-byte
 * aligned).  Memory: 8 bytes per blend event and 8 per pixel, against none
 * for gs_render_bwd's recompute.
 */
gs_status gs_list_workspace_size(int64_t total_pixels, size_t *bytes);
gs_status gs_render_fwd_lists(const gs_projected *proj, const gs_binning *binning, const gs_camera *cams,
                              int32_t n_views, const gs_raster_cfg *cfg, const gs_frame *frame, int64_t *list_offsets,
                              int32_t *list_ids, float *list_alpha, int64_t list_capacity, void *ws, size_t ws_bytes,
                              int32_t *status, gs_stream stream);

/*
 * Backward of compositing from the stored lists, then through the projection
 * as gs_render_bwd (same outputs, same workspace layout): one thread per
 * pixel walks its events from the back, T_j = T_{j+1} / (1 - alpha_j) from
 * the stored alpha, the colour behind carried; alpha below alpha_max counts
 * as unclamped (exp(power) = alpha / opacity).  No depth term.  The lists
 * must come from a gs_render_fwd_lists call of the same frame that did not
 * overflow.
 */
gs_status gs_render_bwd_lists(const gs_params *params, const gs_camera *cams, int32_t n_views,
                              const gs_raster_cfg *cfg, const gs_projected *proj, const gs_frame *frame,
                              const int64_t *list_offsets, const int32_t *list_ids, const float *list_alpha,
                              int64_t list_capacity, const float *dL_dimg, const float *target,
                              const float *loss_per_view, float tau_err, const gs_params *grads, int32_t accumulate,
                              const gs_stats *stats, void *ws, size_t ws_bytes, gs_stream stream);

/*
 * The projection half of gs_render_bwd: chain rule from the per-record
 * screen-space gradients in ws (left by gs_render_bwd with grads = NULL)
 * through colour (SH), opacity, the EWA covariance and the pinhole
 * projection to every parameter plane; folds the lifecycle statistics into
 * stats (nullable) as gs_render_bwd does.
 */
gs_status gs_project_bwd(const gs_params *params, const gs_camera *cams, int32_t n_views,
                         const gs_raster_cfg *cfg, const gs_projected *proj, const void *ws, size_t ws_bytes,
                         const float *loss_per_view, const gs_params *grads, int32_t accumulate,
                         const gs_stats *stats, gs_stream stream);

/*
 * gs_project_bwd (accumulate = 0) that writes only the gradient rows of the
 * Gaussians some view sees: rows[g] (device, [grads->ld] bytes, 4-byte
 * aligned) becomes 1 for those and 0 for every other row (padding included),
 * whose gradient is zero and whose grads entries are left as they were.  For
 * gs_adam_rows, which reads such a row's gradient as zero: the pair moves
 * 8 bytes less per parameter element of the Gaussians no view sees.
 */
gs_status gs_project_bwd_rows(const gs_params *params, const gs_camera *cams, int32_t n_views,
                              const gs_raster_cfg *cfg, const gs_projected *proj, const void *ws,
                              size_t ws_bytes, const float *loss_per_view, const gs_params *grads,
                              const gs_stats *stats, uint8_t *rows, gs_stream stream);

/*
 * gs_project_bwd followed by gs_adam without the gradient buffer: each
 * Gaussian's gradient (the projection chain from the per-record gradients in
 * ws, plus grads_in when set, plus the isotropic term's gradient
 * iso_weight / n * dL_iso/dlog-scale when iso_weight > 0, Supp. D.4) is applied
 * at once as one Adam step to params, exp_avg and exp_avg_sq, with the rates,
 * betas, eps and step rules of gs_adam.  Saves writing and re-reading the
 * gradient (8 bytes per parameter element).  stats as gs_project_bwd.
 */
gs_status gs_project_bwd_adam(const gs_params *params, const gs_camera *cams, int32_t n_views,
                              const gs_raster_cfg *cfg, const gs_projected *proj, const void *ws,
                              size_t ws_bytes, const float *loss_per_view, const gs_params *grads_in,
                              float iso_weight, const gs_params *exp_avg, const gs_params *exp_avg_sq,
                              const float lr_groups[6], float beta1, float beta2, float eps, int64_t step,
                              const int64_t *step_device, const gs_stats *stats, gs_stream stream);

/*
 * Adam (Kingma & Ba) with bias correction over every parameter plane, dense:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr m^ / (sqrt(v^) + eps),
 * m^ = m/(1-b1^step), v^ = v/(1-b2^step).  lr_groups (host) holds six rates:
 * means, log-scales, quaternion, opacity, SH degree 0, SH degree >= 1.
 * step_device (nullable device int64): when set, the step count is read from
 * it when the kernel runs and `step` is ignored, so a captured CUDA graph can
 * replay the update with a counter the caller advances.
 * The paper trains in PyTorch and prints no optimiser settings (Sec. 4.1).
 */
gs_status gs_adam(const gs_params *params, const gs_params *grads, const gs_params *exp_avg,
                  const gs_params *exp_avg_sq, const float lr_groups[6], float beta1, float beta2,
                  float eps, int64_t step, const int64_t *step_device, gs_stream stream);

/*
 * gs_adam with the gradient of Gaussian g taken as zero, and grads not read
 * there, where rows[g] == 0 (device, [params->ld] bytes, 4-byte aligned: the
 * marks of gs_project_bwd_rows).  The same update as gs_adam after a
 * backward that wrote those rows as zeros.
 */
gs_status gs_adam_rows(const gs_params *params, const gs_params *grads, const gs_params *exp_avg,
                       const gs_params *exp_avg_sq, const uint8_t *rows, const float lr_groups[6],
                       float beta1, float beta2, float eps, int64_t step, const int64_t *step_device,
                       gs_stream stream);

/*
 * gs_adam_rows in two parts that write disjoint elements.  part 2 updates,
 * with a zero gradient, only the Gaussians whose radius ([n_views][ld] int32
 * of gs_project, 16-byte aligned) is 0 in every view; it reads neither grads
 * nor rows (either may be NULL), so it may run right after gs_project, on
 * another stream, beside the rest of the step: it is a background kernel of
 * one CTA per SM, with streaming cache hints.  part 1 updates only the rows
 * marked in rows (gs_project_bwd_rows).  Part 1 after the backward and part 2
 * after the same projection give gs_adam_rows' result exactly.
 */
gs_status gs_adam_part(const gs_params *params, const gs_params *grads, const gs_params *exp_avg,
                       const gs_params *exp_avg_sq, const uint8_t *rows, const int32_t *radius,
                       int32_t n_views, int32_t part, const float lr_groups[6], float beta1, float beta2,
                       float eps, int64_t step, const int64_t *step_device, gs_stream stream);

/*
 * Chunk scores and global decisions (Supp. E.1, E.2; Sec. 3.3.2) from the
 * accumulators of one chunk: S_d = kappa / n_views; L = log(1 + gamma);
 * S_p = (L - min L) / (max L - min L) over Gaussians with |Omega| > 0 (0 for
 * the others, and 0 for all when max = min); densify |= S_d > tau_d;
 * prune_max = max(prune_max, S_p); prune = prune_max > tau_p.
 * ws: gs_prune_workspace_size bytes.
 */
gs_status gs_prune_stats(const gs_stats *stats, int64_t n, int32_t n_views, float tau_d,
                         float tau_p, const gs_chunk_scores *out, void *ws, size_t ws_bytes,
                         gs_stream stream);

/*
 * Densify / prune actions (Sec. 3.3.2 decisions applied per explicit
 * Gaussian; the paper spawns anchors, clone / split is the reading here).
 * Source Gaussian i emits, in source order: nothing when prune[i]; itself
 * when not densify[i]; otherwise two rows: when its largest log-scale
 * exceeds split_log_scale, two children mu + R S xi_j (xi_0 = noise planes
 * 0-2, xi_1 = planes 3-5 of noise [6][src->ld], standard normal samples the
 * caller draws; R S the covariance factor) with every log-scale reduced by
 * log(split_factor), else itself and an identical clone.  dst (same SH
 * degree) receives the rows; its capacity is dst->ld (dst->n is ignored).
 * src_m / src_v and dst_m / dst_v (nullable together) are the Adam moments:
 * the survivor keeps its own, clones and split children start at zero.
 * n_out (device int64) receives the rows needed; rows past the capacity are
 * dropped and status gets bit 1<<GS_ERR_CAPACITY.  densify, prune: [n]
 * bytes (0 / 1), e.g. gs_chunk_scores or gs_mlp_forward decisions.
 * ws: gs_actions_workspace_size bytes.
 */
gs_status gs_actions_workspace_size(int64_t n, size_t *bytes);
gs_status gs_densify_prune(const gs_params *src, const gs_params *src_m, const gs_params *src_v,
                           const uint8_t *densify, const uint8_t *prune, const float *noise,
                           float split_log_scale, float split_factor, const gs_params *dst,
                           const gs_params *dst_m, const gs_params *dst_v, int64_t *n_out,
                           int32_t *status, void *ws, size_t ws_bytes, gs_stream stream);

/*
 * Spatial order of the Gaussians (not a step of the paper's method: a layout
 * of its parameter planes, e.g. after the actions above).  Reorders, in place,
 * the rows 0..n-1 of params and of every extra plane set (Adam moments,
 * per-Gaussian statistics: same ld as params) into the Morton order of the
 * means, so that the Gaussians one view sees are near each other in memory.
 * The order, exactly:
 *   lo_a, hi_a  minimum and maximum of the means' axis a over the n rows
 *   scale       1024 / max_a (hi_a - lo_a) in FP32, 0 when that is 0 or not finite
 *   q_a         with t = (m_a - lo_a) * scale in FP32 (rounded per operation):
 *               1023 if t >= 1023, else (int) t if t > 0, else 0
 *   code        bit b of q_x at bit 3b, of q_y at 3b + 1, of q_z at 3b + 2
 *   order       rows by increasing code, equal codes in their previous order.
 * perm (nullable, [n] int32, device): new row i is previous row perm[i].
 * Padding rows [n, ld) are left as they are; every buffer keeps its address.
 * ws: gs_reorder_workspace_size(n, ld, largest plane count of params and the
 * extra sets) bytes, 256-byte aligned.  n_extra <= 16.
 */
typedef struct {
    float *data;    /* [planes][ld] */
    int64_t ld;
    int32_t planes;
} gs_plane_set;

gs_status gs_reorder_workspace_size(int64_t n, int64_t ld, int32_t max_planes, size_t *bytes);
gs_status gs_reorder(const gs_params *params, const gs_plane_set *extra, int32_t n_extra, int32_t *perm,
                     void *ws, size_t ws_bytes, gs_stream stream);

/*
 * Learned densify / prune predictor (not in the paper: an MLP trained on the
 * decisions of the plain criterion above, which stays the fallback and the
 * reference for its error).  16 inputs -> 64 -> 64 (ReLU) -> 2 logits (sigmoid):
 * output 0 = densify, 1 = prune.  Weights: one FP32 array of GS_MLP_WEIGHTS
 * floats, W1[64][16] at 0, b1[64] at 1024, W2[64][64] at 1088, b2[64] at
 * 5184, W3[2][64] at 5248, b3[2] at 5376.  Layers 1 and 2, the data
 * gradient through layer 2 and the hidden layers' weight and bias gradients
 * run on the tensor cores with BF16 operands (inputs, weights, hidden
 * activations, dL/dh divided by 2n) and FP32 accumulation; biases, the
 * output layer and its gradient stay FP32.
 */
#define GS_MLP_INPUTS 16
#define GS_MLP_HIDDEN 64
#define GS_MLP_WEIGHTS 5378
#define GS_MLP_RING 8

/*
 * Moves plane 3 of stats (max T*alpha since the last push) into plane slot
 * (0 <= slot < GS_MLP_RING) of ring [GS_MLP_RING][ring_ld] and zeroes it,
 * once per view (or per batch of views) rendered with statistics.
 */
gs_status gs_mlp_push_blend(const gs_stats *stats, int64_t n, float *ring, int64_t ring_ld, int32_t slot,
                            gs_stream stream);

/*
 * The 16 inputs per Gaussian, planes of params->ld in feat [16][ld]:
 * 0 sigmoid(opacity logit); 1-3 log-scales; 4 log(1 + views seen);
 * 5 log(1 + 1e4 * accumulated ||dL/d(u,v)||); 6-13 max T*alpha of the last
 * 8 views, most recent first (ring planes head, head-1, ... mod 8);
 * 14 log(1 + ||mu - cam_centre||); 15 log(1 + mean |Omega_v| over the views
 * seen).  stats: the lifecycle accumulators (ld = params->ld); ring
 * [GS_MLP_RING][params->ld]; cam_centre (host) e.g. the chunk's last camera.
 */
gs_status gs_mlp_features(const gs_params *params, const gs_stats *stats, const float *ring, int32_t head,
                          const float cam_centre[3], float *feat, gs_stream stream);

/*
 * Inference over n rows of feat [16][ld]: prob [2][ld] (nullable) gets the
 * sigmoid outputs; densify / prune [n] bytes (nullable) get logit > 0.
 * max_polls bounds each wait for a tile's tensor-core products (mbarrier
 * polls; negative selects the default 2^24, 0 gives up at the first wait).
 * A wait that gives up stops the CTA: it issues no further products, waits
 * (at the default bound) for the one in flight, frees its tensor memory,
 * writes nothing more and sets bit 1<<GS_ERR_TIMEOUT in status (nullable);
 * the call itself returns GS_OK, and rows of CTAs that gave up keep their
 * previous prob / densify / prune contents.
 */
gs_status gs_mlp_forward(const float *feat, int64_t n, int64_t ld, const float *weights, float *prob,
                         uint8_t *densify, uint8_t *prune, int32_t *status, int64_t max_polls, gs_stream stream);

/*
 * Mean binary cross-entropy over the n rows and both outputs against the
 * labels y_densify, y_prune ([n] bytes, 0 / 1) and its gradient: grad
 * [GS_MLP_WEIGHTS] and loss [1] (device) are overwritten.
 */
gs_status gs_mlp_train_grad(const float *feat, const uint8_t *y_densify, const uint8_t *y_prune, int64_t n,
                            int64_t ld, const float *weights, float *grad, float *loss, int32_t *status,
                            gs_stream stream);

/* Adam with bias correction (as gs_adam) over the GS_MLP_WEIGHTS weights. */
gs_status gs_mlp_adam(float *weights, const float *grad, float *exp_avg, float *exp_avg_sq, float lr,
                      float beta1, float beta2, float eps, int64_t step, gs_stream stream);

/*
 * Probabilistic initialisation of new anchors at a keyframe (Sec. 3.3.1)
 * and the voxel hash of the dynamic map expansion (Supp. D.5).
 *
 * P = min(lambda DoG + (1 - lambda) minmax(||grad D||), 1) with DoG =
 * min(scale |(G_s1 - G_s2) * Y|, 1), Y = (R + G + B) / 3 (scale 255 takes
 * [0, 1] images in 8-bit intensity units), G_s the sampled 2D
 * Gaussian of radius ceil(3 s) normalised to sum 1, ||grad D|| by central
 * differences, borders replicated and the min-max over the keyframe (a flat
 * map normalises to 0).  For a keyframe after the first, P_kf = max(P - P^,
 * 0) with P^ the same map of the rendered image and depth.  A pixel spawns
 * an anchor candidate when P_kf is the strict maximum of its 3x3 window
 * (equal values go to the lower raster index v W + u), P_kf > 0, the
 * caller's uniform draw there is below P_kf, and depth > near_z; its centre at that depth,
 * x_w = R^T (d ((u+0.5-cx)/fx, (v+0.5-cy)/fy, 1) - t), goes to the first
 * level l with ||x_c|| < max_dist[l] (none: skipped) and to the voxel
 * idx = floor(x_w / voxel[l]) (skipped unless -2^19 <= idx < 2^19).  A voxel
 * (l, idx) holds one anchor at p = idx * voxel[l]; voxels already in the
 * table stay as they are, and each new voxel becomes an anchor numbered in
 * raster order of the first pixel that reached it.  The decisions are taken
 * in FP32.
 */
#define GS_INIT_MAX_LEVELS 8
#define GS_INIT_MAX_RADIUS 16  /* ceil(3 sigma) of either blur */

/* host struct; defaults: 1.0, 1.6, 0.9, 255, 0.2, 5, voxel (0.1, 0.25, 1, 5,
 * 25) m, max_dist (10, 25, 100, 500, +inf) m */
typedef struct {
    float sigma1, sigma2;                /* DoG blur widths in pixels */
    float lambda;                        /* DoG / depth-gradient balance */
    float intensity_scale;               /* the DoG's intensity units per image unit */
    float near_z;                        /* pixels at depth <= near_z spawn nothing */
    int32_t levels;                      /* LoD levels m, 1..GS_INIT_MAX_LEVELS */
    float voxel[GS_INIT_MAX_LEVELS];     /* voxel size eps_l of level l */
    float max_dist[GS_INIT_MAX_LEVELS];  /* increasing upper camera distances */
} gs_init_cfg;

/* Open-addressing voxel table (linear probing).  A voxel key packs (l, ix,
 * iy, iz) as l << 60 | (ix + 2^19) << 40 | (iy + 2^19) << 20 | (iz + 2^19);
 * a free slot holds all ones.  capacity: a power of two >= 1024, each array
 * 16-byte aligned; keep the load below ~1/2 for short probe runs. */
typedef struct {
    uint64_t *keys;    /* [capacity] */
    int32_t *ids;      /* [capacity] anchor id of the slot's voxel, -1: none */
    int32_t *owner;    /* [capacity] work state of gs_init_insert (INT32_MAX free, -1 settled) */
    int64_t capacity;
} gs_voxel_table;

/* Anchor records, appended by gs_init_insert. */
typedef struct {
    float *pos;        /* [3][ld] planes: idx * voxel[l] */
    int32_t *level;    /* [ld] */
    int32_t *pixel;    /* [ld] spawning pixel v W + u of its keyframe */
    int64_t *count;    /* device int64: anchors in use; receives the new total */
    int64_t ld;        /* capacity */
} gs_anchor_set;

/* Marks every slot free. */
gs_status gs_voxel_table_reset(const gs_voxel_table *table, gs_stream stream);

/* Workspace of gs_init_probability and gs_init_insert for a W x H keyframe. */
gs_status gs_init_workspace_size(int32_t width, int32_t height, size_t *bytes);

/*
 * prob [H][W] = P of (img [3][H][W], depth [H][W]), or P_kf when img_r /
 * depth_r (the rendered pair; null together) are given.
 */
gs_status gs_init_probability(const float *img, const float *depth, const float *img_r, const float *depth_r,
                              int32_t width, int32_t height, const gs_init_cfg *cfg, float *prob, void *ws,
                              size_t ws_bytes, gs_stream stream);

/*
 * Candidates of prob (the output above) with the caller's uniform draws
 * [H][W] and depth [H][W] under camera cam; new voxels enter the table and
 * become anchors [count, count + new) of the set (count += new).  Anchors
 * past anchors->ld are not written, their slots get id -1 and status gets
 * bit 1<<GS_ERR_CAPACITY (a keyframe adds at most ceil(W/2) ceil(H/2)); a
 * full table skips the pixel with the same bit.  selected [H][W] bytes
 * (nullable): 1 where a candidate got a voxel.  Uses the same workspace.
 */
gs_status gs_init_insert(const float *prob, const float *uniform, const float *depth, const gs_camera *cam,
                         const gs_init_cfg *cfg, const gs_voxel_table *table, const gs_anchor_set *anchors,
                         uint8_t *selected, int32_t *status, void *ws, size_t ws_bytes, gs_stream stream);

/*
 * ids [n] = the anchor id of voxel (level, ix, iy, iz) = planes 0-3 of vox
 * [4][ld] (int32), -1 when the voxel is free or out of range.
 */
gs_status gs_voxel_lookup(const gs_voxel_table *table, const int32_t *vox, int64_t n, int64_t ld, int32_t *ids,
                          gs_stream stream);

/*
 * Scaffold-GS anchors (Sec. 3.2.1, Supp. D.1 decoding, Supp. D.3 LoD mask).
 * An anchor i at a fixed position p (e.g. a voxel of gs_init_insert, with
 * its level l) holds a feature f (32), a log-scale log l (3) and K = 10
 * offsets O_k (3 each).  For a camera centre c, d = ||p - c||, its decoder
 * (one hidden layer of 64 with ReLU; weights W1[64][36], b1[64],
 * W2[140][64], b2[140] in one array) maps (f, (p - c)/d, log(1 + d)) to 14
 * outputs per Gaussian k: colour (sigmoid), opacity a (tanh), rotation
 * (1, 0, 0, 0) + output, scale factor ds (sigmoid), offset dO.  Gaussian k
 * has mean p + (O_k + dO_k) * l, scale l * ds, and opacity a where d lies in
 * the level's band [max_dist[l-1], max_dist[l]) (0 below the first) and
 * a > 0; otherwise it is dropped.
 */
#define GS_ANCHOR_K 10
#define GS_ANCHOR_FEAT 32
#define GS_ANCHOR_PLANES 65      /* 0-31 feature, 32-34 log-scale, 35 + 3k + c offset k */
#define GS_ANCHOR_WEIGHTS 11468

typedef struct {
    float *data;           /* [GS_ANCHOR_PLANES][ld] */
    const float *pos;      /* [3][ld] positions (not optimised) */
    const int32_t *level;  /* [ld] LoD level of each anchor */
    int64_t n, ld;         /* anchors, plane stride (a multiple of 4) */
} gs_anchor_params;

/*
 * Decodes every anchor for a camera centre (host float[3]) into out: an SH
 * degree 0 gs_params with out->n == GS_ANCHOR_K * a->ld; Gaussian k of
 * anchor i is column k * a->ld + i.  Dropped Gaussians (and the padding
 * anchors i >= n) get opacity logit -30, which the projection culls, so out
 * renders directly through gs_project ... gs_render_bwd.  max_dist: host
 * float[levels] (the bands of gs_init_cfg), 1 <= levels <= 8.
 * The decoder's two layers run on the tensor cores with bfloat16 operands
 * (the input x, W1, the hidden activation, W2) and FP32 sums; the biases and
 * everything after the hidden layer are FP32.  max_polls and status
 * (nullable device int32) as in gs_mlp_forward: a CTA whose wait for its
 * tensor-core products gives up sets bit 1<<GS_ERR_TIMEOUT and writes no
 * further tiles.
 */
gs_status gs_anchor_decode(const gs_anchor_params *a, const float *weights, const float cam_centre[3],
                           const float *max_dist, int32_t levels, const gs_params *out, int32_t *status,
                           int64_t max_polls, gs_stream stream);

/*
 * Gradient of a loss with respect to the anchors (grad_anchor
 * [GS_ANCHOR_PLANES][a->ld], overwritten) and the decoder's weights
 * (grad_weights [GS_ANCHOR_WEIGHTS], overwritten) from its gradient with
 * respect to the decoded Gaussians (grad_out, laid out as out above, e.g.
 * the gradient buffer of gs_render_bwd / gs_project_bwd).  The products
 * with W2, W1 and the weight gradients' sums over anchors run on the tensor
 * cores with dL/dz and dL/d(pre-activation) rounded to bfloat16 (FP32
 * sums); the rest is FP32.  max_polls and status as in gs_anchor_decode; a
 * timed-out CTA adds nothing to grad_weights.
 */
gs_status gs_anchor_decode_bwd(const gs_anchor_params *a, const float *weights, const float cam_centre[3],
                               const float *max_dist, int32_t levels, const gs_params *grad_out,
                               float *grad_anchor, float *grad_weights, int32_t *status, int64_t max_polls,
                               gs_stream stream);

/* Adam with bias correction over n contiguous floats (p, g, m, v device).
 * step_device (nullable device int64): as in gs_adam, the step count read
 * when the kernel runs (`step` ignored), for captured CUDA graphs. */
gs_status gs_adam_flat(float *p, const float *g, float *m, float *v, int64_t n, float lr, float beta1, float beta2,
                       float eps, int64_t step, const int64_t *step_device, gs_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* GS_H */
