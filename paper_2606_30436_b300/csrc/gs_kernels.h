// gs_kernels.h -- internal launchers of the sm_103a kernels (host side).
#pragma once

#include <cuda_runtime.h>

#include "gs_internal.cuh"

namespace gs {

// Per-record accumulator planes written by the compositing backward and read by
// the projection backward, record-major: value p of record r at
// acc[r * kAccStride + p], so the sums of one record sit in one 64-byte line
// and a lane adds four of them with one vector atomic.
enum AccPlane {
    kAccU = 0, kAccV, kAccA, kAccB, kAccC, kAccO, kAccR, kAccG, kAccBl, kAccZ,
    kAccOmega, kAccKappa, kAccMaxW, kAccPlanes
};
constexpr int kAccStride = 16;
static_assert(kAccU == 0 && kAccC == 4 && kAccBl == 8 && kAccOmega == 10 && kAccKappa == 11 && kAccMaxW == 12,
              "the vector reads and atomics group the sums four by four");

void launch_project(const float *P, long long n, long long ld, int D, const ViewTable &vt, const RasterCfg &cfg,
                    float2 *xy, float4 *co, float4 *rgbd, int *radius, int *touched, int *status, float4 *cj,
                    cudaStream_t s);

void launch_project_bwd(const float *P, long long n, long long ld, int D, const ViewTable &vt, const RasterCfg &cfg,
                        const int *radius, const float *acc, long long nrec, float *G, int accumulate,
                        const float *loss_per_view, float *stats, long long stats_ld, const float4 *cj,
                        uint8_t *rows, cudaStream_t s);
void launch_project_bwd_adam(float *P, long long n, long long ld, int D, const ViewTable &vt, const RasterCfg &cfg,
                             const int *radius, const float *acc, long long nrec, const float *G_in, float *m,
                             float *v, const float lr[6], float beta1, float beta2, float eps, long long step,
                             const long long *step_dev, float iso_weight, const float *loss_per_view, float *stats,
                             long long stats_ld, cudaStream_t s);

// Binning: workspace layout and launch of the whole sort pipeline.
size_t sort_workspace_bytes(long long nrec, long long max_pairs);
cudaError_t launch_sort(const int *radius, const int *touched, const float2 *xy, const float4 *co, const float4 *rgbd,
                        long long nrec, long long ld, const ViewTable &vt, float alpha_min, int *gauss_ids,
                        int2 *tile_ranges, uint8_t *block_mask, int *tile_order, int *counts, long long max_pairs,
                        void *ws, int *status, cudaStream_t s);

// Stable LSD radix sort of count (device) 32-bit keys with 32-bit values on bits [0, bits):
// k0/v0 hold the input, k1/v1 the same capacity; the sorted values land in final_v.
size_t key_sort_scratch_bytes();
void launch_key_sort(uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, const int *count, long long cap,
                     int bits, void *scratch, uint32_t *final_v, cudaStream_t s);

// Spatial (Morton) order of the Gaussians (reorder.cu).
size_t reorder_workspace_bytes(long long n, long long ld, int max_planes);
cudaError_t launch_reorder(float *P, long long n, long long ld, int planes, float *const *extra,
                           const int *extra_planes, int n_extra, int *perm, void *ws, cudaStream_t s);

void launch_render_fwd(const ViewTable &vt, const RasterCfg &cfg, const int2 *ranges, const int *ids,
                       const uint8_t *masks, const int *order, const float2 *xy, const float4 *co,
                       const float4 *rgbd, float *img, float *T_final, int *last, float *depth, const SegWs &seg,
                       cudaStream_t s);

size_t list_scan_bytes(long long npx);
void launch_render_fwd_lists(const ViewTable &vt, const RasterCfg &cfg, const int2 *ranges, const int *ids,
                             const uint8_t *masks, const int *order, const float2 *xy, const float4 *co,
                             const float4 *rgbd, float *img, float *T_final, int *last, float *depth, long long npx,
                             long long *count_off, int *lid, float *lal, long long cap, void *scan_ws, int *status,
                             cudaStream_t s);
void launch_render_bwd_lists(const ViewTable &vt, const RasterCfg &cfg, long long npx, const long long *off,
                             const int *lid, const float *lal, long long cap, const float2 *xy, const float4 *co,
                             const float4 *rgbd, const float *img, const float *T_final, const float *dL_dimg,
                             const float *target, float tau_err, bool stats, float *acc, cudaStream_t s);
void launch_render_bwd(const ViewTable &vt, const RasterCfg &cfg, const int2 *ranges, const int *ids,
                       const uint8_t *masks, const int *order, const float2 *xy, const float4 *co, const float4 *rgbd,
                       const float *img, const float *T_final,
                       const int *last, const float *dL_dimg, const float *dL_ddepth, const float *target,
                       float tau_err, bool stats, float *acc, long long nrec, const float *depth, const SegWs &seg,
                       cudaStream_t s);

size_t loss_workspace_bytes(int h, int w);
bool loss_static_fits(int h, int w);
long long loss_static_max_pixels();
cudaError_t loss_static_scratch(void **out);
cudaError_t launch_loss(const float *img, const float *target, int h, int w, float lambda, float *loss_out,
                        float *dL_dimg, void *ws, cudaStream_t s);

// rows (nullable, [ld] bytes): where rows[i] == 0 the gradient of Gaussian i is zero and g is not read.
// part (with rows): 0 every row, 1 the marked rows only; part 2: only the Gaussians whose radius
// ([n_views][ld]) is 0 in every view, rows and g unused.
void launch_adam(float *p, const float *g, float *m, float *v, long long ld, int planes, const float lr[6],
                 float beta1, float beta2, float eps, long long step, const long long *step_dev,
                 const uint8_t *rows, cudaStream_t s, int part = 0, const int *radius = nullptr,
                 int n_views = 0);

size_t reg_workspace_bytes();
cudaError_t launch_geo(const float *depth, const float *prior, long long npx, float weight, float *loss, float *dL,
                       void *ws, cudaStream_t s);
cudaError_t launch_iso(const float *P, long long n, long long ld, float weight, float *loss, float *G, void *ws,
                       cudaStream_t s);

size_t prune_workspace_bytes(long long n);
void launch_prune(const float *acc, long long ld, long long n, int n_views, float tau_d, float tau_p, float *S_d,
                  float *S_p, float *prune_max, unsigned char *densify, unsigned char *prune, void *ws,
                  cudaStream_t s);

size_t actions_workspace_bytes(long long n);
cudaError_t launch_actions(const float *src, const float *src_m, const float *src_v, long long n, long long ld,
                           int planes, const uint8_t *dens, const uint8_t *prune, const float *noise,
                           float split_log_scale, float log_split_factor, float *dst, float *dst_m, float *dst_v,
                           long long dld, long long *n_out, int *status, void *ws, cudaStream_t s);

int mlp_num_weights();
cudaError_t launch_mlp_push_blend(float *stats, long long sld, long long n, float *ring, long long ld, int slot,
                                  cudaStream_t s);
cudaError_t launch_mlp_features(const float *P, long long n, long long ld, const float *stats, long long sld,
                                const float *ring, int head, const float cam[3], float *feat, cudaStream_t s);
cudaError_t launch_mlp_forward(const float *feat, long long n, long long ld, const float *w, float *prob,
                               uint8_t *densify, uint8_t *prune, int *status, long long max_polls, cudaStream_t s);
cudaError_t launch_mlp_train(const float *feat, const uint8_t *y_densify, const uint8_t *y_prune, long long n,
                             long long ld, const float *w, float *grad, float *loss, int *status, cudaStream_t s);
cudaError_t launch_mlp_adam(float *w, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                            long long step, cudaStream_t s);

// Probabilistic initialisation (init.cu).  Blur weights w[k] of offset +-k
// (normalised, radius r <= GS_INIT_MAX_RADIUS; R = the larger radius).
struct InitBlur {
    float w1[GS_INIT_MAX_RADIUS + 1], w2[GS_INIT_MAX_RADIUS + 1];
    float scale;  // intensity units of the DoG
    int r1, r2, R;
};
struct InitCam {
    float R[9], t[3], fx, fy, cx, cy;
};
struct InitLod {
    float voxel[GS_INIT_MAX_LEVELS], max_dist[GS_INIT_MAX_LEVELS];
    float near_z;
    int levels;
};
size_t init_workspace_bytes(int W, int H);
cudaError_t launch_init_probability(const float *img, const float *depth, const float *img_r, const float *depth_r,
                                    int W, int H, const InitBlur &bw, float lambda, float *prob, void *ws,
                                    cudaStream_t s);
cudaError_t launch_init_insert(const float *prob, const float *uniform, const float *depth, int W, int H,
                               const InitCam &cam, const InitLod &lod, unsigned long long *keys, int *ids, int *owner,
                               long long cap, float *pos, int *level, int *pixel, long long *count, long long ld,
                               uint8_t *selected, int *status, void *ws, cudaStream_t s);
cudaError_t launch_voxel_lookup(const unsigned long long *keys, const int *ids, long long cap, const int *vox,
                                long long n, long long ld, int *out, cudaStream_t s);
cudaError_t launch_voxel_reset(unsigned long long *keys, int *ids, int *owner, long long cap, cudaStream_t s);

// Scaffold-GS anchors (anchors.cu): camera centre and the LoD band [lo, hi) of each level.
struct AnchorView {
    float c[3];
    float lo[GS_INIT_MAX_LEVELS], hi[GS_INIT_MAX_LEVELS];
    int levels;
};
cudaError_t launch_anchor_decode(const float *A, const float *pos, const int *level, long long n, long long ld,
                                 const float *w, const AnchorView &v, float *G, long long gld, int *status,
                                 long long max_polls, cudaStream_t s);
cudaError_t launch_anchor_decode_bwd(const float *A, const float *pos, const int *level, long long n, long long ld,
                                     const float *w, const AnchorView &v, const float *GG, long long gld, float *gA,
                                     float *gw, int *status, long long max_polls, cudaStream_t s);
cudaError_t launch_adam_flat(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                             float eps, long long step, const long long *step_dev, cudaStream_t s);

}  // namespace gs
