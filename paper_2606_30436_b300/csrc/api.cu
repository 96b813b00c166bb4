// api.cu -- the extern "C" entry points declared in include/gs.h: argument
// validation, the per-call view table, and the kernel launches on the caller's
// stream.  No entry point allocates device memory or synchronises the host.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "gs_internal.cuh"
#include "gs_kernels.h"

#define GS_API extern "C" __attribute__((visibility("default")))

using namespace gs;

namespace {

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

gs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ERR_CUDA; }

gs_status check_cfg(const gs_raster_cfg *cfg) {
    if (!cfg) return GS_ERR_INVALID;
    const int tw = cfg->tile_w, th = cfg->tile_h;
    const bool shape_ok = (tw == 16 && th == 16) || (tw == 8 && th == 32) || (tw == 32 && th == 8);
    if (!shape_ok) return GS_ERR_INVALID;
    if (!(cfg->near_z > 0.0f) || !(cfg->alpha_max > 0.0f && cfg->alpha_max < 1.0f) || !(cfg->alpha_min >= 0.0f) ||
        !(cfg->t_min >= 0.0f) || !(cfg->dilation >= 0.0f) || !(cfg->tan_clamp > 0.0f))
        return GS_ERR_INVALID;
    if (cfg->batch != 0 && cfg->batch != 128 && cfg->batch != 256 && cfg->batch != 512) return GS_ERR_INVALID;
    const int sg = cfg->segment;
    if (sg != 0 && (sg < 32 || sg > 65536 || (sg & (sg - 1)))) return GS_ERR_INVALID;
    return GS_OK;
}

// The split workspace of a frame (no split: all null, capacities 0); its
// capacities follow from the bytes the caller gave.
gs_status seg_of(const gs_raster_cfg *cfg, const gs_frame *frame, SegWs &seg) {
    seg = SegWs{nullptr, nullptr, 0, nullptr, nullptr, 0, nullptr, nullptr, 0};
    if (cfg->segment == 0) return GS_OK;
    if (!frame->seg_ws || ((uintptr_t)frame->seg_ws & 255u)) return GS_ERR_INVALID;
    const long long F = seg_items_in(frame->seg_ws_bytes);
    if (F < 16 || F > 0x7fffffffll) return GS_ERR_INVALID;
    const long long hcap = seg_heavy_for(F);
    unsigned char *b = (unsigned char *)frame->seg_ws;
    size_t off = 256;
    seg.count = (int *)b;
    seg.heavy = (int4 *)(b + off);
    off += align_up(sizeof(int4) * (size_t)hcap, 256);
    seg.fres = (float *)(b + off);
    off += align_up(sizeof(float) * kFresFloats * (size_t)F, 256);
    seg.tasks = (int4 *)(b + off);
    off += align_up(sizeof(int4) * (size_t)F, 256);
    seg.items = (int2 *)(b + off);
    off += align_up(sizeof(int2) * (size_t)F, 256);
    seg.ckpt = (float *)(b + off);
    seg.hcap = (int)hcap;
    seg.fcap = (int)F;
    seg.cap = (int)F;
    return GS_OK;
}

gs_status build_views(const gs_camera *cams, int n_views, const gs_raster_cfg *cfg, ViewTable &vt, RasterCfg &rc) {
    if (!cams || n_views < 1 || n_views > GS_MAX_VIEWS) return GS_ERR_INVALID;
    gs_status st = check_cfg(cfg);
    if (st != GS_OK) return st;
    std::memset(&vt, 0, sizeof(vt));
    vt.n_views = n_views;
    vt.tile_w = cfg->tile_w;
    vt.tile_h = cfg->tile_h;
    long long tiles = 0, pix = 0;
    for (int v = 0; v < n_views; ++v) {
        const gs_camera &c = cams[v];
        if (c.width <= 0 || c.height <= 0 || c.width > 65536 || c.height > 65536 || !(c.fx > 0.0f) || !(c.fy > 0.0f))
            return GS_ERR_INVALID;
        ViewDesc &d = vt.v[v];
        for (int k = 0; k < 9; ++k) d.R[k] = c.R[k];
        for (int k = 0; k < 3; ++k) d.t[k] = c.t[k];
        d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
        for (int k = 0; k < 3; ++k)  // camera centre -R^T t, in double then rounded
            d.campos[k] = (float)(-((double)c.R[k] * c.t[0] + (double)c.R[3 + k] * c.t[1] + (double)c.R[6 + k] * c.t[2]));
        d.limx = (float)((double)cfg->tan_clamp * c.width / (2.0 * c.fx));
        d.limy = (float)((double)cfg->tan_clamp * c.height / (2.0 * c.fy));
        d.W = c.width; d.H = c.height;
        d.GW = (c.width + cfg->tile_w - 1) / cfg->tile_w;
        d.GH = (c.height + cfg->tile_h - 1) / cfg->tile_h;
        d.tile_offset = (int)tiles;
        d.pix_offset = pix;
        tiles += (long long)d.GW * d.GH;
        pix += (long long)c.width * c.height;
        if (tiles > 0xffffffll) return GS_ERR_INVALID;  // tile ids share a 32-bit sort key with an 8-bit mask
    }
    vt.total_tiles = (int)tiles;
    rc.near_z = cfg->near_z; rc.dilation = cfg->dilation; rc.alpha_min = cfg->alpha_min;
    rc.alpha_max = cfg->alpha_max; rc.t_min = cfg->t_min; rc.tan_clamp = cfg->tan_clamp;
    rc.logit_min = (float)std::log((double)cfg->alpha_min / (1.0 - (double)cfg->alpha_min));
    for (int k = 0; k < 3; ++k) rc.bg[k] = cfg->bg[k];
    rc.tile_w = cfg->tile_w; rc.tile_h = cfg->tile_h;
    rc.batch = cfg->batch == 0 ? 512 : cfg->batch;
    rc.seg_shift = -1;
    for (int k = 5; k <= 16; ++k)
        if (cfg->segment == (1 << k)) rc.seg_shift = k;
    return GS_OK;
}

gs_status check_params(const gs_params *p) {
    if (!p || !p->data || p->n < 0 || p->ld < p->n || (p->ld & 3) || p->sh_degree < 0 || p->sh_degree > 3 ||
        !aligned16(p->data))
        return GS_ERR_INVALID;
    return GS_OK;
}

gs_status check_proj(const gs_projected *pr, long long ld) {
    if (!pr || !pr->xy || !pr->conic_opacity || !pr->rgb_depth || !pr->radius || !pr->tiles_touched) return GS_ERR_INVALID;
    if (pr->ld != ld) return GS_ERR_INVALID;
    if (!aligned16(pr->xy) || !aligned16(pr->conic_opacity) || !aligned16(pr->rgb_depth)) return GS_ERR_INVALID;
    if (pr->color_jac && !aligned16(pr->color_jac)) return GS_ERR_INVALID;
    return GS_OK;
}

gs_status check_binning(const gs_binning *b) {
    if (!b || !b->gauss_ids || !b->tile_ranges || !b->counts || !b->block_mask || !b->tile_order || b->max_pairs < 0 ||
        b->max_pairs > 0x7fffffffll)
        return GS_ERR_INVALID;
    if (((uintptr_t)b->tile_ranges & 7u) != 0 || !aligned16(b->block_mask)) return GS_ERR_INVALID;
    return GS_OK;
}

}  // namespace

GS_API const char *gs_status_string(gs_status s) {
    switch (s) {
        case GS_OK: return "ok";
        case GS_ERR_INVALID: return "invalid argument";
        case GS_ERR_CUDA: return "CUDA error";
        case GS_ERR_CAPACITY: return "pair capacity exceeded";
        case GS_ERR_TIMEOUT: return "bounded wait timed out";
        case GS_ERR_NUMERIC: return "non-finite value";
    }
    return "unknown status";
}

GS_API int32_t gs_version(void) { return 10000 + 1030; }

GS_API gs_status gs_view_layout(const gs_camera *cams, int32_t n_views, const gs_raster_cfg *cfg,
                                int64_t *total_tiles, int64_t *total_pixels, int64_t *tile_offset,
                                int64_t *pixel_offset) {
    ViewTable vt;
    RasterCfg rc;
    gs_status st = build_views(cams, n_views, cfg, vt, rc);
    if (st != GS_OK) return st;
    long long pix = 0;
    for (int v = 0; v < n_views; ++v) {
        if (tile_offset) tile_offset[v] = vt.v[v].tile_offset;
        if (pixel_offset) pixel_offset[v] = vt.v[v].pix_offset;
        pix += (long long)vt.v[v].W * vt.v[v].H;
    }
    if (total_tiles) *total_tiles = vt.total_tiles;
    if (total_pixels) *total_pixels = pix;
    return GS_OK;
}

GS_API gs_status gs_sort_workspace_size(int64_t n_records, int64_t max_pairs, size_t *bytes) {
    if (!bytes || n_records < 0 || max_pairs < 0 || n_records > 0x7fffffffll || max_pairs > 0x7fffffffll)
        return GS_ERR_INVALID;
    *bytes = sort_workspace_bytes(n_records, max_pairs);
    return GS_OK;
}

GS_API gs_status gs_block_mask_size(int64_t max_pairs, size_t *bytes) {
    if (!bytes || max_pairs < 0 || max_pairs > 0x7fffffffll) return GS_ERR_INVALID;
    *bytes = (size_t)block_mask_bytes(max_pairs);
    return GS_OK;
}

GS_API gs_status gs_loss_workspace_size(int32_t h, int32_t w, size_t *bytes) {
    if (!bytes || h <= 0 || w <= 0) return GS_ERR_INVALID;
    *bytes = loss_workspace_bytes(h, w);
    return GS_OK;
}

GS_API gs_status gs_segment_workspace_size(int64_t max_pairs, int32_t segment, size_t *bytes) {
    if (!bytes || max_pairs < 0 || segment < 32 || segment > 65536 || (segment & (segment - 1))) return GS_ERR_INVALID;
    *bytes = seg_bytes_for(seg_items_worst(max_pairs, segment));
    return GS_OK;
}

GS_API gs_status gs_segment_workspace_size_items(int64_t items, size_t *bytes) {
    if (!bytes || items < 0 || items > 0x7fffffffll) return GS_ERR_INVALID;
    *bytes = seg_bytes_for(items < 16 ? 16 : items);
    return GS_OK;
}

GS_API gs_status gs_bwd_workspace_size(int64_t n_records, size_t *bytes) {
    if (!bytes || n_records < 0) return GS_ERR_INVALID;
    *bytes = align_up(sizeof(float) * (size_t)kAccStride * (size_t)n_records, 256);
    return GS_OK;
}

GS_API gs_status gs_prune_workspace_size(int64_t n, size_t *bytes) {
    if (!bytes || n < 0) return GS_ERR_INVALID;
    *bytes = prune_workspace_bytes(n);
    return GS_OK;
}

GS_API gs_status gs_project(const gs_params *params, const gs_camera *cams, int32_t n_views, const gs_raster_cfg *cfg,
                            const gs_projected *out, int32_t *status, gs_stream stream) {
    ViewTable vt;
    RasterCfg rc;
    gs_status st = build_views(cams, n_views, cfg, vt, rc);
    if (st == GS_OK) st = check_params(params);
    if (st == GS_OK) st = check_proj(out, params->ld);
    if (st != GS_OK) return st;
    launch_project(params->data, params->n, params->ld, params->sh_degree, vt, rc, (float2 *)out->xy,
                   (float4 *)out->conic_opacity, (float4 *)out->rgb_depth, out->radius, out->tiles_touched, status,
                   (float4 *)out->color_jac, (cudaStream_t)stream);
    return cuda_status(cudaGetLastError());
}

GS_API gs_status gs_sort(const gs_projected *proj, const gs_camera *cams, int32_t n_views, const gs_raster_cfg *cfg,
                         const gs_binning *binning, void *ws, size_t ws_bytes, int32_t *status, gs_stream stream) {
    ViewTable vt;
    RasterCfg rc;
    gs_status st = build_views(cams, n_views, cfg, vt, rc);
    if (st != GS_OK) return st;
    if (!proj) return GS_ERR_INVALID;
    if ((st = check_proj(proj, proj->ld)) != GS_OK) return st;
    if ((st = check_binning(binning)) != GS_OK) return st;
    const long long nrec = (long long)n_views * proj->ld;
    if (nrec > 0x7fffffffll) return GS_ERR_INVALID;
    if (!ws || ((uintptr_t)ws & 255u) || ws_bytes < sort_workspace_bytes(nrec, binning->max_pairs)) return GS_ERR_INVALID;
    return cuda_status(launch_sort(proj->radius, proj->tiles_touched, (const float2 *)proj->xy,
                                   (const float4 *)proj->conic_opacity, (const float4 *)proj->rgb_depth, nrec,
                                   proj->ld, vt, rc.alpha_min, binning->gauss_ids, (int2 *)binning->tile_ranges,
                                   binning->block_mask, binning->tile_order, binning->counts, binning->max_pairs, ws,
                                   status,
                                   (cudaStream_t)stream));
}

GS_API gs_status gs_render_fwd(const gs_projected *proj, const gs_binning *binning, const gs_camera *cams,
                               int32_t n_views, const gs_raster_cfg *cfg, const gs_frame *frame, gs_stream stream) {
    ViewTable vt;
    RasterCfg rc;
    gs_status st = build_views(cams, n_views, cfg, vt, rc);
    if (st != GS_OK) return st;
    if (!proj || (st = check_proj(proj, proj->ld)) != GS_OK) return GS_ERR_INVALID;
    if ((st = check_binning(binning)) != GS_OK) return st;
    if (!frame || !frame->img || !frame->T_final || !frame->last) return GS_ERR_INVALID;
    SegWs seg;
    if ((st = seg_of(cfg, frame, seg)) != GS_OK) return st;
    launch_render_fwd(vt, rc, (const int2 *)binning->tile_ranges, binning->gauss_ids, binning->block_mask,
                      binning->tile_order, (const float2 *)proj->xy,
                      (const float4 *)proj->conic_opacity, (const float4 *)proj->rgb_depth, frame->img,
                      frame->T_final, frame->last, frame->depth, seg, (cudaStream_t)stream);
    return cuda_status(cudaGetLastError());
}

GS_API gs_status gs_loss(const float *img, const float *target, const gs_camera *cams, int32_t n_views,
                         float lambda_dssim, float *loss_per_view, float *dL_dimg, void *ws, size_t ws_bytes,
                         gs_stream stream) {
    if (!img || !target || !cams || !loss_per_view || n_views < 1 || n_views > GS_MAX_VIEWS || !ws) return GS_ERR_INVALID;
    if (!(lambda_dssim >= 0.0f && lambda_dssim <= 1.0f) || ((uintptr_t)ws & 255u)) return GS_ERR_INVALID;
    long long off = 0;
    for (int v = 0; v < n_views; ++v) {
        const int h = cams[v].height, w = cams[v].width;
        if (h <= 0 || w <= 0 || ws_bytes < loss_workspace_bytes(h, w)) return GS_ERR_INVALID;
    }
    for (int v = 0; v < n_views; ++v) {
        const int h = cams[v].height, w = cams[v].width;
        cudaError_t e = launch_loss(img + off, target + off, h, w, lambda_dssim, loss_per_view + v,
                                    dL_dimg ? dL_dimg + off : nullptr, ws, (cudaStream_t)stream);
        if (e != cudaSuccess) return GS_ERR_CUDA;
        off += 3ll * h * w;
    }
    return GS_OK;
}

GS_API gs_status gs_loss_static(const float *img, const float *target, const gs_camera *cams, int32_t n_views,
                                float lambda_dssim, float *loss_per_view, float *dL_dimg, gs_stream stream) {
    if (!img || !target || !cams || !loss_per_view || n_views < 1 || n_views > GS_MAX_VIEWS) return GS_ERR_INVALID;
    if (!(lambda_dssim >= 0.0f && lambda_dssim <= 1.0f)) return GS_ERR_INVALID;
    for (int v = 0; v < n_views; ++v)
        if (!loss_static_fits(cams[v].height, cams[v].width)) return GS_ERR_INVALID;  // view beyond the array
    void *scratch = nullptr;
    if (loss_static_scratch(&scratch) != cudaSuccess) return GS_ERR_CUDA;
    long long off = 0;
    for (int v = 0; v < n_views; ++v) {
        const int h = cams[v].height, w = cams[v].width;
        cudaError_t e = launch_loss(img + off, target + off, h, w, lambda_dssim, loss_per_view + v,
                                    dL_dimg ? dL_dimg + off : nullptr, scratch, (cudaStream_t)stream);
        if (e != cudaSuccess) return GS_ERR_CUDA;
        off += 3ll * h * w;
    }
    return GS_OK;
}

GS_API gs_status gs_reg_workspace_size(size_t *bytes) {
    if (!bytes) return GS_ERR_INVALID;
    *bytes = reg_workspace_bytes();
    return GS_OK;
}

GS_API gs_status gs_geo_loss(const float *depth, const float *prior, const gs_camera *cams, int32_t n_views,
                             float weight, float *loss_per_view, float *dL_ddepth, void *ws, size_t ws_bytes,
                             gs_stream stream) {
    if (!depth || !prior || !cams || !loss_per_view || n_views < 1 || n_views > GS_MAX_VIEWS) return GS_ERR_INVALID;
    if (!ws || ((uintptr_t)ws & 255u) || ws_bytes < reg_workspace_bytes() || !(weight >= 0.0f)) return GS_ERR_INVALID;
    long long off = 0;
    for (int v = 0; v < n_views; ++v) {
        const long long npx = (long long)cams[v].width * cams[v].height;
        if (npx <= 0) return GS_ERR_INVALID;
        cudaError_t e = launch_geo(depth + off, prior + off, npx, weight, loss_per_view + v,
                                   dL_ddepth ? dL_ddepth + off : nullptr, ws, (cudaStream_t)stream);
        if (e != cudaSuccess) return GS_ERR_CUDA;
        off += npx;
    }
    return GS_OK;
}

GS_API gs_status gs_iso_loss(const gs_params *params, float weight, float *loss, const gs_params *grads, void *ws,
                             size_t ws_bytes, gs_stream stream) {
    gs_status st = check_params(params);
    if (st == GS_OK && grads) st = check_params(grads);
    if (st != GS_OK) return st;
    if (grads && (grads->ld != params->ld || grads->n != params->n)) return GS_ERR_INVALID;
    if (!loss || !ws || ((uintptr_t)ws & 255u) || ws_bytes < reg_workspace_bytes() || !(weight >= 0.0f))
        return GS_ERR_INVALID;
    return cuda_status(launch_iso(params->data, params->n, params->ld, weight, loss, grads ? grads->data : nullptr, ws,
                                  (cudaStream_t)stream));
}

GS_API gs_status gs_render_bwd(const gs_params *params, const gs_camera *cams, int32_t n_views,
                               const gs_raster_cfg *cfg, const gs_projected *proj, const gs_binning *binning,
                               const gs_frame *frame, const float *dL_dimg, const float *dL_ddepth,
                               const float *target, const float *loss_per_view, float tau_err, const gs_params *grads,
                               int32_t accumulate, const gs_stats *stats, void *ws, size_t ws_bytes,
                               gs_stream stream) {
    ViewTable vt;
    RasterCfg rc;
    gs_status st = build_views(cams, n_views, cfg, vt, rc);
    if (st == GS_OK) st = check_params(params);
    if (st == GS_OK && grads) st = check_params(grads);
    if (st != GS_OK) return st;
    if (grads && (grads->ld != params->ld || grads->n != params->n || grads->sh_degree != params->sh_degree))
        return GS_ERR_INVALID;
    if (!proj || check_proj(proj, params->ld) != GS_OK || check_binning(binning) != GS_OK) return GS_ERR_INVALID;
    if (!frame || !frame->img || !frame->T_final || !frame->last || !dL_dimg) return GS_ERR_INVALID;
    SegWs seg;
    if ((st = seg_of(cfg, frame, seg)) != GS_OK) return st;
    const bool want_stats = stats != nullptr;
    if (want_stats && (!stats->acc || stats->ld < params->n || !target)) return GS_ERR_INVALID;
    const long long nrec = (long long)n_views * params->ld;
    size_t need = 0;
    gs_bwd_workspace_size(nrec, &need);
    if (!ws || ((uintptr_t)ws & 255u) || ws_bytes < need) return GS_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    float *acc = (float *)ws;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(float) * (size_t)kAccStride * nrec, s);
    if (e != cudaSuccess) return GS_ERR_CUDA;
    launch_render_bwd(vt, rc, (const int2 *)binning->tile_ranges, binning->gauss_ids, binning->block_mask,
                      binning->tile_order, (const float2 *)proj->xy,
                      (const float4 *)proj->conic_opacity, (const float4 *)proj->rgb_depth, frame->img,
                      frame->T_final, frame->last, dL_dimg, dL_ddepth, target, tau_err, want_stats, acc, nrec,
                      frame->depth, seg, s);
    if (grads)
        launch_project_bwd(params->data, params->n, params->ld, params->sh_degree, vt, rc, proj->radius, acc, nrec,
                           grads->data, accumulate, loss_per_view, want_stats ? stats->acc : nullptr,
                           want_stats ? stats->ld : 0, (const float4 *)proj->color_jac, nullptr, s);
    return cuda_status(cudaGetLastError());
}

GS_API gs_status gs_list_workspace_size(int64_t total_pixels, size_t *bytes) {
    if (!bytes || total_pixels < 0) return GS_ERR_INVALID;
    *bytes = list_scan_bytes(total_pixels);
    return GS_OK;
}

GS_API gs_status gs_render_fwd_lists(const gs_projected *proj, const gs_binning *binning, const gs_camera *cams,
                                     int32_t n_views, const gs_raster_cfg *cfg, const gs_frame *frame,
                                     int64_t *list_offsets, int32_t *list_ids, float *list_alpha,
                                     int64_t list_capacity, void *ws, size_t ws_bytes, int32_t *status,
                                     gs_stream stream) {
    ViewTable vt;
    RasterCfg rc;
    gs_status st = build_views(cams, n_views, cfg, vt, rc);
    if (st != GS_OK) return st;
    if (!proj || check_proj(proj, proj->ld) != GS_OK || check_binning(binning) != GS_OK) return GS_ERR_INVALID;
    if (!frame || !frame->img || !frame->T_final || !frame->last) return GS_ERR_INVALID;
    if (!list_offsets || ((uintptr_t)list_offsets & 7u) || list_capacity < 0) return GS_ERR_INVALID;
    if (list_capacity > 0 && (!list_ids || !list_alpha)) return GS_ERR_INVALID;
    long long npx = 0;
    for (int v = 0; v < n_views; ++v) npx += (long long)cams[v].width * cams[v].height;
    if (!ws || ((uintptr_t)ws & 255u) || ws_bytes < list_scan_bytes(npx)) return GS_ERR_INVALID;
    launch_render_fwd_lists(vt, rc, (const int2 *)binning->tile_ranges, binning->gauss_ids, binning->block_mask,
                            binning->tile_order, (const float2 *)proj->xy, (const float4 *)proj->conic_opacity,
                            (const float4 *)proj->rgb_depth, frame->img, frame->T_final, frame->last, frame->depth, npx,
                            (long long *)list_offsets, list_ids, list_alpha, list_capacity, ws, status,
                            (cudaStream_t)stream);
    return cuda_status(cudaGetLastError());
}

GS_API gs_status gs_render_bwd_lists(const gs_params *params, const gs_camera *cams, int32_t n_views,
                                     const gs_raster_cfg *cfg, const gs_projected *proj, const gs_frame *frame,
                                     const int64_t *list_offsets, const int32_t *list_ids, const float *list_alpha,
                                     int64_t list_capacity, const float *dL_dimg, const float *target,
                                     const float *loss_per_view, float tau_err, const gs_params *grads,
                                     int32_t accumulate, const gs_stats *stats, void *ws, size_t ws_bytes,
                                     gs_stream stream) {
    ViewTable vt;
    RasterCfg rc;
    gs_status st = build_views(cams, n_views, cfg, vt, rc);
    if (st == GS_OK) st = check_params(params);
    if (st == GS_OK && grads) st = check_params(grads);
    if (st != GS_OK) return st;
    if (grads && (grads->ld != params->ld || grads->n != params->n || grads->sh_degree != params->sh_degree))
        return GS_ERR_INVALID;
    if (!proj || check_proj(proj, params->ld) != GS_OK) return GS_ERR_INVALID;
    if (!frame || !frame->img || !frame->T_final || !dL_dimg) return GS_ERR_INVALID;
    if (!list_offsets || list_capacity < 0 || (list_capacity > 0 && (!list_ids || !list_alpha))) return GS_ERR_INVALID;
    const bool want_stats = stats != nullptr;
    if (want_stats && (!stats->acc || stats->ld < params->n || !target)) return GS_ERR_INVALID;
    const long long nrec = (long long)n_views * params->ld;
    size_t need = 0;
    gs_bwd_workspace_size(nrec, &need);
    if (!ws || ((uintptr_t)ws & 255u) || ws_bytes < need) return GS_ERR_INVALID;
    long long npx = 0;
    for (int v = 0; v < n_views; ++v) npx += (long long)cams[v].width * cams[v].height;
    cudaStream_t s = (cudaStream_t)stream;
    float *acc = (float *)ws;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(float) * (size_t)kAccStride * nrec, s);
    if (e != cudaSuccess) return GS_ERR_CUDA;
    launch_render_bwd_lists(vt, rc, npx, (const long long *)list_offsets, list_ids, list_alpha, list_capacity,
                            (const float2 *)proj->xy, (const float4 *)proj->conic_opacity,
                            (const float4 *)proj->rgb_depth, frame->img, frame->T_final, dL_dimg, target, tau_err,
                            want_stats, acc, s);
    if (grads)
        launch_project_bwd(params->data, params->n, params->ld, params->sh_degree, vt, rc, proj->radius, acc, nrec,
                           grads->data, accumulate, loss_per_view, want_stats ? stats->acc : nullptr,
                           want_stats ? stats->ld : 0, (const float4 *)proj->color_jac, nullptr, s);
    return cuda_status(cudaGetLastError());
}

static gs_status project_bwd(const gs_params *params, const gs_camera *cams, int32_t n_views,
                             const gs_raster_cfg *cfg, const gs_projected *proj, const void *ws, size_t ws_bytes,
                             const float *loss_per_view, const gs_params *grads, int32_t accumulate,
                             const gs_stats *stats, uint8_t *rows, gs_stream stream) {
    ViewTable vt;
    RasterCfg rc;
    gs_status st = build_views(cams, n_views, cfg, vt, rc);
    if (st == GS_OK) st = check_params(params);
    if (st == GS_OK) st = check_params(grads);
    if (st != GS_OK) return st;
    if (grads->ld != params->ld || grads->n != params->n || grads->sh_degree != params->sh_degree) return GS_ERR_INVALID;
    if (!proj || check_proj(proj, params->ld) != GS_OK) return GS_ERR_INVALID;
    if (stats && (!stats->acc || stats->ld < params->n)) return GS_ERR_INVALID;
    const long long nrec = (long long)n_views * params->ld;
    size_t need = 0;
    gs_bwd_workspace_size(nrec, &need);
    if (!ws || ((uintptr_t)ws & 255u) || ws_bytes < need) return GS_ERR_INVALID;
    launch_project_bwd(params->data, params->n, params->ld, params->sh_degree, vt, rc, proj->radius,
                       (const float *)ws, nrec, grads->data, accumulate, loss_per_view,
                       stats ? stats->acc : nullptr, stats ? stats->ld : 0, (const float4 *)proj->color_jac, rows,
                       (cudaStream_t)stream);
    return cuda_status(cudaGetLastError());
}

GS_API gs_status gs_project_bwd(const gs_params *params, const gs_camera *cams, int32_t n_views,
                                const gs_raster_cfg *cfg, const gs_projected *proj, const void *ws, size_t ws_bytes,
                                const float *loss_per_view, const gs_params *grads, int32_t accumulate,
                                const gs_stats *stats, gs_stream stream) {
    return project_bwd(params, cams, n_views, cfg, proj, ws, ws_bytes, loss_per_view, grads, accumulate, stats,
                       nullptr, stream);
}

GS_API gs_status gs_project_bwd_rows(const gs_params *params, const gs_camera *cams, int32_t n_views,
                                     const gs_raster_cfg *cfg, const gs_projected *proj, const void *ws,
                                     size_t ws_bytes, const float *loss_per_view, const gs_params *grads,
                                     const gs_stats *stats, uint8_t *rows, gs_stream stream) {
    if (!rows || ((uintptr_t)rows & 3u)) return GS_ERR_INVALID;
    return project_bwd(params, cams, n_views, cfg, proj, ws, ws_bytes, loss_per_view, grads, 0, stats, rows,
                       stream);
}

GS_API gs_status gs_project_bwd_adam(const gs_params *params, const gs_camera *cams, int32_t n_views,
                                     const gs_raster_cfg *cfg, const gs_projected *proj, const void *ws,
                                     size_t ws_bytes, const float *loss_per_view, const gs_params *grads_in,
                                     float iso_weight, const gs_params *exp_avg, const gs_params *exp_avg_sq,
                                     const float lr_groups[6], float beta1, float beta2, float eps, int64_t step,
                                     const int64_t *step_device, const gs_stats *stats, gs_stream stream) {
    ViewTable vt;
    RasterCfg rc;
    gs_status st = build_views(cams, n_views, cfg, vt, rc);
    if (st == GS_OK) st = check_params(params);
    if (st == GS_OK) st = check_params(exp_avg);
    if (st == GS_OK) st = check_params(exp_avg_sq);
    if (st == GS_OK && grads_in) st = check_params(grads_in);
    if (st != GS_OK) return st;
    for (const gs_params *q : {exp_avg, exp_avg_sq, grads_in})
        if (q && (q->ld != params->ld || q->n != params->n || q->sh_degree != params->sh_degree)) return GS_ERR_INVALID;
    if (!proj || check_proj(proj, params->ld) != GS_OK) return GS_ERR_INVALID;
    if (!lr_groups || (step < 1 && !step_device) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps >= 0.0f) || !(iso_weight >= 0.0f))
        return GS_ERR_INVALID;
    if (step_device && ((uintptr_t)step_device & 7u)) return GS_ERR_INVALID;
    if (stats && (!stats->acc || stats->ld < params->n)) return GS_ERR_INVALID;
    const long long nrec = (long long)n_views * params->ld;
    size_t need = 0;
    gs_bwd_workspace_size(nrec, &need);
    if (!ws || ((uintptr_t)ws & 255u) || ws_bytes < need) return GS_ERR_INVALID;
    launch_project_bwd_adam(params->data, params->n, params->ld, params->sh_degree, vt, rc, proj->radius,
                            (const float *)ws, nrec, grads_in ? grads_in->data : nullptr, exp_avg->data,
                            exp_avg_sq->data, lr_groups, beta1, beta2, eps, step, (const long long *)step_device,
                            iso_weight, loss_per_view, stats ? stats->acc : nullptr, stats ? stats->ld : 0,
                            (cudaStream_t)stream);
    return cuda_status(cudaGetLastError());
}

static gs_status adam(const gs_params *params, const gs_params *grads, const gs_params *exp_avg,
                      const gs_params *exp_avg_sq, const float lr_groups[6], float beta1, float beta2, float eps,
                      int64_t step, const int64_t *step_device, const uint8_t *rows, gs_stream stream,
                      int part = 0, const int32_t *radius = nullptr, int n_views = 0) {
    gs_status st = check_params(params);
    if (st == GS_OK) st = check_params(grads);
    if (st == GS_OK) st = check_params(exp_avg);
    if (st == GS_OK) st = check_params(exp_avg_sq);
    if (st != GS_OK) return st;
    for (const gs_params *q : {grads, exp_avg, exp_avg_sq})
        if (q->ld != params->ld || q->n != params->n || q->sh_degree != params->sh_degree) return GS_ERR_INVALID;
    if (!lr_groups || (step < 1 && !step_device) || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps >= 0.0f))
        return GS_ERR_INVALID;
    if (step_device && ((uintptr_t)step_device & 7u)) return GS_ERR_INVALID;
    launch_adam(params->data, grads->data, exp_avg->data, exp_avg_sq->data, params->ld, GS_PLANES(params->sh_degree),
                lr_groups, beta1, beta2, eps, step, (const long long *)step_device, rows, (cudaStream_t)stream, part,
                radius, n_views);
    return cuda_status(cudaGetLastError());
}

GS_API gs_status gs_adam(const gs_params *params, const gs_params *grads, const gs_params *exp_avg,
                         const gs_params *exp_avg_sq, const float lr_groups[6], float beta1, float beta2, float eps,
                         int64_t step, const int64_t *step_device, gs_stream stream) {
    return adam(params, grads, exp_avg, exp_avg_sq, lr_groups, beta1, beta2, eps, step, step_device, nullptr,
                stream);
}

GS_API gs_status gs_adam_rows(const gs_params *params, const gs_params *grads, const gs_params *exp_avg,
                              const gs_params *exp_avg_sq, const uint8_t *rows, const float lr_groups[6],
                              float beta1, float beta2, float eps, int64_t step, const int64_t *step_device,
                              gs_stream stream) {
    if (!rows || ((uintptr_t)rows & 3u)) return GS_ERR_INVALID;
    return adam(params, grads, exp_avg, exp_avg_sq, lr_groups, beta1, beta2, eps, step, step_device, rows, stream);
}

GS_API gs_status gs_adam_part(const gs_params *params, const gs_params *grads, const gs_params *exp_avg,
                              const gs_params *exp_avg_sq, const uint8_t *rows, const int32_t *radius,
                              int32_t n_views, int32_t part, const float lr_groups[6], float beta1, float beta2,
                              float eps, int64_t step, const int64_t *step_device, gs_stream stream) {
    if (part == 1) {
        if (!rows || ((uintptr_t)rows & 3u)) return GS_ERR_INVALID;
    } else if (part == 2) {
        if (!radius || ((uintptr_t)radius & 15u) || n_views < 1 || n_views > GS_MAX_VIEWS) return GS_ERR_INVALID;
        if (!grads) grads = params;  // not read
    } else {
        return GS_ERR_INVALID;
    }
    return adam(params, grads, exp_avg, exp_avg_sq, lr_groups, beta1, beta2, eps, step, step_device, rows, stream,
                part, radius, n_views);
}

GS_API gs_status gs_prune_stats(const gs_stats *stats, int64_t n, int32_t n_views, float tau_d, float tau_p,
                                const gs_chunk_scores *out, void *ws, size_t ws_bytes, gs_stream stream) {
    if (!stats || !stats->acc || n < 0 || stats->ld < n || n_views < 1 || !out || !out->S_d || !out->S_p ||
        !out->prune_max || !out->densify || !out->prune || !ws || ws_bytes < prune_workspace_bytes(n))
        return GS_ERR_INVALID;
    launch_prune(stats->acc, stats->ld, n, n_views, tau_d, tau_p, out->S_d, out->S_p, out->prune_max, out->densify,
                 out->prune, ws, (cudaStream_t)stream);
    return cuda_status(cudaGetLastError());
}

GS_API gs_status gs_reorder_workspace_size(int64_t n, int64_t ld, int32_t max_planes, size_t *bytes) {
    if (n < 0 || ld < n || max_planes < 1 || !bytes) return GS_ERR_INVALID;
    *bytes = reorder_workspace_bytes(n, ld, max_planes);
    return GS_OK;
}

GS_API gs_status gs_reorder(const gs_params *params, const gs_plane_set *extra, int32_t n_extra, int32_t *perm,
                            void *ws, size_t ws_bytes, gs_stream stream) {
    constexpr int kMaxExtra = 16;
    gs_status st = check_params(params);
    if (st != GS_OK) return st;
    if (n_extra < 0 || n_extra > kMaxExtra || (n_extra > 0 && !extra) || ((uintptr_t)perm & 3u)) return GS_ERR_INVALID;
    float *sets[kMaxExtra];
    int planes[kMaxExtra];
    int maxp = GS_PLANES(params->sh_degree);
    for (int e = 0; e < n_extra; ++e) {
        const gs_plane_set &x = extra[e];
        if (!x.data || !aligned16(x.data) || x.ld != params->ld || x.planes < 1 || x.planes > 65535 ||
            x.data == params->data)
            return GS_ERR_INVALID;
        sets[e] = x.data;
        planes[e] = x.planes;
        maxp = std::max(maxp, (int)x.planes);
    }
    if (!ws || ((uintptr_t)ws & 255u) || ws_bytes < reorder_workspace_bytes(params->n, params->ld, maxp))
        return GS_ERR_INVALID;
    return cuda_status(launch_reorder(params->data, params->n, params->ld, GS_PLANES(params->sh_degree), sets,
                                      planes, n_extra, perm, ws, (cudaStream_t)stream));
}

GS_API gs_status gs_actions_workspace_size(int64_t n, size_t *bytes) {
    if (n < 0 || !bytes) return GS_ERR_INVALID;
    *bytes = actions_workspace_bytes(n);
    return GS_OK;
}

GS_API gs_status gs_densify_prune(const gs_params *src, const gs_params *src_m, const gs_params *src_v,
                                  const uint8_t *densify, const uint8_t *prune, const float *noise,
                                  float split_log_scale, float split_factor, const gs_params *dst,
                                  const gs_params *dst_m, const gs_params *dst_v, int64_t *n_out, int32_t *status,
                                  void *ws, size_t ws_bytes, gs_stream stream) {
    gs_status st = check_params(src);
    if (st == GS_OK) st = check_params(dst);
    if (st != GS_OK) return st;
    const bool moments = src_m || src_v || dst_m || dst_v;
    if (moments) {
        for (const gs_params *q : {src_m, src_v, dst_m, dst_v})
            if ((st = check_params(q)) != GS_OK) return st;
        for (const gs_params *q : {src_m, src_v})
            if (q->ld != src->ld || q->n != src->n || q->sh_degree != src->sh_degree) return GS_ERR_INVALID;
        for (const gs_params *q : {dst_m, dst_v})
            if (q->ld != dst->ld || q->sh_degree != dst->sh_degree) return GS_ERR_INVALID;
    }
    if (dst->sh_degree != src->sh_degree || !densify || !prune || !noise || !aligned16(noise) || !n_out ||
        ((uintptr_t)n_out & 7u) || !(split_factor > 0.0f) || !(split_log_scale == split_log_scale) || !ws ||
        ((uintptr_t)ws & 255u) || ws_bytes < actions_workspace_bytes(src->n) || dst->data == src->data)
        return GS_ERR_INVALID;
    return cuda_status(launch_actions(src->data, moments ? src_m->data : nullptr, moments ? src_v->data : nullptr,
                                      src->n, src->ld, GS_PLANES(src->sh_degree), densify, prune, noise,
                                      split_log_scale, (float)std::log((double)split_factor), dst->data,
                                      moments ? dst_m->data : nullptr, moments ? dst_v->data : nullptr, dst->ld,
                                      (long long *)n_out, status, ws, (cudaStream_t)stream));
}

GS_API gs_status gs_mlp_push_blend(const gs_stats *stats, int64_t n, float *ring, int64_t ring_ld, int32_t slot,
                                   gs_stream stream) {
    if (!stats || !stats->acc || n < 0 || stats->ld < n || !ring || !aligned16(ring) || ring_ld < n ||
        slot < 0 || slot >= GS_MLP_RING)
        return GS_ERR_INVALID;
    return cuda_status(launch_mlp_push_blend(stats->acc, stats->ld, n, ring, ring_ld, slot, (cudaStream_t)stream));
}

GS_API gs_status gs_mlp_features(const gs_params *params, const gs_stats *stats, const float *ring, int32_t head,
                                 const float cam_centre[3], float *feat, gs_stream stream) {
    gs_status st = check_params(params);
    if (st != GS_OK) return st;
    if (!stats || !stats->acc || stats->ld != params->ld || !ring || !aligned16(ring) || head < 0 ||
        head >= GS_MLP_RING || !cam_centre || !feat || !aligned16(feat))
        return GS_ERR_INVALID;
    return cuda_status(launch_mlp_features(params->data, params->n, params->ld, stats->acc, stats->ld, ring, head,
                                           cam_centre, feat, (cudaStream_t)stream));
}

GS_API gs_status gs_mlp_forward(const float *feat, int64_t n, int64_t ld, const float *weights, float *prob,
                                uint8_t *densify, uint8_t *prune, int32_t *status, int64_t max_polls,
                                gs_stream stream) {
    if (!feat || !aligned16(feat) || n < 0 || ld < n || (ld & 3) || !weights || !aligned16(weights) ||
        (prob && !aligned16(prob)))
        return GS_ERR_INVALID;
    return cuda_status(launch_mlp_forward(feat, n, ld, weights, prob, densify, prune, status, max_polls,
                                         (cudaStream_t)stream));
}

GS_API gs_status gs_mlp_train_grad(const float *feat, const uint8_t *y_densify, const uint8_t *y_prune, int64_t n,
                                   int64_t ld, const float *weights, float *grad, float *loss, int32_t *status,
                                   gs_stream stream) {
    if (!feat || !aligned16(feat) || n < 1 || ld < n || (ld & 3) || !y_densify || !y_prune || !weights ||
        !aligned16(weights) || !grad || !aligned16(grad) || !loss)
        return GS_ERR_INVALID;
    return cuda_status(launch_mlp_train(feat, y_densify, y_prune, n, ld, weights, grad, loss, status,
                                        (cudaStream_t)stream));
}

GS_API gs_status gs_mlp_adam(float *weights, const float *grad, float *exp_avg, float *exp_avg_sq, float lr,
                             float beta1, float beta2, float eps, int64_t step, gs_stream stream) {
    if (!weights || !grad || !exp_avg || !exp_avg_sq || step < 1 || !(beta1 >= 0.0f && beta1 < 1.0f) ||
        !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps >= 0.0f) || !(lr >= 0.0f))
        return GS_ERR_INVALID;
    return cuda_status(launch_mlp_adam(weights, grad, exp_avg, exp_avg_sq, lr, beta1, beta2, eps, step,
                                       (cudaStream_t)stream));
}

namespace {

// Normalised 1D weights of the sampled Gaussian (their outer product is the
// normalised 2D kernel).
gs_status init_blur(const gs_init_cfg *cfg, InitBlur &bw) {
    bw = InitBlur{};
    const float sig[2] = {cfg->sigma1, cfg->sigma2};
    for (int j = 0; j < 2; ++j) {
        if (!(sig[j] > 0.0f) || std::ceil(3.0 * (double)sig[j]) > GS_INIT_MAX_RADIUS) return GS_ERR_INVALID;
        const int r = (int)std::ceil(3.0 * (double)sig[j]);
        double w[GS_INIT_MAX_RADIUS + 1], sum = 0.0;
        for (int k = 0; k <= r; ++k) {
            w[k] = std::exp(-(double)(k * k) / (2.0 * (double)sig[j] * (double)sig[j]));
            sum += k ? 2.0 * w[k] : w[k];
        }
        float *dst = j ? bw.w2 : bw.w1;
        for (int k = 0; k <= r; ++k) dst[k] = (float)(w[k] / sum);
        (j ? bw.r2 : bw.r1) = r;
    }
    bw.R = bw.r1 > bw.r2 ? bw.r1 : bw.r2;
    if (!(cfg->intensity_scale > 0.0f) || !std::isfinite(cfg->intensity_scale)) return GS_ERR_INVALID;
    bw.scale = cfg->intensity_scale;
    return GS_OK;
}

gs_status init_lod(const gs_init_cfg *cfg, InitLod &lod) {
    lod = InitLod{};
    if (cfg->levels < 1 || cfg->levels > GS_INIT_MAX_LEVELS || !(cfg->near_z >= 0.0f)) return GS_ERR_INVALID;
    for (int l = 0; l < cfg->levels; ++l) {
        if (!(cfg->voxel[l] > 0.0f) || !std::isfinite(cfg->voxel[l]) || !(cfg->max_dist[l] > 0.0f) ||
            (l && !(cfg->max_dist[l] > cfg->max_dist[l - 1])))
            return GS_ERR_INVALID;
        lod.voxel[l] = cfg->voxel[l];
        lod.max_dist[l] = cfg->max_dist[l];
    }
    lod.levels = cfg->levels;
    lod.near_z = cfg->near_z;
    return GS_OK;
}

bool init_size_ok(long long W, long long H) { return W >= 1 && H >= 1 && W * H <= 0x7fffffffll; }

gs_status check_table(const gs_voxel_table *t) {
    if (!t || !t->keys || !t->ids || !t->owner || !aligned16(t->keys) || !aligned16(t->ids) || !aligned16(t->owner) ||
        t->capacity < 1024 || t->capacity > (1ll << 30) || (t->capacity & (t->capacity - 1)))
        return GS_ERR_INVALID;
    return GS_OK;
}

}  // namespace

GS_API gs_status gs_voxel_table_reset(const gs_voxel_table *table, gs_stream stream) {
    gs_status st = check_table(table);
    if (st != GS_OK) return st;
    return cuda_status(launch_voxel_reset((unsigned long long *)table->keys, table->ids, table->owner,
                                          table->capacity, (cudaStream_t)stream));
}

GS_API gs_status gs_init_workspace_size(int32_t width, int32_t height, size_t *bytes) {
    if (!bytes || !init_size_ok(width, height)) return GS_ERR_INVALID;
    *bytes = init_workspace_bytes(width, height);
    return GS_OK;
}

GS_API gs_status gs_init_probability(const float *img, const float *depth, const float *img_r, const float *depth_r,
                                     int32_t width, int32_t height, const gs_init_cfg *cfg, float *prob, void *ws,
                                     size_t ws_bytes, gs_stream stream) {
    if (!cfg || !init_size_ok(width, height) || !img || !depth || !aligned16(img) || !aligned16(depth) ||
        (!img_r) != (!depth_r) || (img_r && (!aligned16(img_r) || !aligned16(depth_r))) || !prob ||
        !aligned16(prob) || !ws || ((uintptr_t)ws & 255u) || ws_bytes < init_workspace_bytes(width, height) ||
        !(cfg->lambda >= 0.0f && cfg->lambda <= 1.0f))
        return GS_ERR_INVALID;
    InitBlur bw;
    gs_status st = init_blur(cfg, bw);
    if (st != GS_OK) return st;
    return cuda_status(launch_init_probability(img, depth, img_r, depth_r, width, height, bw, cfg->lambda, prob, ws,
                                               (cudaStream_t)stream));
}

GS_API gs_status gs_init_insert(const float *prob, const float *uniform, const float *depth, const gs_camera *cam,
                                const gs_init_cfg *cfg, const gs_voxel_table *table, const gs_anchor_set *anchors,
                                uint8_t *selected, int32_t *status, void *ws, size_t ws_bytes, gs_stream stream) {
    if (!cam || !cfg || !init_size_ok(cam->width, cam->height) || !(cam->fx > 0.0f) || !(cam->fy > 0.0f) || !prob ||
        !uniform || !depth || !aligned16(prob) || !aligned16(uniform) || !aligned16(depth) || !anchors ||
        !anchors->pos || !aligned16(anchors->pos) || !anchors->level || !anchors->pixel || !anchors->count ||
        ((uintptr_t)anchors->count & 7u) || anchors->ld < 0 || !ws || ((uintptr_t)ws & 255u) ||
        ws_bytes < init_workspace_bytes(cam->width, cam->height))
        return GS_ERR_INVALID;
    gs_status st = check_table(table);
    if (st != GS_OK) return st;
    InitLod lod;
    if ((st = init_lod(cfg, lod)) != GS_OK) return st;
    InitCam c;
    for (int i = 0; i < 9; ++i) c.R[i] = cam->R[i];
    for (int i = 0; i < 3; ++i) c.t[i] = cam->t[i];
    c.fx = cam->fx;
    c.fy = cam->fy;
    c.cx = cam->cx;
    c.cy = cam->cy;
    return cuda_status(launch_init_insert(prob, uniform, depth, cam->width, cam->height, c, lod,
                                          (unsigned long long *)table->keys, table->ids, table->owner,
                                          table->capacity, anchors->pos, anchors->level, anchors->pixel,
                                          (long long *)anchors->count, anchors->ld, selected, status, ws,
                                          (cudaStream_t)stream));
}

GS_API gs_status gs_voxel_lookup(const gs_voxel_table *table, const int32_t *vox, int64_t n, int64_t ld, int32_t *ids,
                                 gs_stream stream) {
    gs_status st = check_table(table);
    if (st != GS_OK) return st;
    if (n < 0 || ld < n || (n > 0 && (!vox || !ids || !aligned16(vox)))) return GS_ERR_INVALID;
    return cuda_status(launch_voxel_lookup((const unsigned long long *)table->keys, table->ids, table->capacity, vox,
                                           n, ld, ids, (cudaStream_t)stream));
}

namespace {

gs_status anchor_view(const gs_anchor_params *a, const float cam_centre[3], const float *max_dist, int levels,
                      AnchorView &v) {
    if (!a || !a->data || !a->pos || !a->level || !aligned16(a->data) || !aligned16(a->pos) || a->n < 0 ||
        a->ld < a->n || (a->ld & 3) || !cam_centre || !max_dist || levels < 1 || levels > GS_INIT_MAX_LEVELS)
        return GS_ERR_INVALID;
    v = AnchorView{};
    for (int k = 0; k < 3; ++k) v.c[k] = cam_centre[k];
    for (int l = 0; l < levels; ++l) {
        if (!(max_dist[l] > 0.0f) || (l && !(max_dist[l] > max_dist[l - 1]))) return GS_ERR_INVALID;
        v.lo[l] = l ? max_dist[l - 1] : 0.0f;
        v.hi[l] = max_dist[l];
    }
    v.levels = levels;
    return GS_OK;
}

gs_status check_decoded(const gs_anchor_params *a, const gs_params *out) {
    gs_status st = check_params(out);
    if (st != GS_OK) return st;
    if (out->sh_degree != 0 || out->n != (int64_t)GS_ANCHOR_K * a->ld) return GS_ERR_INVALID;
    return GS_OK;
}

}  // namespace

GS_API gs_status gs_anchor_decode(const gs_anchor_params *a, const float *weights, const float cam_centre[3],
                                  const float *max_dist, int32_t levels, const gs_params *out, int32_t *status,
                                  int64_t max_polls, gs_stream stream) {
    AnchorView v;
    gs_status st = anchor_view(a, cam_centre, max_dist, levels, v);
    if (st == GS_OK) st = check_decoded(a, out);
    if (st != GS_OK) return st;
    if (!weights || !aligned16(weights)) return GS_ERR_INVALID;
    return cuda_status(launch_anchor_decode(a->data, a->pos, a->level, a->n, a->ld, weights, v, out->data, out->ld,
                                            status, max_polls, (cudaStream_t)stream));
}

GS_API gs_status gs_anchor_decode_bwd(const gs_anchor_params *a, const float *weights, const float cam_centre[3],
                                      const float *max_dist, int32_t levels, const gs_params *grad_out,
                                      float *grad_anchor, float *grad_weights, int32_t *status, int64_t max_polls,
                                      gs_stream stream) {
    AnchorView v;
    gs_status st = anchor_view(a, cam_centre, max_dist, levels, v);
    if (st == GS_OK) st = check_decoded(a, grad_out);
    if (st != GS_OK) return st;
    if (!weights || !aligned16(weights) || !grad_anchor || !aligned16(grad_anchor) || !grad_weights ||
        !aligned16(grad_weights))
        return GS_ERR_INVALID;
    return cuda_status(launch_anchor_decode_bwd(a->data, a->pos, a->level, a->n, a->ld, weights, v, grad_out->data,
                                                grad_out->ld, grad_anchor, grad_weights, status, max_polls,
                                                (cudaStream_t)stream));
}

GS_API gs_status gs_adam_flat(float *p, const float *g, float *m, float *v, int64_t n, float lr, float beta1,
                              float beta2, float eps, int64_t step, const int64_t *step_device, gs_stream stream) {
    if (n < 0 || (n > 0 && (!p || !g || !m || !v)) || (step < 1 && !step_device) ||
        !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps >= 0.0f) || !(lr >= 0.0f) ||
        ((uintptr_t)step_device & 7u))
        return GS_ERR_INVALID;
    return cuda_status(launch_adam_flat(p, g, m, v, n, lr, beta1, beta2, eps, step, (const long long *)step_device,
                                        (cudaStream_t)stream));
}
