// render.cu -- per-tile compositing kernels: front-to-back forward and
// back-to-front backward (Supp. D.2: C = sum_j c_j alpha_j T_j, T_j =
// prod_{m<j}(1 - alpha_m)).  One CTA per tile of 256 pixels (16x16, 8x32 or
// 32x8), one thread per pixel; the tile's Gaussians are staged through shared
// memory kBatch at a time with coalesced gathers of the projection records.
#include "gs_internal.cuh"
#include "gs_kernels.h"

namespace gs {

struct TileCtx {
    int view, px, py;
    bool inside;
    long long pix;  // pixel index in the frame layout (per-pixel planes)
    long long img;  // index of the red plane entry in the frame layout
    long long plane;
};

__device__ __forceinline__ TileCtx tile_ctx(const ViewTable &vt, int tile) {
    TileCtx t;
    t.view = view_of_tile(vt, tile);
    const ViewDesc &c = vt.v[t.view];
    const int local = tile - c.tile_offset;
    const int ty = local / c.GW, tx = local - ty * c.GW;
    t.px = tx * vt.tile_w + (int)(threadIdx.x % vt.tile_w);
    t.py = ty * vt.tile_h + (int)(threadIdx.x / vt.tile_w);
    t.inside = t.px < c.W && t.py < c.H;
    t.plane = (long long)c.W * c.H;
    t.pix = c.pix_offset + (long long)t.py * c.W + t.px;
    t.img = 3 * c.pix_offset + (long long)t.py * c.W + t.px;
    return t;
}

__global__ void __launch_bounds__(kTilePixels) k_render_fwd(ViewTable vt, RasterCfg cfg,
                                                              const int2 *__restrict__ ranges,
                                                              const int *__restrict__ ids,
                                                              const float2 *__restrict__ xy,
                                                              const float4 *__restrict__ co,
                                                              const float4 *__restrict__ rgbd,
                                                              float *__restrict__ img, float *__restrict__ T_final,
                                                              int *__restrict__ last, float *__restrict__ depth) {
    __shared__ float2 s_xy[kBatch];
    __shared__ float4 s_co[kBatch];
    __shared__ float4 s_rgbd[kBatch];
    const int tile = blockIdx.x;
    const TileCtx t = tile_ctx(vt, tile);
    const int2 rg = ranges[tile];
    const int n = rg.y - rg.x;
    const float fx = t.px + 0.5f, fy = t.py + 0.5f;

    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, Dd = 0.0f;
    int lastc = 0;
    bool done = !t.inside;
    for (int b = 0; b < n; b += kBatch) {
        if (__syncthreads_count(done) == kTilePixels) break;
        const int j = b + (int)threadIdx.x;
        if (j < n) {
            const int g = ids[rg.x + j];
            s_xy[threadIdx.x] = xy[g];
            s_co[threadIdx.x] = co[g];
            s_rgbd[threadIdx.x] = rgbd[g];
        }
        __syncthreads();
        const int cnt = min(kBatch, n - b);
        for (int k = 0; k < cnt && !done; ++k) {
            const float2 p = s_xy[k];
            const float4 q = s_co[k];
            const float power = gauss_power(q.x, q.y, q.z, fx - p.x, fy - p.y);
            if (power > 0.0f) continue;
            const float alpha = fminf(cfg.alpha_max, q.w * __expf(power));
            if (alpha < cfg.alpha_min) continue;
            const float Tn = T * (1.0f - alpha);
            if (Tn < cfg.t_min) { done = true; break; }
            const float4 c = s_rgbd[k];
            const float w = alpha * T;
            C0 += c.x * w; C1 += c.y * w; C2 += c.z * w; Dd += c.w * w;
            T = Tn;
            lastc = b + k + 1;
        }
    }
    if (t.inside) {
        img[t.img] = C0 + T * cfg.bg[0];
        img[t.img + t.plane] = C1 + T * cfg.bg[1];
        img[t.img + 2 * t.plane] = C2 + T * cfg.bg[2];
        T_final[t.pix] = T;
        last[t.pix] = lastc;
        if (depth) depth[t.pix] = Dd;
    }
}

__device__ __forceinline__ float warp_sum(float v) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <bool STATS>
__global__ void __launch_bounds__(kTilePixels) k_render_bwd(ViewTable vt, RasterCfg cfg,
                                                              const int2 *__restrict__ ranges,
                                                              const int *__restrict__ ids,
                                                              const float2 *__restrict__ xy,
                                                              const float4 *__restrict__ co,
                                                              const float4 *__restrict__ rgbd,
                                                              const float *__restrict__ img,
                                                              const float *__restrict__ T_final,
                                                              const int *__restrict__ last,
                                                              const float *__restrict__ dL_dimg,
                                                              const float *__restrict__ dL_ddepth,
                                                              const float *__restrict__ target, float tau_err,
                                                              float *__restrict__ acc, long long nrec) {
    __shared__ float2 s_xy[kBatch];
    __shared__ float4 s_co[kBatch];
    __shared__ float4 s_rgbd[kBatch];
    __shared__ int s_id[kBatch];
    __shared__ int s_max;
    const int tile = blockIdx.x;
    const TileCtx t = tile_ctx(vt, tile);
    const int2 rg = ranges[tile];
    const float fx = t.px + 0.5f, fy = t.py + 0.5f;
    const int lane = threadIdx.x & 31;

    float T = 1.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f, gD = 0.0f, mask = 0.0f;
    int lst = 0;
    if (t.inside) {
        T = T_final[t.pix];
        lst = last[t.pix];
        g0 = dL_dimg[t.img];
        g1 = dL_dimg[t.img + t.plane];
        g2 = dL_dimg[t.img + 2 * t.plane];
        if (dL_ddepth) gD = dL_ddepth[t.pix];
        if (STATS) {
            const float e = fabsf(target[t.img] - img[t.img]) + fabsf(target[t.img + t.plane] - img[t.img + t.plane]) +
                            fabsf(target[t.img + 2 * t.plane] - img[t.img + 2 * t.plane]);
            mask = e > tau_err ? 1.0f : 0.0f;
        }
    }
    // colour (and depth) behind the current Gaussian, normalised by the
    // transmittance in front of it; starts as the background
    float R0 = cfg.bg[0], R1 = cfg.bg[1], R2 = cfg.bg[2], RD = 0.0f;

    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    atomicMax(&s_max, lst);
    __syncthreads();
    const int nmax = s_max;

    for (int bend = nmax; bend > 0; bend -= kBatch) {
        const int bstart = max(0, bend - kBatch);
        __syncthreads();
        {
            const int j = bstart + (int)threadIdx.x;
            if (j < bend) {
                const int g = ids[rg.x + j];
                s_id[threadIdx.x] = g;
                s_xy[threadIdx.x] = xy[g];
                s_co[threadIdx.x] = co[g];
                s_rgbd[threadIdx.x] = rgbd[g];
            }
        }
        __syncthreads();
        for (int j = bend - 1; j >= bstart; --j) {
            const int k = j - bstart;
            bool on = j < lst;
            float alpha = 0.0f, G = 0.0f, dx = 0.0f, dy = 0.0f;
            const float2 p = s_xy[k];
            const float4 q = s_co[k];
            if (on) {
                dx = fx - p.x;
                dy = fy - p.y;
                const float power = gauss_power(q.x, q.y, q.z, dx, dy);
                if (power > 0.0f) {
                    on = false;
                } else {
                    G = __expf(power);
                    alpha = fminf(cfg.alpha_max, q.w * G);
                    if (alpha < cfg.alpha_min) on = false;
                }
            }
            float vu = 0, vv = 0, va = 0, vb = 0, vc = 0, vo = 0, vr = 0, vg = 0, vbl = 0, vz = 0;
            float som = 0, ska = 0, smw = 0;
            if (on) {
                const float4 c = s_rgbd[k];
                T = T / (1.0f - alpha);  // transmittance in front of this Gaussian
                const float w = alpha * T;
                vr = g0 * w; vg = g1 * w; vbl = g2 * w; vz = gD * w;
                const float dLda = T * (g0 * (c.x - R0) + g1 * (c.y - R1) + g2 * (c.z - R2) + gD * (c.w - RD));
                R0 = alpha * c.x + (1.0f - alpha) * R0;
                R1 = alpha * c.y + (1.0f - alpha) * R1;
                R2 = alpha * c.z + (1.0f - alpha) * R2;
                RD = alpha * c.w + (1.0f - alpha) * RD;
                if (q.w * G <= cfg.alpha_max) {  // alpha not clamped
                    vo = dLda * G;
                    const float dp = dLda * q.w * G;
                    vu = dp * (q.x * dx + q.y * dy);
                    vv = dp * (q.z * dy + q.y * dx);
                    va = -0.5f * dp * dx * dx;
                    vb = -dp * dx * dy;
                    vc = -0.5f * dp * dy * dy;
                }
                if (STATS) { som = 1.0f; ska = mask; smw = w; }
            }
            if (__any_sync(0xffffffffu, on)) {
                vu = warp_sum(vu); vv = warp_sum(vv); va = warp_sum(va); vb = warp_sum(vb); vc = warp_sum(vc);
                vo = warp_sum(vo); vr = warp_sum(vr); vg = warp_sum(vg); vbl = warp_sum(vbl);
                if (dL_ddepth) vz = warp_sum(vz);
                if (STATS) { som = warp_sum(som); ska = warp_sum(ska); smw = warp_max(smw); }
                if (lane == 0) {
                    const long long r = s_id[k];
                    atomicAdd(&acc[kAccU * nrec + r], vu);
                    atomicAdd(&acc[kAccV * nrec + r], vv);
                    atomicAdd(&acc[kAccA * nrec + r], va);
                    atomicAdd(&acc[kAccB * nrec + r], vb);
                    atomicAdd(&acc[kAccC * nrec + r], vc);
                    atomicAdd(&acc[kAccO * nrec + r], vo);
                    atomicAdd(&acc[kAccR * nrec + r], vr);
                    atomicAdd(&acc[kAccG * nrec + r], vg);
                    atomicAdd(&acc[kAccBl * nrec + r], vbl);
                    if (dL_ddepth) atomicAdd(&acc[kAccZ * nrec + r], vz);
                    if (STATS) {
                        atomicAdd(&acc[kAccOmega * nrec + r], som);
                        if (ska > 0.0f) atomicAdd(&acc[kAccKappa * nrec + r], ska);
                        atomicMax((int *)&acc[kAccMaxW * nrec + r], __float_as_int(smw));  // w >= 0
                    }
                }
            }
        }
    }
}

static int total_tiles(const ViewTable &vt) { return vt.total_tiles; }

void launch_render_fwd(const ViewTable &vt, const RasterCfg &cfg, const int2 *ranges, const int *ids, const float2 *xy,
                       const float4 *co, const float4 *rgbd, float *img, float *T_final, int *last, float *depth,
                       cudaStream_t s) {
    const int nt = total_tiles(vt);
    if (nt <= 0) return;
    k_render_fwd<<<nt, kTilePixels, 0, s>>>(vt, cfg, ranges, ids, xy, co, rgbd, img, T_final, last, depth);
}

void launch_render_bwd(const ViewTable &vt, const RasterCfg &cfg, const int2 *ranges, const int *ids,
                       const float2 *xy, const float4 *co, const float4 *rgbd, const float *img, const float *T_final,
                       const int *last, const float *dL_dimg, const float *dL_ddepth, const float *target,
                       float tau_err, bool stats, float *acc, long long nrec, cudaStream_t s) {
    const int nt = total_tiles(vt);
    if (nt <= 0) return;
    if (stats)
        k_render_bwd<true><<<nt, kTilePixels, 0, s>>>(vt, cfg, ranges, ids, xy, co, rgbd, img, T_final, last, dL_dimg,
                                                      dL_ddepth, target, tau_err, acc, nrec);
    else
        k_render_bwd<false><<<nt, kTilePixels, 0, s>>>(vt, cfg, ranges, ids, xy, co, rgbd, img, T_final, last,
                                                       dL_dimg, dL_ddepth, target, tau_err, acc, nrec);
}

}  // namespace gs
