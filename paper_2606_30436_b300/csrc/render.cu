// render.cu -- compositing kernels: front-to-back forward and back-to-front
// backward (Supp. D.2: C = sum_j c_j alpha_j T_j, T_j = prod_{m<j}(1 - alpha_m)).
//
// Work unit = one warp = one 8x4 pixel block of a tile (a tile of 256 pixels,
// 16x16, 8x32 or 32x8, has eight blocks); lane = pixel.  Each warp walks its
// tile's depth-ordered pair list on its own, 32 pairs per step, with the
// records of the next 32 pairs already in flight (ids two steps ahead).  A
// pair is evaluated only if the Gaussian's alpha >= alpha_min ellipse can reach
// the warp's block (a conservative bounding-box test, so skipping is exact);
// the relevant records go through warp-private shared memory.  There is no
// CTA-wide barrier, so a block whose pixels saturate early retires at once
// while the few deep blocks of a vanishing-point tile run on their own warps.
#include "gs_internal.cuh"
#include "gs_kernels.h"

namespace gs {

constexpr int kWarps = 4;  // warps (work units) per CTA

struct Unit {
    int view, px, py;
    float bx0, by0;  // block's first pixel centre minus 0.5 (pixel-index space)
    bool inside;
    long long pix, img, plane;
};

__device__ __forceinline__ Unit unit_ctx(const ViewTable &vt, int tile, int blk) {
    Unit t;
    t.view = view_of_tile(vt, tile);
    const ViewDesc &c = vt.v[t.view];
    const int local = tile - c.tile_offset;
    const int ty = local / c.GW, tx = local - ty * c.GW;
    const int ncols = vt.tile_w >> 3;
    const int ox = tx * vt.tile_w + 8 * (blk % ncols), oy = ty * vt.tile_h + 4 * (blk / ncols);
    const int lane = threadIdx.x & 31;
    t.px = ox + (lane & 7);
    t.py = oy + (lane >> 3);
    t.bx0 = (float)ox;
    t.by0 = (float)oy;
    t.inside = t.px < c.W && t.py < c.H;
    t.plane = (long long)c.W * c.H;
    t.pix = c.pix_offset + (long long)t.py * c.W + t.px;
    t.img = 3 * c.pix_offset + (long long)t.py * c.W + t.px;
    return t;
}

// Can the Gaussian reach alpha >= alpha_min at a pixel centre of the 8x4 block
// with first pixel (bx0, by0)?  alpha >= alpha_min iff d^T Q d <= tau,
// tau = 2 ln(o / alpha_min); the ellipse's bounding box has half-widths
// sqrt(tau Sigma'_xx), sqrt(tau Sigma'_yy) with Sigma' = Q^-1.  tau gets an
// additive margin (alpha relative errors up to 1%) and the box 0.05 px, so
// rounding never skips a Gaussian the per-pixel test would keep.
__device__ __forceinline__ bool reaches_block(float2 p, float4 q, float alpha_min, float bx0, float by0) {
    if (q.w < alpha_min) return false;
    const float tau = 2.0f * __logf(q.w / alpha_min) + 0.02f;
    const float det = q.x * q.z - q.y * q.y;
    if (!(det > 0.0f)) return true;
    const float idet = 1.0f / det;
    const float ex = sqrtf(tau * q.z * idet) + 0.05f;
    const float ey = sqrtf(tau * q.x * idet) + 0.05f;
    // pixel i has centre i + 0.5: compare in pixel-index space
    const float cx = p.x - 0.5f, cy = p.y - 0.5f;
    return cx + ex >= bx0 && cx - ex <= bx0 + 7.0f && cy + ey >= by0 && cy - ey <= by0 + 3.0f;
}

struct Rec {
    float2 p;
    float4 q, c;
    int id;
};

__device__ __forceinline__ void load_rec(Rec &r, const float2 *__restrict__ xy, const float4 *__restrict__ co,
                                         const float4 *__restrict__ rgbd, int id, bool valid) {
    r.id = id;
    if (valid) {
        r.p = xy[id];
        r.q = co[id];
        r.c = rgbd[id];
    } else {
        r.p = make_float2(0.f, 0.f);
        r.q = make_float4(0.f, 0.f, 0.f, 0.f);  // opacity 0: never reaches a block
        r.c = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__global__ void __launch_bounds__(32 * kWarps) k_render_fwd(ViewTable vt, RasterCfg cfg,
                                                              const int2 *__restrict__ ranges,
                                                              const int *__restrict__ ids,
                                                              const float2 *__restrict__ xy,
                                                              const float4 *__restrict__ co,
                                                              const float4 *__restrict__ rgbd,
                                                              float *__restrict__ img, float *__restrict__ T_final,
                                                              int *__restrict__ last, float *__restrict__ depth) {
    __shared__ float2 s_p[kWarps][32];
    __shared__ float4 s_q[kWarps][32];
    __shared__ float4 s_c[kWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int unit = blockIdx.x * kWarps + warp;
    if (unit >= vt.total_tiles * 8) return;
    const int tile = unit >> 3;
    const Unit t = unit_ctx(vt, tile, unit & 7);
    const int2 rg = ranges[tile];
    const int n = rg.y - rg.x;
    const float fx = t.px + 0.5f, fy = t.py + 0.5f;

    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, Dd = 0.0f;
    int lastc = 0;
    bool done = !t.inside;

    Rec cur, nxt;
    int id2 = (32 + lane < n) ? ids[rg.x + 32 + lane] : 0;
    load_rec(cur, xy, co, rgbd, lane < n ? ids[rg.x + lane] : 0, lane < n);
    for (int base = 0; base < n && !__all_sync(0xffffffffu, done); base += 32) {
        // prefetch: records of the next step, ids of the one after
        const bool v1 = base + 32 + lane < n;
        load_rec(nxt, xy, co, rgbd, id2, v1);
        id2 = (base + 64 + lane < n) ? ids[rg.x + base + 64 + lane] : 0;

        uint32_t m = __ballot_sync(0xffffffffu, reaches_block(cur.p, cur.q, cfg.alpha_min, t.bx0, t.by0));
        if (m) {
            s_p[warp][lane] = cur.p;
            s_q[warp][lane] = cur.q;
            s_c[warp][lane] = cur.c;
            __syncwarp();
            while (m) {
                const int k = __ffs(m) - 1;
                m &= m - 1;
                if (done) continue;
                const float2 p = s_p[warp][k];
                const float4 q = s_q[warp][k];
                const float power = gauss_power(q.x, q.y, q.z, fx - p.x, fy - p.y);
                if (power > 0.0f) continue;
                const float alpha = fminf(cfg.alpha_max, q.w * __expf(power));
                if (alpha < cfg.alpha_min) continue;
                const float Tn = T * (1.0f - alpha);
                if (Tn < cfg.t_min) { done = true; continue; }
                const float4 c = s_c[warp][k];
                const float w = alpha * T;
                C0 += c.x * w; C1 += c.y * w; C2 += c.z * w; Dd += c.w * w;
                T = Tn;
                lastc = base + k + 1;
            }
            __syncwarp();
        }
        cur = nxt;
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

constexpr int kAccGrad = 10;   // u v a b c o r g b z
constexpr int kDirectLanes = 4;  // up to this many active lanes: each issues its own reductions

template <bool STATS>
__global__ void __launch_bounds__(32 * kWarps) k_render_bwd(ViewTable vt, RasterCfg cfg,
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
    __shared__ float2 s_p[kWarps][32];
    __shared__ float4 s_q[kWarps][32];
    __shared__ float4 s_c[kWarps][32];
    __shared__ int s_id[kWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int unit = blockIdx.x * kWarps + warp;
    if (unit >= vt.total_tiles * 8) return;
    const int tile = unit >> 3;
    const Unit t = unit_ctx(vt, tile, unit & 7);
    const int2 rg = ranges[tile];
    const float fx = t.px + 0.5f, fy = t.py + 0.5f;
    const bool has_depth = dL_ddepth != nullptr;

    float T = 1.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f, gD = 0.0f, mask = 0.0f;
    int lst = 0;
    if (t.inside) {
        T = T_final[t.pix];
        lst = last[t.pix];
        g0 = dL_dimg[t.img];
        g1 = dL_dimg[t.img + t.plane];
        g2 = dL_dimg[t.img + 2 * t.plane];
        if (has_depth) gD = dL_ddepth[t.pix];
        if (STATS) {
            const float e = fabsf(target[t.img] - img[t.img]) + fabsf(target[t.img + t.plane] - img[t.img + t.plane]) +
                            fabsf(target[t.img + 2 * t.plane] - img[t.img + 2 * t.plane]);
            mask = e > tau_err ? 1.0f : 0.0f;
        }
    }
    int wmax = lst;
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    if (wmax == 0) return;

    // colour (and depth) behind the current Gaussian, normalised by the
    // transmittance in front of it; starts as the background
    float R0 = cfg.bg[0], R1 = cfg.bg[1], R2 = cfg.bg[2], RD = 0.0f;

    // steps of 32 pairs from the one holding position wmax-1 down to 0
    int base = ((wmax - 1) >> 5) << 5;
    Rec cur, nxt;
    {
        const int j0 = base + lane;
        load_rec(cur, xy, co, rgbd, j0 < wmax ? ids[rg.x + j0] : 0, j0 < wmax);
    }
    int id2 = (base >= 32) ? ids[rg.x + base - 32 + lane] : 0;
    for (; base >= 0; base -= 32) {
        load_rec(nxt, xy, co, rgbd, id2, base >= 32);
        id2 = (base >= 64) ? ids[rg.x + base - 64 + lane] : 0;

        uint32_t m = __ballot_sync(0xffffffffu, base + lane < wmax &&
                                                    reaches_block(cur.p, cur.q, cfg.alpha_min, t.bx0, t.by0));
        if (m) {
            s_p[warp][lane] = cur.p;
            s_q[warp][lane] = cur.q;
            s_c[warp][lane] = cur.c;
            s_id[warp][lane] = cur.id;
            __syncwarp();
            while (m) {
                const int k = 31 - __clz(m);
                m &= ~(1u << k);
                bool on = base + k < lst;
                float alpha = 0.0f, G = 0.0f, dx = 0.0f, dy = 0.0f;
                const float2 p = s_p[warp][k];
                const float4 q = s_q[warp][k];
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
                const uint32_t act = __ballot_sync(0xffffffffu, on);
                if (act == 0u) continue;
                float v[kAccPlanes];
                #pragma unroll
                for (int c = 0; c < kAccPlanes; ++c) v[c] = 0.0f;
                if (on) {
                    const float4 c = s_c[warp][k];
                    T = __fdividef(T, 1.0f - alpha);  // transmittance in front of this Gaussian
                    const float w = alpha * T;
                    v[kAccR] = g0 * w; v[kAccG] = g1 * w; v[kAccBl] = g2 * w; v[kAccZ] = gD * w;
                    const float dLda = T * (g0 * (c.x - R0) + g1 * (c.y - R1) + g2 * (c.z - R2) + gD * (c.w - RD));
                    R0 = alpha * c.x + (1.0f - alpha) * R0;
                    R1 = alpha * c.y + (1.0f - alpha) * R1;
                    R2 = alpha * c.z + (1.0f - alpha) * R2;
                    RD = alpha * c.w + (1.0f - alpha) * RD;
                    if (q.w * G <= cfg.alpha_max) {  // alpha not clamped
                        v[kAccO] = dLda * G;
                        const float dp = dLda * q.w * G;
                        v[kAccU] = dp * (q.x * dx + q.y * dy);
                        v[kAccV] = dp * (q.z * dy + q.y * dx);
                        v[kAccA] = -0.5f * dp * dx * dx;
                        v[kAccB] = -dp * dx * dy;
                        v[kAccC] = -0.5f * dp * dy * dy;
                    }
                    if (STATS) { v[kAccOmega] = 1.0f; v[kAccKappa] = mask; v[kAccMaxW] = w; }
                }
                const long long r = s_id[warp][k];
                bool issue = on;
                if (__popc(act) > kDirectLanes) {
                    #pragma unroll
                    for (int c = 0; c < kAccGrad; ++c)
                        if (c != kAccZ || has_depth) v[c] = warp_sum(v[c]);
                    if (STATS) {
                        v[kAccOmega] = warp_sum(v[kAccOmega]);
                        v[kAccKappa] = warp_sum(v[kAccKappa]);
                        v[kAccMaxW] = warp_max(v[kAccMaxW]);
                    }
                    issue = lane == 0;
                }
                if (issue) {
                    #pragma unroll
                    for (int c = 0; c < kAccGrad; ++c)
                        if (c != kAccZ || has_depth) atomicAdd(&acc[c * nrec + r], v[c]);
                    if (STATS) {
                        atomicAdd(&acc[kAccOmega * nrec + r], v[kAccOmega]);
                        if (v[kAccKappa] > 0.0f) atomicAdd(&acc[kAccKappa * nrec + r], v[kAccKappa]);
                        atomicMax((int *)&acc[kAccMaxW * nrec + r], __float_as_int(v[kAccMaxW]));  // w >= 0
                    }
                }
            }
            __syncwarp();
        }
        cur = nxt;
    }
}

void launch_render_fwd(const ViewTable &vt, const RasterCfg &cfg, const int2 *ranges, const int *ids, const float2 *xy,
                       const float4 *co, const float4 *rgbd, float *img, float *T_final, int *last, float *depth,
                       cudaStream_t s) {
    const long long units = 8ll * vt.total_tiles;
    if (units <= 0) return;
    k_render_fwd<<<(unsigned)ceil_div(units, kWarps), 32 * kWarps, 0, s>>>(vt, cfg, ranges, ids, xy, co, rgbd, img,
                                                                           T_final, last, depth);
}

void launch_render_bwd(const ViewTable &vt, const RasterCfg &cfg, const int2 *ranges, const int *ids,
                       const float2 *xy, const float4 *co, const float4 *rgbd, const float *img, const float *T_final,
                       const int *last, const float *dL_dimg, const float *dL_ddepth, const float *target,
                       float tau_err, bool stats, float *acc, long long nrec, cudaStream_t s) {
    const long long units = 8ll * vt.total_tiles;
    if (units <= 0) return;
    const unsigned grid = (unsigned)ceil_div(units, kWarps);
    if (stats)
        k_render_bwd<true><<<grid, 32 * kWarps, 0, s>>>(vt, cfg, ranges, ids, xy, co, rgbd, img, T_final, last,
                                                        dL_dimg, dL_ddepth, target, tau_err, acc, nrec);
    else
        k_render_bwd<false><<<grid, 32 * kWarps, 0, s>>>(vt, cfg, ranges, ids, xy, co, rgbd, img, T_final, last,
                                                         dL_dimg, dL_ddepth, target, tau_err, acc, nrec);
}

}  // namespace gs
