// render.cu -- compositing kernels: front-to-back forward and back-to-front
// backward (Supp. D.2: C = sum_j c_j alpha_j T_j, T_j = prod_{m<j}(1 - alpha_m)).
//
// Work unit = one warp = one 8x4 pixel block of a tile (a tile of 256 pixels,
// 16x16, 8x32 or 32x8, has eight blocks); lane = pixel.  The binning stored,
// for every (Gaussian, tile) pair, the mask of the tile's blocks that the
// Gaussian's alpha >= alpha_min ellipse can reach (conservative, so skipping a
// clear bit is exact).  Each warp scans its tile's masks 512 pairs per step
// with coalesced 16-byte loads, compacts the pairs relevant to its block into
// warp-private shared memory, and composites them with the records of the
// next 32 already in flight.  There is no CTA-wide barrier: a block whose
// pixels saturate early retires at once, and the long chains of a
// vanishing-point tile touch only the pairs that reach each block.
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

struct Rec {
    float2 p;
    float4 q, c;
    int id, pos;
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
        r.q = make_float4(0.f, 0.f, 0.f, 0.f);
        r.c = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}


// Scans the block masks of pairs [w, w + WIN) restricted to [lo, hi) and
// writes, in pair order, the absolute positions whose mask holds `bit` into
// list.  Returns the count (warp-uniform).  Each lane reads WIN/32 masks in
// one aligned load (w is a multiple of 16).
template <int WIN>
__device__ __forceinline__ int scan_window(const uint8_t *__restrict__ masks, int w, int lo, int hi, int bit,
                                           int *list) {
    constexpr int PER = WIN / 32;  // 4, 8 or 16 masks per lane
    const int lane = threadIdx.x & 31;
    const int q0 = w + PER * lane;
    uint32_t wd[4] = {0u, 0u, 0u, 0u};
    if (q0 < hi) {
        if (PER == 16) {
            const uint4 m4 = *reinterpret_cast<const uint4 *>(masks + q0);
            wd[0] = m4.x; wd[1] = m4.y; wd[2] = m4.z; wd[3] = m4.w;
        } else if (PER == 8) {
            const uint2 m2 = *reinterpret_cast<const uint2 *>(masks + q0);
            wd[0] = m2.x; wd[1] = m2.y;
        } else {
            wd[0] = *reinterpret_cast<const uint32_t *>(masks + q0);
        }
    }
    uint32_t rel = 0;
    #pragma unroll
    for (int b = 0; b < PER; ++b) {
        const int pos = q0 + b;
        const uint32_t byte = (wd[b >> 2] >> (8 * (b & 3))) & 0xffu;
        if (pos >= lo && pos < hi && ((byte >> bit) & 1u)) rel |= 1u << b;
    }
    const int cnt = __popc(rel);
    int inc = cnt;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    int off = inc - cnt;
    while (rel) {
        const int b = __ffs(rel) - 1;
        rel &= rel - 1;
        list[off++] = q0 + b;
    }
    const int total = __shfl_sync(0xffffffffu, inc, 31);
    __syncwarp();
    return total;
}

__device__ __forceinline__ void gather(Rec &r, const int *list, int idx, int total, const int *__restrict__ ids,
                                       const float2 *__restrict__ xy, const float4 *__restrict__ co,
                                       const float4 *__restrict__ rgbd) {
    const bool valid = idx < total;
    r.pos = valid ? list[idx] : 0;
    load_rec(r, xy, co, rgbd, valid ? ids[r.pos] : 0, valid);
}

template <int WIN>
__global__ void __launch_bounds__(32 * kWarps) k_render_fwd(ViewTable vt, RasterCfg cfg,
                                                              const int2 *__restrict__ ranges,
                                                              const int *__restrict__ ids,
                                                              const uint8_t *__restrict__ masks,
                                                              const int *__restrict__ order,
                                                              const float2 *__restrict__ xy,
                                                              const float4 *__restrict__ co,
                                                              const float4 *__restrict__ rgbd,
                                                              float *__restrict__ img, float *__restrict__ T_final,
                                                              int *__restrict__ last, float *__restrict__ depth) {
    __shared__ int s_list[kWarps][WIN];
    __shared__ float2 s_p[kWarps][32];
    __shared__ float4 s_q[kWarps][32];
    __shared__ float4 s_c[kWarps][32];
    __shared__ int s_pos[kWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int unit = blockIdx.x * kWarps + warp;
    if (unit >= vt.total_tiles * 8) return;
    const int tile = order[unit >> 3], bit = unit & 7;  // longest tiles first
    const Unit t = unit_ctx(vt, tile, bit);
    const int2 rg = ranges[tile];
    const float fx = t.px + 0.5f, fy = t.py + 0.5f;
    int *list = s_list[warp];

    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, Dd = 0.0f;
    int lastc = 0;
    bool done = !t.inside;
    for (int w = rg.x & ~15; w < rg.y && !__all_sync(0xffffffffu, done); w += WIN) {
        const int total = scan_window<WIN>(masks, w, rg.x, rg.y, bit, list);
        Rec cur, nxt;
        gather(cur, list, lane, total, ids, xy, co, rgbd);
        for (int c = 0; c < total; c += 32) {
            if (c + 32 < total) gather(nxt, list, c + 32 + lane, total, ids, xy, co, rgbd);
            s_p[warp][lane] = cur.p;
            s_q[warp][lane] = cur.q;
            s_c[warp][lane] = cur.c;
            s_pos[warp][lane] = cur.pos;
            __syncwarp();
            const int cnt = min(32, total - c);
            for (int k = 0; k < cnt && !done; ++k) {
                const float2 p = s_p[warp][k];
                const float4 q = s_q[warp][k];
                const float power = gauss_power(q.x, q.y, q.z, fx - p.x, fy - p.y);
                if (power > 0.0f) continue;
                const float alpha = fminf(cfg.alpha_max, q.w * __expf(power));
                if (alpha < cfg.alpha_min) continue;
                const float Tn = T * (1.0f - alpha);
                if (Tn < cfg.t_min) { done = true; break; }
                const float4 cc = s_c[warp][k];
                const float wgt = alpha * T;
                C0 += cc.x * wgt; C1 += cc.y * wgt; C2 += cc.z * wgt; Dd += cc.w * wgt;
                T = Tn;
                lastc = s_pos[warp][k] - rg.x + 1;
            }
            __syncwarp();
            if (__all_sync(0xffffffffu, done)) break;
            cur = nxt;
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

constexpr int kAccGrad = 10;   // u v a b c o r g b z
constexpr int kDirectLanes = 8;  // up to this many active lanes: each issues its own reductions

// Sums 16 values over the warp by recursive halving: at each of the four
// steps a lane swaps half of its partial sums with its partner and keeps the
// other half, so 8+4+2+1+1 = 16 shuffles replace 16 x 5.  Lane l ends with
// the total of value (l >> 1) & 15 (in both lanes of a pair).
__device__ __forceinline__ float warp_transpose_sum16(float (&v)[16]) {
    const int lane = threadIdx.x & 31;
    #pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool hi = lane & 16;
        const float send = hi ? v[i] : v[i + 8], keep = hi ? v[i + 8] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    #pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool hi = lane & 8;
        const float send = hi ? v[i] : v[i + 4], keep = hi ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    #pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool hi = lane & 4;
        const float send = hi ? v[i] : v[i + 2], keep = hi ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool hi = lane & 2;
        const float send = hi ? v[0] : v[1], keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

template <bool STATS, int WIN>
__global__ void __launch_bounds__(32 * kWarps) k_render_bwd(ViewTable vt, RasterCfg cfg,
                                                              const int2 *__restrict__ ranges,
                                                              const int *__restrict__ ids,
                                                              const uint8_t *__restrict__ masks,
                                                              const int *__restrict__ order,
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
    __shared__ int s_list[kWarps][WIN];
    __shared__ float2 s_p[kWarps][32];
    __shared__ float4 s_q[kWarps][32];
    __shared__ float4 s_c[kWarps][32];
    __shared__ int s_id[kWarps][32];
    __shared__ int s_pos[kWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int unit = blockIdx.x * kWarps + warp;
    if (unit >= vt.total_tiles * 8) return;
    const int tile = order[unit >> 3], bit = unit & 7;  // longest tiles first
    const Unit t = unit_ctx(vt, tile, bit);
    const int2 rg = ranges[tile];
    const float fx = t.px + 0.5f, fy = t.py + 0.5f;
    const bool has_depth = dL_ddepth != nullptr;
    int *list = s_list[warp];

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

    const int lo = rg.x, hi = rg.x + wmax;
    const int wbase = rg.x & ~15;
    for (int kw = (hi - 1 - wbase) / WIN; kw >= 0; --kw) {
        const int total = scan_window<WIN>(masks, wbase + kw * WIN, lo, hi, bit, list);
        if (total == 0) continue;
        int c = ((total - 1) >> 5) << 5;
        Rec cur, nxt;
        gather(cur, list, c + lane, total, ids, xy, co, rgbd);
        for (; c >= 0; c -= 32) {
            if (c >= 32) gather(nxt, list, c - 32 + lane, total, ids, xy, co, rgbd);
            s_p[warp][lane] = cur.p;
            s_q[warp][lane] = cur.q;
            s_c[warp][lane] = cur.c;
            s_id[warp][lane] = cur.id;
            s_pos[warp][lane] = cur.pos;
            __syncwarp();
            const int cnt = min(32, total - c);
            for (int k = cnt - 1; k >= 0; --k) {
                bool on = s_pos[warp][k] - rg.x < lst;
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
                float v[16];
                #pragma unroll
                for (int cc = 0; cc < 16; ++cc) v[cc] = 0.0f;
                if (on) {
                    const float4 col = s_c[warp][k];
                    T = __fdividef(T, 1.0f - alpha);  // transmittance in front of this Gaussian
                    const float w = alpha * T;
                    v[kAccR] = g0 * w; v[kAccG] = g1 * w; v[kAccBl] = g2 * w; v[kAccZ] = gD * w;
                    const float dLda = T * (g0 * (col.x - R0) + g1 * (col.y - R1) + g2 * (col.z - R2) +
                                            gD * (col.w - RD));
                    R0 = alpha * col.x + (1.0f - alpha) * R0;
                    R1 = alpha * col.y + (1.0f - alpha) * R1;
                    R2 = alpha * col.z + (1.0f - alpha) * R2;
                    RD = alpha * col.w + (1.0f - alpha) * RD;
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
                if (__popc(act) <= kDirectLanes) {
                    // a single pixel: its lane issues the updates itself
                    if (on) {
                        #pragma unroll
                        for (int cc = 0; cc < kAccGrad; ++cc)
                            if (cc != kAccZ || has_depth) atomicAdd(&acc[cc * nrec + r], v[cc]);
                        if (STATS) {
                            atomicAdd(&acc[kAccOmega * nrec + r], v[kAccOmega]);
                            if (v[kAccKappa] > 0.0f) atomicAdd(&acc[kAccKappa * nrec + r], v[kAccKappa]);
                            atomicMax((int *)&acc[kAccMaxW * nrec + r], __float_as_int(v[kAccMaxW]));  // w >= 0
                        }
                    }
                } else {
                    const float mw = STATS ? warp_max(v[kAccMaxW]) : 0.0f;
                    const float tot = warp_transpose_sum16(v);
                    const int plane = (lane >> 1) & 15;
                    const bool mine = (lane & 1) == 0 && plane < (STATS ? kAccMaxW : kAccGrad) &&
                                      (plane != kAccZ || has_depth) && (plane != kAccKappa || tot > 0.0f);
                    if (mine) atomicAdd(&acc[plane * nrec + r], tot);
                    if (STATS && lane == 1) atomicMax((int *)&acc[kAccMaxW * nrec + r], __float_as_int(mw));
                }
            }
            __syncwarp();
            cur = nxt;
        }
    }
}

void launch_render_fwd(const ViewTable &vt, const RasterCfg &cfg, const int2 *ranges, const int *ids,
                       const uint8_t *masks, const int *order, const float2 *xy, const float4 *co,
                       const float4 *rgbd, float *img, float *T_final, int *last, float *depth, cudaStream_t s) {
    const long long units = 8ll * vt.total_tiles;
    if (units <= 0) return;
    const unsigned grid = (unsigned)ceil_div(units, kWarps);
#define GS_FWD(WN) k_render_fwd<WN><<<grid, 32 * kWarps, 0, s>>>(vt, cfg, ranges, ids, masks, order, xy, co, rgbd, img, \
                                                                 T_final, last, depth)
    if (cfg.batch == 128) GS_FWD(128);
    else if (cfg.batch == 256) GS_FWD(256);
    else GS_FWD(512);
#undef GS_FWD
}

void launch_render_bwd(const ViewTable &vt, const RasterCfg &cfg, const int2 *ranges, const int *ids,
                       const uint8_t *masks, const int *order, const float2 *xy, const float4 *co,
                       const float4 *rgbd, const float *img, const float *T_final, const int *last, const float *dL_dimg,
                       const float *dL_ddepth, const float *target, float tau_err, bool stats, float *acc,
                       long long nrec, cudaStream_t s) {
    const long long units = 8ll * vt.total_tiles;
    if (units <= 0) return;
    const unsigned grid = (unsigned)ceil_div(units, kWarps);
#define GS_BWD(ST, WN) k_render_bwd<ST, WN><<<grid, 32 * kWarps, 0, s>>>(vt, cfg, ranges, ids, masks, order, xy, co, \
                                                                         rgbd, img, T_final, last, dL_dimg, \
                                                                         dL_ddepth, target, tau_err, acc, nrec)
    if (stats) {
        if (cfg.batch == 128) GS_BWD(true, 128);
        else if (cfg.batch == 256) GS_BWD(true, 256);
        else GS_BWD(true, 512);
    } else {
        if (cfg.batch == 128) GS_BWD(false, 128);
        else if (cfg.batch == 256) GS_BWD(false, 256);
        else GS_BWD(false, 512);
    }
#undef GS_BWD
}

}  // namespace gs
