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
#include <algorithm>

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

// Compositing state of one lane's pixel.
struct FwdState {
    float T, C0, C1, C2, D;
    int last;   // pairs of the tile consumed up to and including the last blended one
    bool done;  // stopped (or outside the view)
};

struct FwdShared {
    float2 *p;
    float4 *q, *c;
    int *pos, *list;
    int *id;  // record ids of the staged pairs (only for a blend hook that needs them)
};

// What the forward does besides compositing when a pixel blends a Gaussian
// (k: the pair's slot among the 32 staged, a: its alpha): nothing, normally.
struct NoBlendHook {
    static constexpr bool kNeedsId = false;
    __device__ __forceinline__ void operator()(const FwdShared &, int, float) {}
};

// Front-to-back compositing of the pairs of [lo, hi) (positions in the tile's
// list, rgx its start) relevant to block `bit` into each lane's state, with
// the stop rule of Supp. D.2 (stop before the pair that takes T below t_min).
// alpha of 8 staged pairs at a time (independent, so their latencies overlap),
// then the short serial transmittance update over them.
template <int WIN, class Hook = NoBlendHook>
__device__ __forceinline__ void fwd_range(const RasterCfg &cfg, const uint8_t *__restrict__ masks,
                                          const int *__restrict__ ids, const float2 *__restrict__ xy,
                                          const float4 *__restrict__ co, const float4 *__restrict__ rgbd, int rgx,
                                          int lo, int hi, int bit, float fx, float fy, FwdState &st,
                                          const FwdShared &sh, Hook hook = Hook()) {
    const int lane = threadIdx.x & 31;
    for (int w = lo & ~15; w < hi && !__all_sync(0xffffffffu, st.done); w += WIN) {
        const int total = scan_window<WIN>(masks, w, lo, hi, bit, sh.list);
        Rec cur, nxt;
        gather(cur, sh.list, lane, total, ids, xy, co, rgbd);
        for (int c = 0; c < total; c += 32) {
            if (c + 32 < total) gather(nxt, sh.list, c + 32 + lane, total, ids, xy, co, rgbd);
            sh.p[lane] = cur.p;
            sh.q[lane] = cur.q;
            sh.c[lane] = cur.c;
            sh.pos[lane] = cur.pos;
            if (Hook::kNeedsId) sh.id[lane] = cur.id;
            __syncwarp();
            const int cnt = min(32, total - c);
            for (int k0 = 0; k0 < cnt && !st.done; k0 += 8) {
                float al[8];
                #pragma unroll
                for (int j = 0; j < 8; ++j) {
                    // every lane evaluates every staged Gaussian (slots past cnt hold stale,
                    // in-bounds entries and are masked)
                    const float2 p = sh.p[k0 + j];
                    const float4 q = sh.q[k0 + j];
                    const float power = gauss_power(q.x, q.y, q.z, fx - p.x, fy - p.y);
                    const float a = fminf(cfg.alpha_max, q.w * __expf(power));
                    al[j] = k0 + j < cnt && power <= 0.0f && !(a < cfg.alpha_min) ? a : -1.0f;
                }
                #pragma unroll
                for (int j = 0; j < 8; ++j) {
                    // no divergent branch: a lane that does not take this Gaussian adds
                    // zero-weighted colour and keeps its state
                    const float a = al[j];
                    const bool blend = !st.done && a >= 0.0f;
                    const float Tn = st.T * (1.0f - a);
                    const bool stop = blend && Tn < cfg.t_min;
                    const bool take = blend && !stop;
                    const float4 cc = sh.c[k0 + j];
                    const float wgt = (take ? a : 0.0f) * st.T;
                    st.C0 += cc.x * wgt; st.C1 += cc.y * wgt; st.C2 += cc.z * wgt; st.D += cc.w * wgt;
                    st.T = take ? Tn : st.T;
                    st.last = take ? sh.pos[k0 + j] - rgx + 1 : st.last;
                    st.done = st.done || stop;
                    if (take) hook(sh, k0 + j, a);
                }
            }
            __syncwarp();
            if (__all_sync(0xffffffffu, st.done)) break;
            cur = nxt;
        }
    }
}

__device__ __forceinline__ void fwd_write(const RasterCfg &cfg, const Unit &t, const FwdState &st,
                                          float *__restrict__ img, float *__restrict__ T_final,
                                          int *__restrict__ last, float *__restrict__ depth) {
    if (!t.inside) return;
    img[t.img] = st.C0 + st.T * cfg.bg[0];
    img[t.img + t.plane] = st.C1 + st.T * cfg.bg[1];
    img[t.img + 2 * t.plane] = st.C2 + st.T * cfg.bg[2];
    T_final[t.pix] = st.T;
    last[t.pix] = st.last;
    if (depth) depth[t.pix] = st.D;
}

// Split forward, step 1 (one CTA): the tiles whose list is longer than one
// segment ("long" tiles), in schedule order, each with the base of its
// 8 x S segment items (S segments per 8x4 block) -- a block scan over the
// schedule, so bases increase with the table index.
constexpr int kPlanThreads = 1024;
__global__ void __launch_bounds__(kPlanThreads) k_fwd_plan(const int2 *__restrict__ ranges,
                                                          const int *__restrict__ order, int total_tiles,
                                                          int seg_shift, SegWs seg) {
    griddep_wait();
    __shared__ int s_items[kPlanThreads / 32], s_long[kPlanThreads / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = (total_tiles + kPlanThreads - 1) / kPlanThreads;
    const int lo = min(total_tiles, t * per), hi = min(total_tiles, lo + per);
    int items = 0, nlong = 0;
    for (int i = lo; i < hi; ++i) {
        const int2 rg = ranges[order[i]];
        const int S = (rg.y - rg.x + (1 << seg_shift) - 1) >> seg_shift;
        if (S > 1) { items += 8 * S; ++nlong; }
    }
    int ii = items, il = nlong;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, ii, o), b = __shfl_up_sync(0xffffffffu, il, o);
        if (lane >= o) { ii += a; il += b; }
    }
    if (lane == 31) { s_items[warp] = ii; s_long[warp] = il; }
    __syncthreads();
    if (warp == 0) {
        int a = s_items[lane], b = s_long[lane], ai = a, bi = b;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, ai, o), y = __shfl_up_sync(0xffffffffu, bi, o);
            if (lane >= o) { ai += x; bi += y; }
        }
        s_items[lane] = ai - a;
        s_long[lane] = bi - b;
    }
    __syncthreads();
    int base = s_items[warp] + ii - items, h = s_long[warp] + il - nlong;
    for (int i = lo; i < hi; ++i) {
        const int tile = order[i];
        const int2 rg = ranges[tile];
        const int S = (rg.y - rg.x + (1 << seg_shift) - 1) >> seg_shift;
        if (S > 1) {
            if (h < seg.hcap) seg.heavy[h] = make_int4(i, tile, base, S);
            base += 8 * S;
            ++h;
        }
    }
    if (t == kPlanThreads - 1) {
        // items, long tiles and checkpoints (8 (S - 1) per long tile) against the capacities
        const bool fits = base <= seg.fcap && h <= seg.hcap && base - 8 * h <= seg.cap;
        seg.count[0] = fits ? base : 0;  // segment items
        seg.count[1] = fits ? h : 0;     // long tiles
        seg.count[4] = fits ? 0 : 1;     // no split: every block walks its whole list
        seg.count[5] = base;             // items needed
    }
}

// Item `it` of the split forward: its long tile (the last plan entry whose
// first item is <= it), 8x4 block and segment.
struct ItemRef {
    int4 H;  // (schedule index, tile, first item, segments S)
    int blk, sgi;
};
__device__ __forceinline__ ItemRef item_ref(const SegWs &seg, int it) {
    int a = 0, b = min(seg.count[1], seg.hcap) - 1;
    while (a < b) {
        const int m = (a + b + 1) >> 1;
        if (seg.heavy[m].z <= it) a = m; else b = m - 1;
    }
    ItemRef r;
    r.H = seg.heavy[a];
    const int rel = it - r.H.z;
    r.blk = rel / r.H.w;
    r.sgi = rel - r.blk * r.H.w;
    return r;
}

__device__ __forceinline__ void fres_store(float *r, const FwdState &st, bool flag) {
    const int lane = threadIdx.x & 31;
    r[lane] = st.T; r[32 + lane] = st.C0; r[64 + lane] = st.C1; r[96 + lane] = st.C2; r[128 + lane] = st.D;
    r[160 + lane] = __int_as_float(st.last | (flag ? (int)0x80000000u : 0));
}

// Split forward, step 2: CTAs [0, item_blocks) loop over the segment items,
// compositing one segment of a long tile's block each from T = 1 (a local
// pass with the same stop rule; flag = stopped) into its slot of fres; the
// other CTAs composite the short tiles' blocks whole.
template <int WIN>
__global__ void __launch_bounds__(32 * kWarps, 8) k_render_fwd(ViewTable vt, RasterCfg cfg,
                                                              const int2 *__restrict__ ranges,
                                                              const int *__restrict__ ids,
                                                              const uint8_t *__restrict__ masks,
                                                              const int *__restrict__ order,
                                                              const float2 *__restrict__ xy,
                                                              const float4 *__restrict__ co,
                                                              const float4 *__restrict__ rgbd,
                                                              float *__restrict__ img, float *__restrict__ T_final,
                                                              int *__restrict__ last, float *__restrict__ depth,
                                                              SegWs seg, int item_blocks) {
    griddep_wait();
    __shared__ int s_list[kWarps][WIN];
    __shared__ float2 s_p[kWarps][32];
    __shared__ float4 s_q[kWarps][32];
    __shared__ float4 s_c[kWarps][32];
    __shared__ int s_pos[kWarps][32];
    const int warp = threadIdx.x >> 5;
    const FwdShared sh{s_p[warp], s_q[warp], s_c[warp], s_pos[warp], s_list[warp], nullptr};
    if ((int)blockIdx.x < item_blocks) {
        const int n = min(seg.count[0], seg.fcap);
        for (int it = blockIdx.x * kWarps + warp; it < n; it += item_blocks * kWarps) {
            const ItemRef R = item_ref(seg, it);
            const Unit t = unit_ctx(vt, R.H.y, R.blk);
            const int2 rg = ranges[R.H.y];
            const int lo = rg.x + (R.sgi << cfg.seg_shift), hi = min(rg.y, lo + (1 << cfg.seg_shift));
            FwdState st{1.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0, !t.inside};
            fwd_range<WIN>(cfg, masks, ids, xy, co, rgbd, rg.x, lo, hi, R.blk, t.px + 0.5f, t.py + 0.5f, st, sh);
            fres_store(seg.fres + (long long)it * kFresFloats, st, st.done && t.inside);
        }
        return;
    }
    const int unit = (blockIdx.x - item_blocks) * kWarps + warp;
    if (unit >= vt.total_tiles * 8) return;
    const int tile = order[unit >> 3], bit = unit & 7;  // longest tiles first
    const int2 rg = ranges[tile];
    if (cfg.seg_shift >= 0 && rg.y - rg.x > (1 << cfg.seg_shift) && !seg.count[4]) return;  // long: segment items
    const Unit t = unit_ctx(vt, tile, bit);
    FwdState st{1.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0, !t.inside};
    fwd_range<WIN>(cfg, masks, ids, xy, co, rgbd, rg.x, rg.x, rg.y, bit, t.px + 0.5f, t.py + 0.5f, st, sh);
    fwd_write(cfg, t, st, img, T_final, last, depth);
}

// Split forward, step 3: one warp per block of a long tile chains the local
// passes of its segments in order, T_start(s+1) = T_start(s) T_s and
// C += T_start(s) C_s, recording the state after each segment (the backward's
// checkpoints), until every pixel has either run through all segments or
// reached the segment where its stop falls (the local pass stopped, or the
// chained T after it would be below t_min).  Pixels of the first kind are
// final and written; for each segment where some pixels stop, a re-run task
// (item, lane mask, first checkpoint slot) is registered and the pixels'
// state entering the segment replaces their columns of that item's slot.
constexpr int kSplitCtasPerSm = 8;
__global__ void __launch_bounds__(32 * kWarps) k_render_fwd_combine(ViewTable vt, RasterCfg cfg,
                                                                   float *__restrict__ img,
                                                                   float *__restrict__ T_final,
                                                                   int *__restrict__ last,
                                                                   float *__restrict__ depth, SegWs seg) {
    griddep_wait();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = 8 * min(seg.count[1], seg.hcap);
    for (int u = blockIdx.x * kWarps + warp; u < n; u += gridDim.x * kWarps) {
        const int h = u >> 3, blk = u & 7;
        const int4 H = seg.heavy[h];
        const int S = H.w, unit = 8 * H.x + blk, item0 = H.z + blk * S;
        if ((long long)H.z + 8ll * S > seg.fcap) continue;  // cannot happen: the capacity bounds every plan
        const Unit t = unit_ctx(vt, H.y, blk);
        int slot0 = 0;
        if (lane == 0) slot0 = atomicAdd(&seg.count[2], S - 1);
        slot0 = __shfl_sync(0xffffffffu, slot0, 0);
        FwdState st{1.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0, !t.inside};
        bool pend = false;
        int sstar = 0x7fffffff;
        int sgi_end = S - 1;  // last segment whose boundary state was recorded
        constexpr int B = 8;  // segments whose local states are loaded together
        bool stop_chain = false;
        for (int s0 = 0; s0 < S && !stop_chain; s0 += B) {
            float lT[B], lC0[B], lC1[B], lC2[B], lD[B];
            int lw[B];
            #pragma unroll
            for (int j = 0; j < B; ++j) {
                const float *r = seg.fres + (long long)(item0 + min(s0 + j, S - 1)) * kFresFloats;
                lT[j] = r[lane]; lC0[j] = r[32 + lane]; lC1[j] = r[64 + lane]; lC2[j] = r[96 + lane];
                lD[j] = r[128 + lane]; lw[j] = __float_as_int(r[160 + lane]);
            }
            #pragma unroll
            for (int j = 0; j < B; ++j) {
                const int sgi = s0 + j;
                if (sgi >= S || stop_chain) break;
                if (!st.done && !pend) {
                    if (lw[j] < 0 || st.T * lT[j] < cfg.t_min) {
                        pend = true;  // the stop falls inside this segment
                        sstar = sgi;
                    } else {
                        st.C0 += st.T * lC0[j];
                        st.C1 += st.T * lC1[j];
                        st.C2 += st.T * lC2[j];
                        st.D += st.T * lD[j];
                        if (lw[j] > 0) st.last = lw[j];
                        st.T *= lT[j];
                    }
                }
                const int slot = slot0 + sgi;
                if (sgi < S - 1 && slot < seg.cap) {  // state at boundary sgi + 1
                    float *ck = seg.ckpt + (long long)slot * kCkptFloats;
                    ck[lane] = st.T; ck[32 + lane] = st.C0; ck[64 + lane] = st.C1; ck[96 + lane] = st.C2;
                    ck[128 + lane] = st.D;
                    if (lane == 0) seg.items[slot] = make_int2(unit, sgi + 1);
                }
                if (__all_sync(0xffffffffu, st.done || pend)) {
                    stop_chain = true;
                    sgi_end = sgi;
                }
            }
        }
        // reserved slots past the chain hold no checkpoint (a re-run may claim them)
        if (lane == 0)
            for (int k = sgi_end + 1; k < S - 1; ++k)
                if (slot0 + k < seg.cap) seg.items[slot0 + k] = make_int2(-1, 0);
        if (!pend) fwd_write(cfg, t, st, img, T_final, last, depth);
        // one re-run task per segment where some pixels stop
        bool assigned = !pend;
        while (__any_sync(0xffffffffu, !assigned)) {
            int smin = assigned ? 0x7fffffff : sstar;
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) smin = min(smin, __shfl_xor_sync(0xffffffffu, smin, o));
            const bool mine = !assigned && sstar == smin;
            const unsigned mask = __ballot_sync(0xffffffffu, mine);
            if (mine) fres_store(seg.fres + (long long)(item0 + smin) * kFresFloats, st, false);
            if (lane == 0) {
                const int task = atomicAdd(&seg.count[3], 1);
                if (task < seg.fcap) seg.tasks[task] = make_int4(item0 + smin, (int)mask, slot0, 0);
            }
            assigned = assigned || mine;
        }
    }
}

// Split forward, step 4: each re-run task composites its segment again for
// its pixels from their chained state with the exact stop rule (a pixel that
// does not stop there after all continues through the next segments as the
// chain does), records their state at the following boundaries, and writes
// them.
template <int WIN>
__global__ void __launch_bounds__(32 * kWarps, 1) k_render_fwd_rerun(ViewTable vt, RasterCfg cfg,
                                                                    const int2 *__restrict__ ranges,
                                                                    const int *__restrict__ ids,
                                                                    const uint8_t *__restrict__ masks,
                                                                    const float2 *__restrict__ xy,
                                                                    const float4 *__restrict__ co,
                                                                    const float4 *__restrict__ rgbd,
                                                                    float *__restrict__ img,
                                                                    float *__restrict__ T_final,
                                                                    int *__restrict__ last,
                                                                    float *__restrict__ depth, SegWs seg) {
    griddep_wait();
    __shared__ int s_list[kWarps][WIN];
    __shared__ float2 s_p[kWarps][32];
    __shared__ float4 s_q[kWarps][32];
    __shared__ float4 s_c[kWarps][32];
    __shared__ int s_pos[kWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const FwdShared sh{s_p[warp], s_q[warp], s_c[warp], s_pos[warp], s_list[warp], nullptr};
    const int n = min(seg.count[3], seg.fcap);
    for (int k = blockIdx.x * kWarps + warp; k < n; k += gridDim.x * kWarps) {
        const int4 task = seg.tasks[k];
        const ItemRef R = item_ref(seg, task.x);
        const int S = R.H.w, unit = 8 * R.H.x + R.blk, item0 = task.x - R.sgi, slot0 = task.z;
        const bool in = (task.y >> lane) & 1;
        const Unit t = unit_ctx(vt, R.H.y, R.blk);
        const int2 rg = ranges[R.H.y];
        const float fx = t.px + 0.5f, fy = t.py + 0.5f;
        FwdState st{1.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0, true};
        if (in) {
            const float *r = seg.fres + (long long)task.x * kFresFloats;
            st = FwdState{r[lane], r[32 + lane], r[64 + lane], r[96 + lane], r[128 + lane],
                          __float_as_int(r[160 + lane]), false};
        }
        for (int sgi = R.sgi; sgi < S && __any_sync(0xffffffffu, !st.done); ++sgi) {
            bool exact = sgi == R.sgi;
            if (!exact && !st.done) {
                const float *r = seg.fres + (long long)(item0 + sgi) * kFresFloats;
                const float Tl = r[lane];
                const int lw = __float_as_int(r[160 + lane]);
                if (lw < 0 || st.T * Tl < cfg.t_min) {
                    exact = true;
                } else {
                    st.C0 += st.T * r[32 + lane]; st.C1 += st.T * r[64 + lane]; st.C2 += st.T * r[96 + lane];
                    st.D += st.T * r[128 + lane];
                    if (lw > 0) st.last = lw;
                    st.T *= Tl;
                }
            }
            if (__any_sync(0xffffffffu, exact && !st.done)) {
                const int lo = rg.x + (sgi << cfg.seg_shift), hi = min(rg.y, lo + (1 << cfg.seg_shift));
                FwdState x = st;
                x.done = st.done || !exact;
                fwd_range<WIN>(cfg, masks, ids, xy, co, rgbd, rg.x, lo, hi, R.blk, fx, fy, x, sh);
                if (exact && !st.done) st = x;
            }
            const int slot = slot0 + sgi;
            if (in && sgi < S - 1 && slot < seg.cap) {  // this pixel's state at boundary sgi + 1
                float *ck = seg.ckpt + (long long)slot * kCkptFloats;
                ck[lane] = st.T; ck[32 + lane] = st.C0; ck[64 + lane] = st.C1; ck[96 + lane] = st.C2;
                ck[128 + lane] = st.D;
            }
            if (lane == 0 && sgi < S - 1 && slot < seg.cap) seg.items[slot] = make_int2(unit, sgi + 1);
        }
        if (in) fwd_write(cfg, t, st, img, T_final, last, depth);
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
constexpr int kDirectLanes = 16;  // up to this many active lanes: each issues its own (vector) atomics

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
                                                              float *__restrict__ acc, long long nrec,
                                                              const float *__restrict__ depth, SegWs seg,
                                                              int item_blocks) {
    griddep_wait();
    __shared__ int s_list[kWarps][WIN];
    __shared__ float2 s_p[kWarps][32];
    __shared__ float4 s_q[kWarps][32];
    __shared__ float4 s_c[kWarps][32];
    __shared__ int s_id[kWarps][32];
    __shared__ int s_pos[kWarps][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // one work item: a unit's last segment from T_final and the background
    // (item < 0), or the checkpointed segment bk-1 of a long tile's block
    auto work = [&](const int unit, const int item, const int bk) {
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

    // pair range of this warp: the unit's last segment [S_last << shift, wmax)
    // or, for an item, segment bk-1, which starts from the checkpoint at
    // boundary bk: T there and the colour behind = (final - in front) / T
    int lo = rg.x, hi = rg.x + wmax;
    if (cfg.seg_shift >= 0 && !seg.count[4]) {
        const int s_last = (wmax - 1) >> cfg.seg_shift;
        if (item >= 0) {
            if (bk > s_last) return;  // boundary at or past the unit's last blended pair
            lo = rg.x + ((bk - 1) << cfg.seg_shift);
            hi = rg.x + (bk << cfg.seg_shift);
            const float *ck = seg.ckpt + (long long)item * kCkptFloats;
            if (t.inside) {
                T = ck[lane];
                const float inv = 1.0f / T;
                R0 = (img[t.img] - ck[32 + lane]) * inv;
                R1 = (img[t.img + t.plane] - ck[64 + lane]) * inv;
                R2 = (img[t.img + 2 * t.plane] - ck[96 + lane]) * inv;
                RD = depth ? (depth[t.pix] - ck[128 + lane]) * inv : 0.0f;
            }
        } else {
            lo = rg.x + (s_last << cfg.seg_shift);
        }
    }
    const int wbase = rg.x & ~15;
    for (int kw = (hi - 1 - wbase) / WIN; kw >= (lo - wbase) / WIN; --kw) {
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
                // the test without a divergent branch: every lane evaluates the Gaussian
                const float2 p = s_p[warp][k];
                const float4 q = s_q[warp][k];
                const float dx = fx - p.x, dy = fy - p.y;
                const float power = gauss_power(q.x, q.y, q.z, dx, dy);
                const float G = __expf(power);
                const float alpha = fminf(cfg.alpha_max, q.w * G);
                const bool on = s_pos[warp][k] - rg.x < lst && !(power > 0.0f) && !(alpha < cfg.alpha_min);
                const uint32_t act = __ballot_sync(0xffffffffu, on);
                if (act == 0u) continue;
                // off lanes take alpha = G = 0: their sums below are zero and T, R stay as they are
                // (no divergent branch around the arithmetic)
                const float a_ = on ? alpha : 0.0f;
                const float gu = on && q.w * G <= cfg.alpha_max ? G : 0.0f;  // alpha not clamped
                const float4 col = s_c[warp][k];
                T = __fdividef(T, 1.0f - a_);  // transmittance in front of this Gaussian
                const float w = a_ * T;
                float v[16];
                v[kAccR] = g0 * w; v[kAccG] = g1 * w; v[kAccBl] = g2 * w; v[kAccZ] = gD * w;
                const float dLda = T * (g0 * (col.x - R0) + g1 * (col.y - R1) + g2 * (col.z - R2) + gD * (col.w - RD));
                R0 = a_ * col.x + (1.0f - a_) * R0;
                R1 = a_ * col.y + (1.0f - a_) * R1;
                R2 = a_ * col.z + (1.0f - a_) * R2;
                RD = a_ * col.w + (1.0f - a_) * RD;
                v[kAccO] = dLda * gu;
                const float dp = dLda * q.w * gu;
                v[kAccU] = dp * (q.x * dx + q.y * dy);
                v[kAccV] = dp * (q.z * dy + q.y * dx);
                v[kAccA] = -0.5f * dp * dx * dx;
                v[kAccB] = -dp * dx * dy;
                v[kAccC] = -0.5f * dp * dy * dy;
                v[kAccOmega] = STATS && on ? 1.0f : 0.0f;
                v[kAccKappa] = STATS && on ? mask : 0.0f;
                v[kAccMaxW] = STATS ? w : 0.0f;
                v[13] = v[14] = v[15] = 0.0f;
                float *ar = acc + (long long)s_id[warp][k] * kAccStride;  // this record's sums
                if (__popc(act) <= kDirectLanes) {
                    // a few pixels: each active lane adds its values itself, four per vector atomic
                    if (on) {
                        float4 *a4 = reinterpret_cast<float4 *>(ar);
                        atomicAdd(a4, make_float4(v[kAccU], v[kAccV], v[kAccA], v[kAccB]));
                        atomicAdd(a4 + 1, make_float4(v[kAccC], v[kAccO], v[kAccR], v[kAccG]));
                        atomicAdd(a4 + 2, make_float4(v[kAccBl], v[kAccZ], v[kAccOmega], v[kAccKappa]));
                        if (STATS) atomicMax((int *)&ar[kAccMaxW], __float_as_int(v[kAccMaxW]));  // w >= 0
                    }
                } else {
                    const float mw = STATS ? warp_max(v[kAccMaxW]) : 0.0f;
                    const float tot = warp_transpose_sum16(v);
                    const int plane = (lane >> 1) & 15;
                    const bool mine = (lane & 1) == 0 && plane < (STATS ? kAccMaxW : kAccGrad) &&
                                      (plane != kAccZ || has_depth) && (plane != kAccKappa || tot > 0.0f);
                    if (mine) atomicAdd(&ar[plane], tot);
                    if (STATS && lane == 1) atomicMax((int *)&ar[kAccMaxW], __float_as_int(mw));
                }
            }
            __syncwarp();
            cur = nxt;
        }
    }
    };  // work
    // CTAs [0, item_blocks) loop over the checkpointed segments of long tiles
    if ((int)blockIdx.x < item_blocks) {
        const int n = min(seg.count[2], seg.cap);
        for (int it = blockIdx.x * kWarps + warp; it < n; it += item_blocks * kWarps) {
            const int2 e = seg.items[it];
            if (e.x >= 0) work(e.x, it, e.y);  // x < 0: a reserved slot without a checkpoint
        }
        return;
    }
    const int unit = (blockIdx.x - item_blocks) * kWarps + warp;
    if (unit >= vt.total_tiles * 8) return;
    work(unit, -1, 0);
}

// ---------------------------------------------------------------------------
// Stored per-pixel lists: the alternative to recomputing the blending in the
// backward (the paper composites sorted Gaussians along each ray, Supp. D.2;
// either backward differentiates that sum).  The forward records, for every
// pixel, the record id and alpha of each Gaussian it blends, front to back: a
// counting pass (which also renders), an exclusive scan of the counts into
// offsets, and a storing pass.  The backward walks each pixel's list from the
// back, one thread per pixel, and adds each event's sums to its record with
// vector atomics.  The compositing itself is the unsplit traversal of
// k_render_fwd, bit for bit.

struct ListHook {
    static constexpr bool kNeedsId = true;
    long long base, cap;
    long long *n;  // this lane's count of blend events so far
    int *__restrict__ lid;
    float *__restrict__ lal;
    bool store;
    __device__ __forceinline__ void operator()(const FwdShared &sh, int k, float a) {
        const long long j = base + *n;
        if (store && j < cap) {
            lid[j] = sh.id[k];
            lal[j] = a;
        }
        ++*n;
    }
};

template <int WIN, bool STORE>
__global__ void __launch_bounds__(32 * kWarps) k_render_fwd_lists(ViewTable vt, RasterCfg cfg,
                                                                  const int2 *__restrict__ ranges,
                                                                  const int *__restrict__ ids,
                                                                  const uint8_t *__restrict__ masks,
                                                                  const int *__restrict__ order,
                                                                  const float2 *__restrict__ xy,
                                                                  const float4 *__restrict__ co,
                                                                  const float4 *__restrict__ rgbd,
                                                                  float *__restrict__ img, float *__restrict__ T_final,
                                                                  int *__restrict__ last, float *__restrict__ depth,
                                                                  long long *__restrict__ count_off,
                                                                  int *__restrict__ lid, float *__restrict__ lal,
                                                                  long long cap) {
    griddep_wait();
    __shared__ int s_list[kWarps][WIN];
    __shared__ float2 s_p[kWarps][32];
    __shared__ float4 s_q[kWarps][32];
    __shared__ float4 s_c[kWarps][32];
    __shared__ int s_pos[kWarps][32];
    __shared__ int s_id[kWarps][32];
    const int warp = threadIdx.x >> 5;
    const FwdShared sh{s_p[warp], s_q[warp], s_c[warp], s_pos[warp], s_list[warp], s_id[warp]};
    const int unit = blockIdx.x * kWarps + warp;
    if (unit >= vt.total_tiles * 8) return;
    const int tile = order[unit >> 3], bit = unit & 7;
    const int2 rg = ranges[tile];
    const Unit t = unit_ctx(vt, tile, bit);
    FwdState st{1.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0, !t.inside};
    long long n = 0;
    ListHook hook{STORE && t.inside ? count_off[t.pix] : 0, cap, &n, lid, lal, STORE};
    fwd_range<WIN, ListHook>(cfg, masks, ids, xy, co, rgbd, rg.x, rg.x, rg.y, bit, t.px + 0.5f, t.py + 0.5f, st, sh,
                             hook);
    if (STORE) return;
    fwd_write(cfg, t, st, img, T_final, last, depth);
    if (t.inside) count_off[t.pix] = n;
}

// Exclusive scan of the per-pixel counts into offsets, in place, over 4096
// pixels per CTA (4 per thread); count_off[npx] gets the total.
constexpr int kListScanThreads = 1024, kListScanItems = 4;
constexpr int kListScanTile = kListScanThreads * kListScanItems;

__device__ __forceinline__ long long block_scan_ll(long long x, long long &total, long long *sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long inc = x;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) sm[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const long long wv = sm[lane];  // 32 warps
        long long wi = wv;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        sm[lane] = wi - wv;
        if (lane == 31) sm[32] = wi;
    }
    __syncthreads();
    const long long r = sm[warp] + inc - x;
    total = sm[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kListScanThreads) k_list_scan_sums(const long long *__restrict__ cnt, long long npx,
                                                                     long long *__restrict__ bsum) {
    griddep_wait();
    __shared__ long long sm[33];
    long long x = 0;
    const long long b = (long long)blockIdx.x * kListScanTile + threadIdx.x * kListScanItems;
    #pragma unroll
    for (int i = 0; i < kListScanItems; ++i) x += b + i < npx ? cnt[b + i] : 0;
    long long total;
    block_scan_ll(x, total, sm);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// One CTA: exclusive scan of the CTA sums; the total and the capacity check.
__global__ void __launch_bounds__(kListScanThreads) k_list_scan_top(long long *__restrict__ bsum, int nb,
                                                                    long long *__restrict__ count_off, long long npx,
                                                                    long long cap, int *__restrict__ status) {
    griddep_wait();
    __shared__ long long sm[33];
    long long run = 0;
    for (int b0 = 0; b0 < nb; b0 += kListScanThreads) {
        const int b = b0 + threadIdx.x;
        const long long x = b < nb ? bsum[b] : 0;
        long long total;
        const long long ex = block_scan_ll(x, total, sm);
        if (b < nb) bsum[b] = run + ex;
        run += total;
    }
    if (threadIdx.x == 0) {
        count_off[npx] = run;
        if (run > cap && status) atomicOr(status, 1 << GS_ERR_CAPACITY);
    }
}

__global__ void __launch_bounds__(kListScanThreads) k_list_scan_apply(long long *__restrict__ count_off, long long npx,
                                                                      const long long *__restrict__ bsum) {
    griddep_wait();
    __shared__ long long sm[33];
    const long long b = (long long)blockIdx.x * kListScanTile + threadIdx.x * kListScanItems;
    long long c[kListScanItems], x = 0;
    #pragma unroll
    for (int i = 0; i < kListScanItems; ++i) {
        c[i] = b + i < npx ? count_off[b + i] : 0;
        x += c[i];
    }
    long long total;
    long long run = bsum[blockIdx.x] + block_scan_ll(x, total, sm);
    #pragma unroll
    for (int i = 0; i < kListScanItems; ++i) {
        if (b + i < npx) count_off[b + i] = run;
        run += c[i];
    }
}

// One thread per pixel: the pixel's blend events from the back, T recovered
// by division as in k_render_bwd, the colour behind carried; alpha is the
// stored one (unclamped when below alpha_max, where G = alpha / opacity).
template <bool STATS>
__global__ void __launch_bounds__(256) k_render_bwd_lists(ViewTable vt, RasterCfg cfg, long long npx,
                                                          const long long *__restrict__ off,
                                                          const int *__restrict__ lid, const float *__restrict__ lal,
                                                          long long cap, const float2 *__restrict__ xy,
                                                          const float4 *__restrict__ co,
                                                          const float4 *__restrict__ rgbd,
                                                          const float *__restrict__ img,
                                                          const float *__restrict__ T_final,
                                                          const float *__restrict__ dL_dimg,
                                                          const float *__restrict__ target, float tau_err,
                                                          float *__restrict__ acc) {
    griddep_wait();
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < npx;
         q += (long long)gridDim.x * blockDim.x) {
        int v = 0;
        while (v + 1 < vt.n_views && vt.v[v + 1].pix_offset <= q) ++v;
        const ViewDesc &c = vt.v[v];
        const long long local = q - c.pix_offset;
        const int py = (int)(local / c.W), px = (int)(local - (long long)py * c.W);
        const long long plane = (long long)c.W * c.H, i0 = 3 * c.pix_offset + local;
        const float fx = px + 0.5f, fy = py + 0.5f;
        float T = T_final[q];
        const float g0 = dL_dimg[i0], g1 = dL_dimg[i0 + plane], g2 = dL_dimg[i0 + 2 * plane];
        float mask = 0.0f;
        if (STATS) {
            const float e = fabsf(target[i0] - img[i0]) + fabsf(target[i0 + plane] - img[i0 + plane]) +
                            fabsf(target[i0 + 2 * plane] - img[i0 + 2 * plane]);
            mask = e > tau_err ? 1.0f : 0.0f;
        }
        float R0 = cfg.bg[0], R1 = cfg.bg[1], R2 = cfg.bg[2];
        const long long b = off[q], e = min(off[q + 1], cap);
        for (long long j = e - 1; j >= b; --j) {
            const int r = lid[j];
            const float alpha = lal[j];
            const float2 p = xy[r];
            const float4 qq = co[r];
            const float4 col = rgbd[r];
            const float dx = fx - p.x, dy = fy - p.y;
            T = __fdividef(T, 1.0f - alpha);
            const float w = alpha * T;
            const float dLda = T * (g0 * (col.x - R0) + g1 * (col.y - R1) + g2 * (col.z - R2));
            R0 = alpha * col.x + (1.0f - alpha) * R0;
            R1 = alpha * col.y + (1.0f - alpha) * R1;
            R2 = alpha * col.z + (1.0f - alpha) * R2;
            float vo = 0.0f, vu = 0.0f, vv = 0.0f, va = 0.0f, vb = 0.0f, vc = 0.0f;
            if (alpha < cfg.alpha_max) {  // alpha not clamped
                vo = dLda * alpha / qq.w;
                const float dp = dLda * alpha;
                vu = dp * (qq.x * dx + qq.y * dy);
                vv = dp * (qq.z * dy + qq.y * dx);
                va = -0.5f * dp * dx * dx;
                vb = -dp * dx * dy;
                vc = -0.5f * dp * dy * dy;
            }
            float4 *a4 = reinterpret_cast<float4 *>(acc + (long long)r * kAccStride);
            atomicAdd(a4, make_float4(vu, vv, va, vb));
            atomicAdd(a4 + 1, make_float4(vc, vo, g0 * w, g1 * w));
            atomicAdd(a4 + 2, make_float4(g2 * w, 0.0f, STATS ? 1.0f : 0.0f, mask));
            if (STATS) atomicMax((int *)&acc[(long long)r * kAccStride + kAccMaxW], __float_as_int(w));
        }
    }
}

static int sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    return sms;
}

// CTAs of a grid-stride loop over at most `work` warps of work
static int stride_blocks(long long work) {
    return (int)std::max(1ll, std::min(ceil_div(work, kWarps), (long long)kSplitCtasPerSm * sm_count()));
}

void launch_render_fwd(const ViewTable &vt, const RasterCfg &cfg, const int2 *ranges, const int *ids,
                       const uint8_t *masks, const int *order, const float2 *xy, const float4 *co,
                       const float4 *rgbd, float *img, float *T_final, int *last, float *depth, const SegWs &seg,
                       cudaStream_t s) {
    const long long units = 8ll * vt.total_tiles;
    if (units <= 0) return;
    const bool split = cfg.seg_shift >= 0;
    int item_blocks = 0, cgrid = 0, rgrid = 0;
    if (split) {
        cudaMemsetAsync(seg.count, 0, 8 * sizeof(int), s);
        launch_pdl(k_fwd_plan, 1, kPlanThreads, 0, s, ranges, order, vt.total_tiles, cfg.seg_shift, seg);
        item_blocks = stride_blocks(seg.fcap);
        cgrid = stride_blocks(8ll * seg.hcap);
        rgrid = stride_blocks(seg.fcap);
    }
    const unsigned grid = (unsigned)(item_blocks + ceil_div(units, kWarps));
#define GS_FWD(WN)                                                                                                  \
    do {                                                                                                            \
        launch_pdl(k_render_fwd<WN>, grid, 32 * kWarps, 0, s, vt, cfg, ranges, ids, masks, order, xy, co, rgbd, img,        \
                                                      T_final, last, depth, seg, item_blocks);                      \
        if (split) {                                                                                                \
            launch_pdl(k_render_fwd_combine, cgrid, 32 * kWarps, 0, s, vt, cfg, img, T_final, last, depth, seg);            \
            launch_pdl(k_render_fwd_rerun<WN>, rgrid, 32 * kWarps, 0, s, vt, cfg, ranges, ids, masks, xy, co, rgbd, img,    \
                                                                 T_final, last, depth, seg);                        \
        }                                                                                                           \
    } while (0)
    if (cfg.batch == 128) GS_FWD(128);
    else if (cfg.batch == 256) GS_FWD(256);
    else GS_FWD(512);
#undef GS_FWD
}

void launch_render_bwd(const ViewTable &vt, const RasterCfg &cfg, const int2 *ranges, const int *ids,
                       const uint8_t *masks, const int *order, const float2 *xy, const float4 *co,
                       const float4 *rgbd, const float *img, const float *T_final, const int *last, const float *dL_dimg,
                       const float *dL_ddepth, const float *target, float tau_err, bool stats, float *acc,
                       long long nrec, const float *depth, const SegWs &seg, cudaStream_t s) {
    const long long units = 8ll * vt.total_tiles;
    if (units <= 0) return;
    // segment CTAs first, so the long lists' segments start early
    const int item_blocks = cfg.seg_shift >= 0 ? stride_blocks(seg.cap) : 0;
    const unsigned grid = (unsigned)(item_blocks + ceil_div(units, kWarps));
#define GS_BWD(ST, WN) launch_pdl(k_render_bwd<ST, WN>, grid, 32 * kWarps, 0, s, vt, cfg, ranges, ids, masks, order, xy, co, \
                                                                         rgbd, img, T_final, last, dL_dimg, \
                                                                         dL_ddepth, target, tau_err, acc, nrec, \
                                                                         depth, seg, item_blocks)
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

size_t list_scan_bytes(long long npx) {
    return align_up(sizeof(long long) * (size_t)(ceil_div(npx, kListScanTile) + 1), 256);
}

void launch_render_fwd_lists(const ViewTable &vt, const RasterCfg &cfg, const int2 *ranges, const int *ids,
                             const uint8_t *masks, const int *order, const float2 *xy, const float4 *co,
                             const float4 *rgbd, float *img, float *T_final, int *last, float *depth, long long npx,
                             long long *count_off, int *lid, float *lal, long long cap, void *scan_ws, int *status,
                             cudaStream_t s) {
    const long long units = 8ll * vt.total_tiles;
    if (units <= 0 || npx <= 0) return;
    const unsigned grid = (unsigned)ceil_div(units, kWarps);
    const int nb = (int)ceil_div(npx, kListScanTile);
    long long *bsum = (long long *)scan_ws;
#define GS_FWDL(WN)                                                                                                 \
    do {                                                                                                            \
        launch_pdl(k_render_fwd_lists<WN, false>, grid, 32 * kWarps, 0, s, vt, cfg, ranges, ids, masks, order, xy, co, rgbd, \
                                                                   img, T_final, last, depth, count_off, lid, lal,  \
                                                                   cap);                                            \
        launch_pdl(k_list_scan_sums, nb, kListScanThreads, 0, s, count_off, npx, bsum);                                     \
        launch_pdl(k_list_scan_top, 1, kListScanThreads, 0, s, bsum, nb, count_off, npx, cap, status);                      \
        launch_pdl(k_list_scan_apply, nb, kListScanThreads, 0, s, count_off, npx, bsum);                                    \
        launch_pdl(k_render_fwd_lists<WN, true>, grid, 32 * kWarps, 0, s, vt, cfg, ranges, ids, masks, order, xy, co, rgbd,  \
                                                                  img, T_final, last, depth, count_off, lid, lal,   \
                                                                  cap);                                             \
    } while (0)
    if (cfg.batch == 128) GS_FWDL(128);
    else if (cfg.batch == 256) GS_FWDL(256);
    else GS_FWDL(512);
#undef GS_FWDL
}

void launch_render_bwd_lists(const ViewTable &vt, const RasterCfg &cfg, long long npx, const long long *off,
                             const int *lid, const float *lal, long long cap, const float2 *xy, const float4 *co,
                             const float4 *rgbd, const float *img, const float *T_final, const float *dL_dimg,
                             const float *target, float tau_err, bool stats, float *acc, cudaStream_t s) {
    if (npx <= 0) return;
    const unsigned grid = (unsigned)std::min(ceil_div(npx, 256), (long long)sm_count() * 8);
    if (stats)
        launch_pdl(k_render_bwd_lists<true>, grid, 256, 0, s, vt, cfg, npx, off, lid, lal, cap, xy, co, rgbd, img, T_final,
                                                      dL_dimg, target, tau_err, acc);
    else
        launch_pdl(k_render_bwd_lists<false>, grid, 256, 0, s, vt, cfg, npx, off, lid, lal, cap, xy, co, rgbd, img, T_final,
                                                       dL_dimg, target, tau_err, acc);
}

}  // namespace gs
