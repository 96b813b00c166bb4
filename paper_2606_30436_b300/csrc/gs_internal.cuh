// gs_internal.cuh -- shared device-side definitions of the sm_103a Gaussian
// splatting mapping step (views, tiles, the exact FP32 binning arithmetic and
// the alpha evaluation shared by the forward and backward traversals).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gs.h"

namespace gs {

constexpr int kTilePixels = 256;  // tile_w * tile_h, one thread per pixel
constexpr int kBatch = 256;       // Gaussians staged in shared memory per round

struct ViewDesc {
    float R[9], t[3];
    float fx, fy, cx, cy;
    float campos[3];   // camera centre in world coordinates, -R^T t
    float limx, limy;  // Jacobian clamp of x/z and y/z
    int W, H, GW, GH;
    int tile_offset;          // first global tile of this view
    long long pix_offset;     // first pixel of this view in the frame layout
};

struct ViewTable {
    int n_views;
    int tile_w, tile_h;
    int total_tiles;
    ViewDesc v[GS_MAX_VIEWS];
};

__host__ __device__ __forceinline__ long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

// Programmatic dependent launch: a kernel launched with launch_pdl may have its CTAs scheduled
// while the previous kernel on the stream drains; it must begin with griddep_wait(), which
// holds it until that kernel has finished and its writes are visible.  Every kernel so
// launched waits before anything else, so each one completes after all earlier ones.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Adam's bias corrections from a device step counter t (a non-negative integer) without FP64,
// which issues at a small fraction of the FP32 rate on B300 (two FP64 powers at the start of
// every CTA held the Gaussians' Adam back by about 0.01 ms).  A value is the unevaluated sum
// hi + lo of two floats (double-float arithmetic): a product is rounded and its exact error
// taken with one FMA (Dekker's exact product), a sum's error with Knuth's two-sum, and beta^t
// by binary exponentiation over the bits of t, so 1 - beta^t carries about 44 significant bits
// and each correction is rounded to float once.  The _rn intrinsics keep the compiler from
// fusing the rounded operations these error terms depend on.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p)));
    return ff_two_sum(p, e);
}
__device__ __forceinline__ FF ff_one_minus_pow(float beta, long long t) {
    FF r{1.0f, 0.0f}, x{beta, 0.0f};
    for (; t > 0; t >>= 1) {
        if (t & 1) r = ff_mul(r, x);
        x = ff_mul(x, x);
    }
    const FF d = ff_two_sum(1.0f, -r.hi);
    return ff_two_sum(d.hi, __fsub_rn(d.lo, r.lo));
}
__device__ __forceinline__ float ff_recip(FF a) {  // 1 / (hi + lo): one Newton step from 1 / hi
    const float q = __fdiv_rn(1.0f, a.hi);
    const float e = fmaf(-q, a.lo, fmaf(-q, a.hi, 1.0f));
    return fmaf(q, e, q);
}
__device__ __forceinline__ FF ff_sqrt(FF a) {  // sqrt(hi + lo): one Newton step from sqrt(hi)
    const float s = __fsqrt_rn(a.hi);
    const float r = __fadd_rn(fmaf(-s, s, a.hi), a.lo);
    return ff_two_sum(s, __fdiv_rn(r, __fmul_rn(2.0f, s)));
}
// 1 / (1 - b1^t) and 1 / sqrt(1 - b2^t)
__device__ __forceinline__ void adam_bias_inv(float b1, float b2, long long t, float &inv_bc1, float &inv_sqrt_bc2) {
    inv_bc1 = ff_recip(ff_one_minus_pow(b1, t));
    inv_sqrt_bc2 = ff_recip(ff_sqrt(ff_one_minus_pow(b2, t)));
}
// 1 - b1^t and 1 - b2^t
__device__ __forceinline__ void adam_bias(float b1, float b2, long long t, float &bc1, float &bc2) {
    const FF a = ff_one_minus_pow(b1, t), b = ff_one_minus_pow(b2, t);
    bc1 = __fadd_rn(a.hi, a.lo);
    bc2 = __fadd_rn(b.hi, b.lo);
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

__host__ __device__ __forceinline__ size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct RasterCfg {
    float near_z, dilation, alpha_min, alpha_max, t_min, tan_clamp;
    float logit_min;  // FP32 logit of alpha_min: a Gaussian below it never blends and is culled
    float bg[3];
    int tile_w, tile_h;
    int batch;      // pairs a warp scans per step (128, 256, 512)
    int seg_shift;  // log2 of the backward's segment length, -1 = no split
};

// Workspace of the split compositing kernels.  count[0] segment items of the
// forward, count[1] long tiles, count[2] backward checkpoints.  heavy: per long
// tile (schedule index, tile, first item, segments S); fres: per forward item
// the 32 lanes' local T, C0, C1, C2, depth and last (bit 31: stopped), [6][32];
// items / ckpt: per backward checkpoint (unit, boundary k) and the 32 lanes' T
// and colour in front (C0, C1, C2, depth) after the pairs before the boundary,
// [5][32] floats.
struct SegWs {
    int *count;   // [0] forward items, [1] long tiles, [2] checkpoints, [3] re-run tasks,
                  // [4] 1 = the plan did not fit (no split this launch), [5] items the plan needed
    int4 *heavy;
    int hcap;
    float *fres;
    int4 *tasks;  // forward re-runs: (item, lane mask, first checkpoint slot of the block, 0)
    int fcap;     // items, and re-run tasks (at most one per item)
    int2 *items;
    float *ckpt;
    int cap;
};
constexpr int kCkptFloats = 5 * 32;
constexpr int kFresFloats = 6 * 32;

// Capacities of a split workspace for F forward segment items: long tiles
// <= F / 16 (each has at least two segments of 8 blocks), re-run tasks and
// checkpoints <= F; and the bytes that takes.
__host__ __device__ __forceinline__ long long seg_heavy_for(long long F) { return F / 16 + 1; }
__host__ __device__ __forceinline__ size_t seg_bytes_for(long long F) {
    return 256 + align_up(16 * (size_t)seg_heavy_for(F), 256) + align_up(4 * 192 * (size_t)F, 256) +
           align_up(16 * (size_t)F, 256) + align_up(8 * (size_t)F, 256) + 4 * 160 * (size_t)F;
}
// The largest item capacity that fits in `bytes`.
__host__ __device__ __forceinline__ long long seg_items_in(size_t bytes) {
    if (bytes < seg_bytes_for(16)) return 0;
    long long F = (long long)((bytes - 256 - 5 * 256) / (1 + 768 + 16 + 8 + 640 + 1));  // estimate, then exact
    while (seg_bytes_for(F + 1) <= bytes) ++F;
    while (F > 16 && seg_bytes_for(F) > bytes) --F;
    return F;
}
// Worst case for max_pairs pairs: every pair in a long tile, S_t <= len / segment + 1.
__host__ __device__ __forceinline__ long long seg_items_worst(long long max_pairs, int segment) {
    return 16 * (((max_pairs > 0 ? max_pairs : 1) + segment - 1) / segment + 1);
}

// The view that owns a global tile index (linear scan: <= 64 views, uniform
// across the block, served from the constant bank).
__device__ __forceinline__ int view_of_tile(const ViewTable &vt, int tile) {
    int v = 0;
    #pragma unroll 1
    for (int k = 1; k < vt.n_views; ++k)
        if (vt.v[k].tile_offset <= tile) v = k;
    return v;
}

// Camera-frame point and pixel position in the FP32 evaluation order that the
// binning is defined by: every product, sum and quotient rounds to nearest,
// left to right, with no fused multiply-add.
struct ExactPos { float xc, yc, zc, u, v; };

__device__ __forceinline__ ExactPos exact_position(const ViewDesc &c, float mx, float my, float mz) {
    ExactPos p;
    p.xc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.R[0], mx), __fmul_rn(c.R[1], my)), __fmul_rn(c.R[2], mz)), c.t[0]);
    p.yc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.R[3], mx), __fmul_rn(c.R[4], my)), __fmul_rn(c.R[5], mz)), c.t[1]);
    p.zc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.R[6], mx), __fmul_rn(c.R[7], my)), __fmul_rn(c.R[8], mz)), c.t[2]);
    p.u = __fadd_rn(__fdiv_rn(__fmul_rn(c.fx, p.xc), p.zc), c.cx);
    p.v = __fadd_rn(__fdiv_rn(__fmul_rn(c.fy, p.yc), p.zc), c.cy);
    return p;
}

// Tiles overlapped by [u - r, u + r] x [v - r, v + r], exclusive upper bounds,
// clamped to the view's grid; same FP32 rounding as the definition.
struct Rect { int x0, y0, x1, y1; };

__device__ __forceinline__ Rect tile_rect(float u, float v, int radius, int tw, int th, int GW, int GH) {
    const float rf = (float)radius, twf = (float)tw, thf = (float)th;
    float x0 = floorf(__fdiv_rn(__fsub_rn(u, rf), twf));
    float x1 = __fadd_rn(floorf(__fdiv_rn(__fadd_rn(u, rf), twf)), 1.0f);
    float y0 = floorf(__fdiv_rn(__fsub_rn(v, rf), thf));
    float y1 = __fadd_rn(floorf(__fdiv_rn(__fadd_rn(v, rf), thf)), 1.0f);
    Rect r;
    r.x0 = (int)fminf(fmaxf(x0, 0.0f), (float)GW);
    r.x1 = (int)fminf(fmaxf(x1, 0.0f), (float)GW);
    r.y0 = (int)fminf(fmaxf(y0, 0.0f), (float)GH);
    r.y1 = (int)fminf(fmaxf(y1, 0.0f), (float)GH);
    return r;
}

// power = -(a dx^2 + c dy^2)/2 - b dx dy with a pinned operation order, so the
// forward and the backward traversal take identical skip / stop decisions.
__device__ __forceinline__ float gauss_power(float a, float b, float c, float dx, float dy) {
    float q = __fmaf_rn(a, __fmul_rn(dx, dx), __fmul_rn(c, __fmul_rn(dy, dy)));
    return __fmaf_rn(-0.5f, q, -__fmul_rn(b, __fmul_rn(dx, dy)));
}

// Can a Gaussian (pixel position p, conic/opacity q) reach alpha >= alpha_min
// at a pixel centre of the 8x4 block whose first pixel is (bx0, by0)?
// alpha >= alpha_min iff d^T Q d <= tau, tau = 2 ln(o / alpha_min); the
// ellipse's bounding box has half-widths sqrt(tau Sigma'_xx), sqrt(tau
// Sigma'_yy) with Sigma' = Q^-1.  tau gets an additive margin (alpha relative
// errors up to 1%) and the box 0.05 px, so rounding never drops a Gaussian
// that the per-pixel test would keep: skipping on a clear bit is exact.
struct Reach { float cx, cy, ex, ey; bool any, all; };

__device__ __forceinline__ Reach reach_box(float2 p, float4 q, float alpha_min) {
    Reach r;
    r.any = q.w >= alpha_min;
    r.all = false;
    const float tau = 2.0f * __logf(q.w / alpha_min) + 0.02f;
    const float det = q.x * q.z - q.y * q.y;
    if (!(det > 0.0f)) r.all = true;
    const float idet = 1.0f / det;
    r.ex = sqrtf(fmaxf(tau * q.z * idet, 0.0f)) + 0.05f;
    r.ey = sqrtf(fmaxf(tau * q.x * idet, 0.0f)) + 0.05f;
    r.cx = p.x - 0.5f;  // pixel i has centre i + 0.5: work in pixel-index space
    r.cy = p.y - 0.5f;
    return r;
}

// Bit b (b = 0..7) set when the Gaussian can reach block b of the tile whose
// first pixel is (x0, y0); blocks are 8 wide and 4 tall, row-major, tile_w/8
// per row.
__device__ __forceinline__ uint32_t block_mask_of(const Reach &r, int x0, int y0, int tile_w) {
    if (!r.any) return 0u;
    if (r.all) return 0xffu;
    const int ncols = tile_w >> 3, nrows = 8 / ncols;
    // block column b_x holds pixel indices [8 b_x, 8 b_x + 7]: it meets the box's
    // span [lx0, lx1] iff b_x in [ceil((lx0 - 7) / 8), floor(lx1 / 8)]
    const float lx0 = r.cx - r.ex - (float)x0, lx1 = r.cx + r.ex - (float)x0;
    const float ly0 = r.cy - r.ey - (float)y0, ly1 = r.cy + r.ey - (float)y0;
    const int c0 = max(0, (int)ceilf((lx0 - 7.0f) * 0.125f)), c1 = min(ncols - 1, (int)floorf(lx1 * 0.125f));
    const int r0 = max(0, (int)ceilf((ly0 - 3.0f) * 0.25f)), r1 = min(nrows - 1, (int)floorf(ly1 * 0.25f));
    if (c0 > c1 || r0 > r1) return 0u;
    const uint32_t row = ((1u << (c1 + 1)) - 1u) & ~((1u << c0) - 1u);  // columns c0..c1 of one row
    uint32_t m = 0;
    for (int rr = r0; rr <= r1; ++rr) m |= row << (rr * ncols);
    return m;
}

__device__ __forceinline__ uint32_t block_mask8(float2 p, float4 q, float alpha_min, int x0, int y0, int tile_w) {
    return block_mask_of(reach_box(p, q, alpha_min), x0, y0, tile_w);
}

// Bytes of the per-pair block-mask array for max_pairs pairs: the render
// kernels read it in aligned 16-byte words up to 512 bytes past a range end.
__host__ __device__ __forceinline__ long long block_mask_bytes(long long max_pairs) {
    return max_pairs + 16 + 512;
}



// Rotation matrix (row-major) of the unit quaternion (w, x, y, z).
__device__ __forceinline__ void quat_rotation(float qw, float qx, float qy, float qz, float *R) {
    R[0] = 1.f - 2.f * (qy * qy + qz * qz); R[1] = 2.f * (qx * qy - qw * qz); R[2] = 2.f * (qx * qz + qw * qy);
    R[3] = 2.f * (qx * qy + qw * qz); R[4] = 1.f - 2.f * (qx * qx + qz * qz); R[5] = 2.f * (qy * qz - qw * qx);
    R[6] = 2.f * (qx * qz - qw * qy); R[7] = 2.f * (qy * qz + qw * qx); R[8] = 1.f - 2.f * (qx * qx + qy * qy);
}

// Gradient of gscale * sum_k |s_k - mean(s)|, s = exp(log-scale), with
// respect to the three log-scales, added into g (the isotropic term L_iso,
// Supp. D.4): d|s_k - m|/ds_j = sign(s_k - m) (delta_kj - 1/3).
__device__ __forceinline__ void iso_grad(float ls0, float ls1, float ls2, float gscale, float *g) {
    const float s0 = expf(ls0), s1 = expf(ls1), s2 = expf(ls2);
    const float m = (s0 + s1 + s2) * (1.0f / 3.0f);
    const float d0 = s0 - m, d1 = s1 - m, d2 = s2 - m;
    const float e0 = d0 > 0.f ? 1.f : (d0 < 0.f ? -1.f : 0.f);
    const float e1 = d1 > 0.f ? 1.f : (d1 < 0.f ? -1.f : 0.f);
    const float e2 = d2 > 0.f ? 1.f : (d2 < 0.f ? -1.f : 0.f);
    const float em = (e0 + e1 + e2) * (1.0f / 3.0f);
    g[0] += gscale * (e0 - em) * s0;
    g[1] += gscale * (e1 - em) * s1;
    g[2] += gscale * (e2 - em) * s2;
}

}  // namespace gs
