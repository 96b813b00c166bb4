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

struct RasterCfg {
    float near_z, dilation, alpha_min, alpha_max, t_min, tan_clamp;
    float bg[3];
    int tile_w, tile_h;
};

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

__device__ __forceinline__ float ceil_div_f(float a, float b) { return ceilf(a / b); }

__host__ __device__ __forceinline__ long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

__host__ __device__ __forceinline__ size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace gs
