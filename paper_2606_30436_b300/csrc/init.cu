// init.cu -- probabilistic initialisation of new anchors at a keyframe
// (Sec. 3.3.1) and the voxel hash of the dynamic map expansion (Supp. D.5).
//
// k_init_grad_minmax: the minimum and maximum of ||grad D|| over the
// keyframe (and the rendered depth), reduced per block into two atomics
// (non-negative FP32 bit patterns order like unsigned integers; the minimum
// is kept as the maximum of the complement so that both words start at 0).
// k_init_prob: 32x32 pixel tiles.  The channel mean Y of the tile and a halo
// of the larger blur radius is staged in shared memory, blurred along rows by
// both Gaussians in one pass, then along columns, each thread walking four
// rows with a sliding window (the default radii 3 and 5 are compile-time
// constants); the DoG, the normalised depth gradient and P of the keyframe and
// of the render are combined in registers and only P (or P_kf) is written.
// k_init_select: 3x3 non-maximum suppression from a staged tile, the draw,
// the unprojection, the level and voxel key, and the insertion into the
// table (64-bit compare-and-swap, linear probing bounded by the capacity);
// each slot of a new voxel keeps its lowest claiming pixel (atomicMin).
// k_init_count / k_init_emit: the pixels that own a new voxel are numbered in
// raster order: 1024-pixel blocks count them, and each emitting block sums
// the counts of the blocks before it, ranks its own pixels and writes the
// anchor records; their slots are then settled.
#include <algorithm>
#include <climits>
#include <cstdint>

#include "gs_internal.cuh"
#include "gs_kernels.h"

namespace gs {

namespace {

constexpr int kTW = 32, kTH = 8, kR = GS_INIT_MAX_RADIUS, kThreads = kTW * kTH;
constexpr unsigned long long kEmpty = ~0ull;
constexpr int kIdxBias = 1 << 19;

// splitmix64's output mix (Steele, Lea and Flood's SplitMix; constants of
// Vigna's splitmix64): spreads the packed voxel key over the table.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long voxel_key(int l, int ix, int iy, int iz) {
    return ((unsigned long long)l << 60) | ((unsigned long long)(ix + kIdxBias) << 40) |
           ((unsigned long long)(iy + kIdxBias) << 20) | (unsigned long long)(iz + kIdxBias);
}

__device__ __forceinline__ bool idx_in_range(int v) { return v >= -kIdxBias && v < kIdxBias; }

__device__ __forceinline__ float depth_grad(const float *__restrict__ D, int W, int H, int x, int y) {
    const long long row = (long long)y * W;
    const float gx = (D[row + min(x + 1, W - 1)] - D[row + max(x - 1, 0)]) * 0.5f;
    const float gy = (D[(long long)min(y + 1, H - 1) * W + x] - D[(long long)max(y - 1, 0) * W + x]) * 0.5f;
    return sqrtf(gx * gx + gy * gy);
}

// One block per row (strided): threads walk the row, so no pixel index is divided.
__global__ void __launch_bounds__(kThreads) k_init_grad_minmax(const float *__restrict__ depth,
                                                               const float *__restrict__ depth_r, int W, int H,
                                                               unsigned *__restrict__ minmax) {
    __shared__ unsigned red[2][kThreads / 32];
    const int z = blockIdx.y;
    const float *D = z ? depth_r : depth;
    unsigned lo = 0u, hi = 0u;
    for (int y = blockIdx.x; y < H; y += gridDim.x)
        for (int x = threadIdx.x; x < W; x += kThreads) {
            const unsigned g = __float_as_uint(depth_grad(D, W, H, x, y));
            lo = max(lo, ~g);
            hi = max(hi, g);
        }
    lo = __reduce_max_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = lo;
        red[1][threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < kThreads / 32; ++i) {
            lo = max(lo, red[0][i]);
            hi = max(hi, red[1][i]);
        }
        atomicMax(&minmax[2 * z], lo);
        atomicMax(&minmax[2 * z + 1], hi);
    }
}

constexpr int kPT = 32, kPH = 16;                        // probability tile: 32 x 16 pixels
constexpr int kRowsPerThread = kPH / (kThreads / kPT);  // 2 consecutive rows per thread

// P of one map for the thread's pixels (rows kRowsPerThread ty + j, column
// tx of the tile).  R1, R2 > 0: compile-time radii; 0: the runtime ones.
template <int R1, int R2, int RS>
__device__ __forceinline__ void tile_p(const float *__restrict__ I, const float *__restrict__ D, int W, int H,
                                       int x0, int y0, const InitBlur &bw, const unsigned *__restrict__ minmax, int z,
                                       float lambda, float (*ys)[kPT + 2 * RS], float (*hb)[kPH + 2 * RS][kPT],
                                       float (*ds)[kPT + 2], float *pv) {
    const int r1 = R1 ? R1 : bw.r1, r2 = R2 ? R2 : bw.r2, R = R1 ? RS : bw.R;
    const long long npx = (long long)W * H;
    const int nx = kPT + 2 * R, ny = kPH + 2 * R;
    constexpr float kThird = 1.0f / 3.0f;
    // channel mean with a halo of R and the depth with a halo of 1, edges replicated
    for (int i = threadIdx.x; i < ny * nx; i += kThreads) {
        const int r = i / nx, c = i % nx;
        const int y = min(max(y0 - R + r, 0), H - 1), x = min(max(x0 - R + c, 0), W - 1);
        const long long p = (long long)y * W + x;
        ys[r][c] = (I[p] + I[npx + p] + I[2 * npx + p]) * kThird;
    }
    for (int i = threadIdx.x; i < (kPH + 2) * (kPT + 2); i += kThreads) {
        const int r = i / (kPT + 2), c = i % (kPT + 2);
        const int y = min(max(y0 - 1 + r, 0), H - 1), x = min(max(x0 - 1 + c, 0), W - 1);
        ds[r][c] = D[(long long)y * W + x];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ny * kPT; i += kThreads) {
        const int r = i / kPT, c = i % kPT + R;
        float a = bw.w1[0] * ys[r][c], b = bw.w2[0] * ys[r][c];
        #pragma unroll
        for (int k = 1; k <= (R1 ? R1 : kR); ++k)
            if (R1 || k <= r1) a += bw.w1[k] * (ys[r][c - k] + ys[r][c + k]);
        #pragma unroll
        for (int k = 1; k <= (R2 ? R2 : kR); ++k)
            if (R2 || k <= r2) b += bw.w2[k] * (ys[r][c - k] + ys[r][c + k]);
        hb[0][r][c - R] = a;
        hb[1][r][c - R] = b;
    }
    __syncthreads();
    const int tx = threadIdx.x % kPT, ty = threadIdx.x / kPT, o0 = kRowsPerThread * ty;
    float b1[kRowsPerThread], b2[kRowsPerThread];
    if (R1 && R2) {
        // sliding windows down the column: rows o0 + R - r .. o0 + 3 + R + r of hb
        float c1[kRowsPerThread + 2 * (R1 ? R1 : 1)], c2[kRowsPerThread + 2 * (R2 ? R2 : 1)];
        #pragma unroll
        for (int k = 0; k < kRowsPerThread + 2 * R1; ++k) c1[k] = hb[0][o0 + R - R1 + k][tx];
        #pragma unroll
        for (int k = 0; k < kRowsPerThread + 2 * R2; ++k) c2[k] = hb[1][o0 + R - R2 + k][tx];
        #pragma unroll
        for (int j = 0; j < kRowsPerThread; ++j) {
            float a = bw.w1[0] * c1[j + R1], b = bw.w2[0] * c2[j + R2];
            #pragma unroll
            for (int k = 1; k <= R1; ++k) a += bw.w1[k] * (c1[j + R1 - k] + c1[j + R1 + k]);
            #pragma unroll
            for (int k = 1; k <= R2; ++k) b += bw.w2[k] * (c2[j + R2 - k] + c2[j + R2 + k]);
            b1[j] = a;
            b2[j] = b;
        }
    } else {
        #pragma unroll
        for (int j = 0; j < kRowsPerThread; ++j) {
            const int r = o0 + j + R;
            float a = bw.w1[0] * hb[0][r][tx], b = bw.w2[0] * hb[1][r][tx];
            for (int k = 1; k <= r1; ++k) a += bw.w1[k] * (hb[0][r - k][tx] + hb[0][r + k][tx]);
            for (int k = 1; k <= r2; ++k) b += bw.w2[k] * (hb[1][r - k][tx] + hb[1][r + k][tx]);
            b1[j] = a;
            b2[j] = b;
        }
    }
    const float lo = __uint_as_float(~minmax[2 * z]), hi = __uint_as_float(minmax[2 * z + 1]);
    const int x = x0 + tx;
    #pragma unroll
    for (int j = 0; j < kRowsPerThread; ++j) {
        const int y = y0 + o0 + j;
        float p = 0.0f;
        if (x < W && y < H) {
            const float dog = fminf(bw.scale * fabsf(b1[j] - b2[j]), 1.0f);
            const int r = o0 + j + 1, c = tx + 1;
            const float gx = (ds[r][c + 1] - ds[r][c - 1]) * 0.5f, gy = (ds[r + 1][c] - ds[r - 1][c]) * 0.5f;
            const float gn = hi > lo ? (sqrtf(gx * gx + gy * gy) - lo) / (hi - lo) : 0.0f;
            p = fminf(lambda * dog + (1.0f - lambda) * gn, 1.0f);
        }
        pv[j] = z ? fmaxf(pv[j] - p, 0.0f) : p;  // P_kf = max(P - P^, 0)
    }
}

template <int R1, int R2>
__global__ void __launch_bounds__(kThreads) k_init_prob(const float *__restrict__ img, const float *__restrict__ depth,
                                                        const float *__restrict__ img_r,
                                                        const float *__restrict__ depth_r, int W, int H,
                                                        const __grid_constant__ InitBlur bw,
                                                        const unsigned *__restrict__ minmax, float lambda,
                                                        float *__restrict__ prob) {
    constexpr int RS = R1 && R2 ? (R1 > R2 ? R1 : R2) : kR;
    __shared__ float ys[kPH + 2 * RS][kPT + 2 * RS];
    __shared__ float hb[2][kPH + 2 * RS][kPT];
    __shared__ float ds[kPH + 2][kPT + 2];
    const int x0 = blockIdx.x * kPT, y0 = blockIdx.y * kPH;
    float pv[kRowsPerThread];
    tile_p<R1, R2, RS>(img, depth, W, H, x0, y0, bw, minmax, 0, lambda, ys, hb, ds, pv);
    if (img_r) {
        __syncthreads();  // the tile's shared arrays are reused for the render
        tile_p<R1, R2, RS>(img_r, depth_r, W, H, x0, y0, bw, minmax, 1, lambda, ys, hb, ds, pv);
    }
    const int x = x0 + threadIdx.x % kPT, yb = y0 + kRowsPerThread * (threadIdx.x / kPT);
    #pragma unroll
    for (int j = 0; j < kRowsPerThread; ++j)
        if (x < W && yb + j < H) prob[(long long)(yb + j) * W + x] = pv[j];
}

__global__ void __launch_bounds__(kThreads) k_init_select(const float *__restrict__ prob,
                                                          const float *__restrict__ uniform,
                                                          const float *__restrict__ depth, int W, int H, InitCam cam,
                                                          const __grid_constant__ InitLod lod,
                                                          unsigned long long *__restrict__ keys,
                                                          int *__restrict__ owner, long long cap,
                                                          int *__restrict__ cand, uint8_t *__restrict__ selected,
                                                          int *__restrict__ status) {
    __shared__ float ps[kTH + 2][kTW + 2];
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
    for (int i = threadIdx.x; i < (kTH + 2) * (kTW + 2); i += kThreads) {
        const int r = i / (kTW + 2), c = i % (kTW + 2);
        const int y = y0 - 1 + r, x = x0 - 1 + c;
        // outside the image: below every candidate (candidates have P > 0)
        ps[r][c] = (x >= 0 && x < W && y >= 0 && y < H) ? prob[(long long)y * W + x] : -1.0f;
    }
    __syncthreads();
    const int tx = threadIdx.x % kTW, ty = threadIdx.x / kTW;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= W || y >= H) return;
    const long long p = (long long)y * W + x;
    const float P = ps[ty + 1][tx + 1];
    bool is_max = P > 0.0f;
    #pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
        #pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            if (dy == 0 && dx == 0) continue;
            const float Q = ps[ty + 1 + dy][tx + 1 + dx];
            const bool earlier = dy < 0 || (dy == 0 && dx < 0);  // lower raster index
            if (Q > P || (Q == P && earlier)) is_max = false;
        }
    int slot = -1;
    if (is_max && uniform[p] < P) {
        const float d = depth[p];
        if (d > lod.near_z) {
            // the pixel centre at its depth, camera frame, then world frame
            const float xc[3] = {((x + 0.5f - cam.cx) / cam.fx) * d, ((y + 0.5f - cam.cy) / cam.fy) * d, d};
            const float dist = sqrtf(xc[0] * xc[0] + xc[1] * xc[1] + xc[2] * xc[2]);
            int l = -1;
            for (int k = 0; k < lod.levels; ++k)
                if (l < 0 && dist < lod.max_dist[k]) l = k;
            if (l >= 0) {
                const float e[3] = {xc[0] - cam.t[0], xc[1] - cam.t[1], xc[2] - cam.t[2]};
                int idx[3];
                bool ok = true;
                #pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float xw = cam.R[i] * e[0] + cam.R[3 + i] * e[1] + cam.R[6 + i] * e[2];
                    const float f = floorf(xw / lod.voxel[l]);
                    ok = ok && f >= -(float)kIdxBias && f < (float)kIdxBias;
                    idx[i] = ok ? (int)f : 0;
                }
                if (ok) {
                    const unsigned long long key = voxel_key(l, idx[0], idx[1], idx[2]);
                    const unsigned long long h = mix64(key);
                    for (long long pr = 0; pr < cap; ++pr) {
                        const long long s = (long long)((h + (unsigned long long)pr) & (unsigned long long)(cap - 1));
                        const unsigned long long old = atomicCAS(&keys[s], kEmpty, key);
                        if (old == kEmpty || old == key) {
                            slot = (int)s;
                            break;
                        }
                    }
                    if (slot < 0) {
                        if (status) atomicOr(status, 1 << GS_ERR_CAPACITY);
                    } else {
                        atomicMin(&owner[slot], (int)p);
                    }
                }
            }
        }
    }
    cand[p] = slot;
    if (selected) selected[p] = slot >= 0 ? 1 : 0;
}

__device__ __forceinline__ bool owns_new(const int *cand, const int *owner, long long npx, long long i) {
    if (i >= npx) return false;
    const int s = cand[i];
    return s >= 0 && owner[s] == (int)i;
}

constexpr int kPx = 4 * kThreads;  // pixels per counting / emitting block, four consecutive per thread

template <typename T>
__device__ __forceinline__ T block_sum(T v, T *red) {
    #pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    T t = 0;
    #pragma unroll
    for (int i = 0; i < kThreads / 32; ++i) t += red[i];
    return t;
}

__global__ void __launch_bounds__(kThreads) k_init_count(const int *__restrict__ cand, const int *__restrict__ owner,
                                                         long long npx, int *__restrict__ bsum,
                                                         const long long *__restrict__ count,
                                                         long long *__restrict__ base) {
    __shared__ int red[kThreads / 32];
    const long long i0 = (long long)blockIdx.x * kPx + 4 * threadIdx.x;
    int c = 0;
    #pragma unroll
    for (int j = 0; j < 4; ++j) c += owns_new(cand, owner, npx, i0 + j);
    c = block_sum(c, red);
    if (threadIdx.x == 0) {
        bsum[blockIdx.x] = c;
        if (blockIdx.x == 0) *base = *count;  // the anchors already in use
    }
}

__global__ void __launch_bounds__(kThreads) k_init_emit(const int *__restrict__ cand, int *__restrict__ owner,
                                                        const unsigned long long *__restrict__ keys,
                                                        int *__restrict__ ids, long long npx,
                                                        const int *__restrict__ bsum, const long long *__restrict__ base,
                                                        const __grid_constant__ InitLod lod, float *__restrict__ pos,
                                                        int *__restrict__ level, int *__restrict__ pixel,
                                                        long long ld, long long *__restrict__ count,
                                                        int *__restrict__ status) {
    __shared__ long long red[kThreads / 32];
    __shared__ int wsum[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the new anchors of all earlier blocks
    long long before = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += kThreads) before += bsum[b];
    before = block_sum(before, red);
    // only a voxel's owner settles its slot, so the others' tests are unaffected
    const long long i0 = (long long)blockIdx.x * kPx + 4 * threadIdx.x;
    bool f[4];
    int c = 0;
    #pragma unroll
    for (int j = 0; j < 4; ++j) {
        f[j] = owns_new(cand, owner, npx, i0 + j);
        c += f[j];
    }
    // exclusive scan of the per-thread counts over the block
    int incl = c;
    #pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int woff = 0, total = 0;
    #pragma unroll
    for (int k = 0; k < kThreads / 32; ++k) {
        woff += k < warp ? wsum[k] : 0;
        total += wsum[k];
    }
    const long long b0 = *base;
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *count = b0 + before + total;
    long long id = b0 + before + woff + incl - c;
    #pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (!f[j]) continue;
        const long long i = i0 + j;
        const int s = cand[i];
        const unsigned long long key = keys[s];
        const int l = (int)(key >> 60);
        const int ix = (int)((key >> 40) & 0xfffffu) - kIdxBias, iy = (int)((key >> 20) & 0xfffffu) - kIdxBias,
                  iz = (int)(key & 0xfffffu) - kIdxBias;
        if (id < ld) {
            const float e = lod.voxel[l];
            pos[id] = (float)ix * e;
            pos[ld + id] = (float)iy * e;
            pos[2 * ld + id] = (float)iz * e;
            level[id] = l;
            pixel[id] = (int)i;
            ids[s] = (int)id;
        } else {
            ids[s] = -1;
            if (status) atomicOr(status, 1 << GS_ERR_CAPACITY);
        }
        owner[s] = -1;
        ++id;
    }
}

__global__ void k_voxel_lookup(const unsigned long long *__restrict__ keys, const int *__restrict__ ids, long long cap,
                               const int *__restrict__ vox, long long n, long long ld, int *__restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = vox[i], ix = vox[ld + i], iy = vox[2 * ld + i], iz = vox[3 * ld + i];
    int r = -1;
    if (l >= 0 && l < GS_INIT_MAX_LEVELS && idx_in_range(ix) && idx_in_range(iy) && idx_in_range(iz)) {
        const unsigned long long key = voxel_key(l, ix, iy, iz), h = mix64(key);
        for (long long pr = 0; pr < cap; ++pr) {
            const long long s = (long long)((h + (unsigned long long)pr) & (unsigned long long)(cap - 1));
            const unsigned long long k = keys[s];
            if (k == key) {
                r = ids[s];
                break;
            }
            if (k == kEmpty) break;
        }
    }
    out[i] = r;
}

__global__ void k_voxel_reset(unsigned long long *__restrict__ keys, int *__restrict__ ids, int *__restrict__ owner,
                              long long cap) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += (long long)gridDim.x * blockDim.x) {
        keys[i] = kEmpty;
        ids[i] = -1;
        owner[i] = INT_MAX;
    }
}

struct InitWs {
    unsigned *minmax;
    long long *base;
    int *cand, *bsum;
};

InitWs carve(void *ws, int W, int H) {
    const size_t npx = (size_t)W * H;
    unsigned char *b = (unsigned char *)ws;
    InitWs w;
    w.minmax = (unsigned *)b;
    w.base = (long long *)(b + 64);
    w.cand = (int *)(b + 256);
    w.bsum = (int *)(b + 256 + align_up(sizeof(int) * npx, 256));
    return w;
}

}  // namespace

size_t init_workspace_bytes(int W, int H) {
    const size_t npx = (size_t)W * H, nb = (npx + kPx - 1) / kPx;
    return 256 + align_up(sizeof(int) * npx, 256) + align_up(sizeof(int) * nb, 256);
}

cudaError_t launch_init_probability(const float *img, const float *depth, const float *img_r, const float *depth_r,
                                    int W, int H, const InitBlur &bw, float lambda, float *prob, void *ws,
                                    cudaStream_t s) {
    InitWs w = carve(ws, W, H);
    const int nimg = img_r ? 2 : 1;
    cudaError_t e = cudaMemsetAsync(w.minmax, 0, 4 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const dim3 mgrid((unsigned)std::min(H, 592), (unsigned)nimg);
    k_init_grad_minmax<<<mgrid, kThreads, 0, s>>>(depth, depth_r, W, H, w.minmax);
    const dim3 grid((unsigned)ceil_div(W, kPT), (unsigned)ceil_div(H, kPH));
    if (bw.r1 == 3 && bw.r2 == 5)
        k_init_prob<3, 5><<<grid, kThreads, 0, s>>>(img, depth, img_r, depth_r, W, H, bw, w.minmax, lambda, prob);
    else
        k_init_prob<0, 0><<<grid, kThreads, 0, s>>>(img, depth, img_r, depth_r, W, H, bw, w.minmax, lambda, prob);
    return cudaGetLastError();
}

cudaError_t launch_init_insert(const float *prob, const float *uniform, const float *depth, int W, int H,
                               const InitCam &cam, const InitLod &lod, unsigned long long *keys, int *ids, int *owner,
                               long long cap, float *pos, int *level, int *pixel, long long *count, long long ld,
                               uint8_t *selected, int *status, void *ws, cudaStream_t s) {
    InitWs w = carve(ws, W, H);
    const long long npx = (long long)W * H;
    const int nb = (int)ceil_div(npx, (long long)kPx);
    const dim3 grid((unsigned)ceil_div(W, kTW), (unsigned)ceil_div(H, kTH));
    k_init_select<<<grid, kThreads, 0, s>>>(prob, uniform, depth, W, H, cam, lod, keys, owner, cap, w.cand, selected,
                                            status);
    k_init_count<<<nb, kThreads, 0, s>>>(w.cand, owner, npx, w.bsum, count, w.base);
    k_init_emit<<<nb, kThreads, 0, s>>>(w.cand, owner, keys, ids, npx, w.bsum, w.base, lod, pos, level, pixel, ld,
                                        count, status);
    return cudaGetLastError();
}

cudaError_t launch_voxel_lookup(const unsigned long long *keys, const int *ids, long long cap, const int *vox,
                                long long n, long long ld, int *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_voxel_lookup<<<(unsigned)ceil_div(n, 256ll), 256, 0, s>>>(keys, ids, cap, vox, n, ld, out);
    return cudaGetLastError();
}

cudaError_t launch_voxel_reset(unsigned long long *keys, int *ids, int *owner, long long cap, cudaStream_t s) {
    const long long blocks = std::min<long long>(ceil_div(cap, 256ll), 4096ll);
    k_voxel_reset<<<(unsigned)blocks, 256, 0, s>>>(keys, ids, owner, cap);
    return cudaGetLastError();
}

}  // namespace gs
