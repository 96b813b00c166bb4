// init.cu -- probabilistic initialisation of new anchors at a keyframe
// (Sec. 3.3.1) and the voxel hash of the dynamic map expansion (Supp. B).
//
// k_init_saliency: 32x8 pixel tiles.  The channel mean Y of the tile and a
// halo of the larger blur radius is staged in shared memory, blurred along
// rows by both Gaussians in one pass, then along columns; the DoG and the
// central-difference depth gradient are written as planes and the gradient's
// minimum and maximum are reduced per block into two atomics (non-negative
// FP32 bit patterns order like unsigned integers; the minimum is kept as the
// maximum of the complement so that both words start at zero).  One launch
// covers the keyframe and, when given, the rendered pair (blockIdx.z).
// k_init_combine: P, and P_kf = max(P - P^, 0).
// k_init_select: 3x3 non-maximum suppression from a staged tile, the draw,
// the unprojection, the level and voxel key, and the insertion into the
// table (64-bit compare-and-swap, linear probing bounded by the capacity);
// each slot of a new voxel keeps its lowest claiming pixel (atomicMin).
// k_init_count / k_init_scan / k_init_emit: the pixels that own a new voxel
// are numbered in raster order (block counts, one scan, warp-ballot ranks)
// and write the anchor records; their slots are then settled.
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

__global__ void __launch_bounds__(kThreads) k_init_saliency(const float *__restrict__ img,
                                                            const float *__restrict__ depth,
                                                            const float *__restrict__ img_r,
                                                            const float *__restrict__ depth_r, int W, int H,
                                                            InitBlur bw, float *__restrict__ dog,
                                                            float *__restrict__ grad, unsigned *__restrict__ minmax) {
    __shared__ float ys[kTH + 2 * kR][kTW + 2 * kR];
    __shared__ float hb[2][kTH + 2 * kR][kTW];
    __shared__ unsigned red[2][kThreads / 32];
    const int z = blockIdx.z;
    const float *I = z ? img_r : img;
    const float *D = z ? depth_r : depth;
    const long long npx = (long long)W * H;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH, R = bw.R;
    const int rows = kTH + 2 * R, cols = kTW + 2 * R;
    // channel mean of the tile and its halo, edges replicated
    for (int i = threadIdx.x; i < rows * cols; i += kThreads) {
        const int r = i / cols, c = i % cols;
        const int y = min(max(y0 - R + r, 0), H - 1), x = min(max(x0 - R + c, 0), W - 1);
        const long long p = (long long)y * W + x;
        ys[r][c] = (I[p] + I[npx + p] + I[2 * npx + p]) / 3.0f;
    }
    __syncthreads();
    // rows: both Gaussians
    for (int i = threadIdx.x; i < rows * kTW; i += kThreads) {
        const int r = i / kTW, c = i % kTW + R;
        float a = bw.w1[0] * ys[r][c], b = bw.w2[0] * ys[r][c];
        for (int k = 1; k <= bw.r1; ++k) a += bw.w1[k] * (ys[r][c - k] + ys[r][c + k]);
        for (int k = 1; k <= bw.r2; ++k) b += bw.w2[k] * (ys[r][c - k] + ys[r][c + k]);
        hb[0][r][c - R] = a;
        hb[1][r][c - R] = b;
    }
    __syncthreads();
    const int tx = threadIdx.x % kTW, ty = threadIdx.x / kTW;
    const int x = x0 + tx, y = y0 + ty;
    const bool in = x < W && y < H;
    unsigned gbits = 0u;
    if (in) {
        const int r = ty + R;
        float a = bw.w1[0] * hb[0][r][tx], b = bw.w2[0] * hb[1][r][tx];
        for (int k = 1; k <= bw.r1; ++k) a += bw.w1[k] * (hb[0][r - k][tx] + hb[0][r + k][tx]);
        for (int k = 1; k <= bw.r2; ++k) b += bw.w2[k] * (hb[1][r - k][tx] + hb[1][r + k][tx]);
        const long long p = (long long)y * W + x;
        dog[z * npx + p] = fminf(bw.scale * fabsf(a - b), 1.0f);
        const long long row = (long long)y * W;
        const float gx = (D[row + min(x + 1, W - 1)] - D[row + max(x - 1, 0)]) * 0.5f;
        const float gy = (D[(long long)min(y + 1, H - 1) * W + x] - D[(long long)max(y - 1, 0) * W + x]) * 0.5f;
        const float g = sqrtf(gx * gx + gy * gy);
        grad[z * npx + p] = g;
        gbits = __float_as_uint(g);
    }
    // block minimum (as the maximum of the complement) and maximum of the gradient
    unsigned lo = in ? ~gbits : 0u, hi = gbits;
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

__device__ __forceinline__ float init_p(const float *dog, const float *grad, const unsigned *minmax, int z,
                                        long long npx, long long i, float lambda) {
    const float lo = __uint_as_float(~minmax[2 * z]), hi = __uint_as_float(minmax[2 * z + 1]);
    const float gn = hi > lo ? (grad[z * npx + i] - lo) / (hi - lo) : 0.0f;
    return fminf(lambda * dog[z * npx + i] + (1.0f - lambda) * gn, 1.0f);
}

__global__ void k_init_combine(const float *__restrict__ dog, const float *__restrict__ grad,
                               const unsigned *__restrict__ minmax, long long npx, int rendered, float lambda,
                               float *__restrict__ prob) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npx) return;
    float p = init_p(dog, grad, minmax, 0, npx, i, lambda);
    if (rendered) p = fmaxf(p - init_p(dog, grad, minmax, 1, npx, i, lambda), 0.0f);
    prob[i] = p;
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

__global__ void __launch_bounds__(kThreads) k_init_count(const int *__restrict__ cand, const int *__restrict__ owner,
                                                         long long npx, int *__restrict__ bsum) {
    const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
    const int c = __syncthreads_count(owns_new(cand, owner, npx, i));
    if (threadIdx.x == 0) bsum[blockIdx.x] = c;
}

// Exclusive scan of the block counts in one block; count (the anchors in
// use) is the base and receives the new total.
__global__ void __launch_bounds__(1024) k_init_scan(const int *__restrict__ bsum, int nb, long long *__restrict__ boff,
                                                    long long *__restrict__ count) {
    __shared__ long long wsum[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = *count;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const long long v = i < nb ? bsum[i] : 0;
        long long s = v;
        #pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += u;
        }
        if (lane == 31) wsum[warp] = s;
        __syncthreads();
        if (warp == 0) {
            long long w = wsum[lane];
            #pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const long long u = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += u;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const long long incl = s + (warp ? wsum[warp - 1] : 0);
        if (i < nb) boff[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = carry;
}

__global__ void __launch_bounds__(kThreads) k_init_emit(const int *__restrict__ cand, int *__restrict__ owner,
                                                        const unsigned long long *__restrict__ keys,
                                                        int *__restrict__ ids, long long npx,
                                                        const long long *__restrict__ boff,
                                                        const __grid_constant__ InitLod lod,
                                                        float *__restrict__ pos, int *__restrict__ level,
                                                        int *__restrict__ pixel, long long ld,
                                                        int *__restrict__ status) {
    __shared__ int wcount[kThreads / 32];
    const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
    // only a voxel's owner settles its slot, so the others' tests are unaffected
    const bool f = owns_new(cand, owner, npx, i);
    const unsigned ballot = __ballot_sync(0xffffffffu, f);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) wcount[warp] = __popc(ballot);
    __syncthreads();
    if (!f) return;
    int woff = 0;
    for (int k = 0; k < warp; ++k) woff += wcount[k];
    const long long id = boff[blockIdx.x] + woff + __popc(ballot & ((1u << lane) - 1u));
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
    float *dog, *grad;
    int *cand, *bsum;
    long long *boff;
};

InitWs carve(void *ws, int W, int H) {
    const size_t npx = (size_t)W * H, nb = (npx + kThreads - 1) / kThreads;
    unsigned char *b = (unsigned char *)ws;
    InitWs w;
    size_t off = 0;
    w.minmax = (unsigned *)(b + off);
    off += 256;
    w.dog = (float *)(b + off);
    off += align_up(sizeof(float) * 2 * npx, 256);
    w.grad = (float *)(b + off);
    off += align_up(sizeof(float) * 2 * npx, 256);
    w.cand = (int *)(b + off);
    off += align_up(sizeof(int) * npx, 256);
    w.bsum = (int *)(b + off);
    off += align_up(sizeof(int) * nb, 256);
    w.boff = (long long *)(b + off);
    return w;
}

}  // namespace

size_t init_workspace_bytes(int W, int H) {
    const size_t npx = (size_t)W * H, nb = (npx + kThreads - 1) / kThreads;
    return 256 + 2 * align_up(sizeof(float) * 2 * npx, 256) + align_up(sizeof(int) * npx, 256) +
           align_up(sizeof(int) * nb, 256) + align_up(sizeof(long long) * nb, 256);
}

cudaError_t launch_init_probability(const float *img, const float *depth, const float *img_r, const float *depth_r,
                                    int W, int H, const InitBlur &bw, float lambda, float *prob, void *ws,
                                    cudaStream_t s) {
    InitWs w = carve(ws, W, H);
    const int nimg = img_r ? 2 : 1;
    cudaError_t e = cudaMemsetAsync(w.minmax, 0, 4 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)ceil_div(W, kTW), (unsigned)ceil_div(H, kTH), (unsigned)nimg);
    k_init_saliency<<<grid, kThreads, 0, s>>>(img, depth, img_r, depth_r, W, H, bw, w.dog, w.grad, w.minmax);
    const long long npx = (long long)W * H;
    k_init_combine<<<(unsigned)ceil_div(npx, 256ll), 256, 0, s>>>(w.dog, w.grad, w.minmax, npx, nimg == 2, lambda,
                                                                    prob);
    return cudaGetLastError();
}

cudaError_t launch_init_insert(const float *prob, const float *uniform, const float *depth, int W, int H,
                               const InitCam &cam, const InitLod &lod, unsigned long long *keys, int *ids, int *owner,
                               long long cap, float *pos, int *level, int *pixel, long long *count, long long ld,
                               uint8_t *selected, int *status, void *ws, cudaStream_t s) {
    InitWs w = carve(ws, W, H);
    const long long npx = (long long)W * H;
    const int nb = (int)ceil_div(npx, (long long)kThreads);
    const dim3 grid((unsigned)ceil_div(W, kTW), (unsigned)ceil_div(H, kTH));
    k_init_select<<<grid, kThreads, 0, s>>>(prob, uniform, depth, W, H, cam, lod, keys, owner, cap, w.cand, selected,
                                            status);
    k_init_count<<<nb, kThreads, 0, s>>>(w.cand, owner, npx, w.bsum);
    k_init_scan<<<1, 1024, 0, s>>>(w.bsum, nb, w.boff, count);
    k_init_emit<<<nb, kThreads, 0, s>>>(w.cand, owner, keys, ids, npx, w.boff, lod, pos, level, pixel, ld, status);
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
