// actions.cu -- densify / prune actions on the explicit Gaussians: the
// decisions of the lifecycle criterion (Sec. 3.3.2, Supp. E) or of the learned
// predictor turned into a new parameter set.  Gaussian i emits, in source
// order, 0 rows when pruned, 1 when kept, 2 when densified: a clone (itself
// plus an identical copy) or, when its largest log-scale exceeds a threshold,
// a split into two samples mu + R S xi of its own N(mu, Sigma) with the scales
// divided by a factor (the paper spawns anchors; clone / split is the reading
// for explicit Gaussians).  Adam moments follow the survivor; clones and split
// children start at zero.
//
// Three launches: per-block emission counts, one block scanning the block
// counts into row offsets (and the total into n_out), and the scatter, whose
// grid runs over (source block, group of 8 planes) so that each CTA streams
// eight planes of three arrays (parameters, m, v) and recomputes its block's
// exclusive scan from the decision bytes.  Pure copy traffic: HBM bound.
#include "gs_internal.cuh"
#include "gs_kernels.h"

namespace gs {

constexpr int kActThreads = 256;  // sources per block
constexpr int kActPlanes = 8;     // planes per scatter CTA
constexpr int kScanThreads = 1024;

__device__ __forceinline__ int emit_count(const uint8_t *__restrict__ dens, const uint8_t *__restrict__ prune,
                                          long long i, long long n) {
    if (i >= n || prune[i]) return 0;
    return dens[i] ? 2 : 1;
}

__global__ void __launch_bounds__(kActThreads) k_act_count(const uint8_t *__restrict__ dens,
                                                           const uint8_t *__restrict__ prune, long long n,
                                                           long long *__restrict__ block_sum) {
    const long long i = (long long)blockIdx.x * kActThreads + threadIdx.x;
    const int c = emit_count(dens, prune, i, n);
    const int ones = __syncthreads_count(c >= 1), twos = __syncthreads_count(c == 2);
    if (threadIdx.x == 0) block_sum[blockIdx.x] = ones + twos;
}

// Exclusive scan of nb block counts in one CTA; total -> *n_out, capacity flag.
__global__ void __launch_bounds__(kScanThreads) k_act_scan(long long *__restrict__ block_sum, long long nb,
                                                           long long cap, long long *__restrict__ n_out,
                                                           int *__restrict__ status) {
    __shared__ long long warp_tot[kScanThreads / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const long long per = ceil_div(nb, (long long)kScanThreads);
    const long long lo = min(nb, t * per), hi = min(nb, lo + per);
    long long local = 0;
    for (long long b = lo; b < hi; ++b) local += block_sum[b];
    long long incl = local;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        long long w = warp_tot[lane], wi = w;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        warp_tot[lane] = wi - w;  // exclusive warp offsets
    }
    __syncthreads();
    long long run = warp_tot[warp] + incl - local;
    for (long long b = lo; b < hi; ++b) {
        const long long c = block_sum[b];
        block_sum[b] = run;
        run += c;
    }
    if (t == kScanThreads - 1) {
        *n_out = run;
        if (run > cap && status) atomicOr(status, 1 << GS_ERR_CAPACITY);
    }
}

struct ActArrays {
    const float *src, *src_m, *src_v;
    float *dst, *dst_m, *dst_v;
    long long ld, dld, cap;
};

__global__ void __launch_bounds__(kActThreads) k_act_scatter(ActArrays a, const uint8_t *__restrict__ dens,
                                                             const uint8_t *__restrict__ prune,
                                                             const float *__restrict__ noise, long long n, int planes,
                                                             float split_log_scale, float log_split_factor,
                                                             const long long *__restrict__ block_off) {
    __shared__ int warp_tot[kActThreads / 32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const long long i = (long long)blockIdx.x * kActThreads + t;
    const int c = emit_count(dens, prune, i, n);
    int incl = c;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += warp_tot[w];
    if (c == 0) return;
    const long long o = block_off[blockIdx.x] + before + incl - c;
    const int p0 = blockIdx.y * kActPlanes, p1 = min(planes, p0 + kActPlanes);
    const float *S = a.src;
    bool split = false;
    float d0[3] = {0.f, 0.f, 0.f}, d1[3] = {0.f, 0.f, 0.f};
    if (c == 2 && p0 < 6) {
        split = fmaxf(S[3 * a.ld + i], fmaxf(S[4 * a.ld + i], S[5 * a.ld + i])) > split_log_scale;
        if (split && p0 < 3) {  // child offsets R S xi_j
            float qw = S[6 * a.ld + i], qx = S[7 * a.ld + i], qy = S[8 * a.ld + i], qz = S[9 * a.ld + i];
            const float nq = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
            float R[9];
            quat_rotation(qw / nq, qx / nq, qy / nq, qz / nq, R);
            float sx[3];
            #pragma unroll
            for (int k = 0; k < 3; ++k) sx[k] = expf(S[(3 + k) * a.ld + i]);
            #pragma unroll
            for (int r = 0; r < 3; ++r)
                #pragma unroll
                for (int k = 0; k < 3; ++k) {
                    d0[r] += R[3 * r + k] * sx[k] * noise[(long long)k * a.ld + i];
                    d1[r] += R[3 * r + k] * sx[k] * noise[(long long)(3 + k) * a.ld + i];
                }
        }
    } else if (c == 2) {
        split = fmaxf(S[3 * a.ld + i], fmaxf(S[4 * a.ld + i], S[5 * a.ld + i])) > split_log_scale;
    }
    const bool w0 = o < a.cap, w1 = c == 2 && o + 1 < a.cap;
    for (int p = p0; p < p1; ++p) {
        const float x = S[(long long)p * a.ld + i];
        float x0 = x, x1 = x;
        if (split && p < 3) { x0 = x + d0[p]; x1 = x + d1[p]; }
        if (split && p >= 3 && p < 6) { x0 = x - log_split_factor; x1 = x0; }
        float *D = a.dst + (long long)p * a.dld;
        if (w0) D[o] = x0;
        if (w1) D[o + 1] = x1;
        if (a.dst_m) {
            const float m = split ? 0.0f : a.src_m[(long long)p * a.ld + i];
            const float v = split ? 0.0f : a.src_v[(long long)p * a.ld + i];
            if (w0) { a.dst_m[(long long)p * a.dld + o] = m; a.dst_v[(long long)p * a.dld + o] = v; }
            if (w1) { a.dst_m[(long long)p * a.dld + o + 1] = 0.0f; a.dst_v[(long long)p * a.dld + o + 1] = 0.0f; }
        }
    }
}

size_t actions_workspace_bytes(long long n) {
    return align_up(sizeof(long long) * (size_t)ceil_div(n > 0 ? n : 1, kActThreads), 256);
}

cudaError_t launch_actions(const float *src, const float *src_m, const float *src_v, long long n, long long ld,
                           int planes, const uint8_t *dens, const uint8_t *prune, const float *noise,
                           float split_log_scale, float log_split_factor, float *dst, float *dst_m, float *dst_v,
                           long long dld, long long *n_out, int *status, void *ws, cudaStream_t s) {
    long long *block = (long long *)ws;
    if (n <= 0) return cudaMemsetAsync(n_out, 0, sizeof(long long), s);
    const long long nb = ceil_div(n, (long long)kActThreads);
    k_act_count<<<(unsigned)nb, kActThreads, 0, s>>>(dens, prune, n, block);
    k_act_scan<<<1, kScanThreads, 0, s>>>(block, nb, dld, n_out, status);
    ActArrays a{src, src_m, src_v, dst, dst_m, dst_v, ld, dld, dld};
    const dim3 grid((unsigned)nb, (unsigned)ceil_div(planes, kActPlanes));
    k_act_scatter<<<grid, kActThreads, 0, s>>>(a, dens, prune, noise, n, planes, split_log_scale, log_split_factor,
                                               block);
    return cudaGetLastError();
}

}  // namespace gs
