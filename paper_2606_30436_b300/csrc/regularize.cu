// regularize.cu -- the geometric and isotropic terms of the mapping loss
// L_total = L_photo + lambda_g L_geo + lambda_iso L_iso (Sec. 3.2.3, Supp. D.4):
//   L_geo = mean over pixels of [D > 0] |D - D^| (rendered depth D^ against the
//           metric-depth prior D; 0 marks a pixel without a prior),
//   L_iso = mean over Gaussians of sum_k |s_k - mean(s)|, s = exp(log-scale).
// Both are streaming passes; their sums are reduced per CTA and then in a
// fixed order, so the scalar is deterministic.
#include <algorithm>

#include "gs_internal.cuh"
#include "gs_kernels.h"

namespace gs {

constexpr int kRegBlocks = 148 * 4;

__device__ __forceinline__ double block_sum_dbl(double v, double *sm) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sm[i];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(256) k_geo(const float *__restrict__ depth, const float *__restrict__ prior,
                                              long long npx, float gscale, float *__restrict__ dL,
                                              double *__restrict__ partials) {
    __shared__ double sm[8];
    double s = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npx;
         p += (long long)gridDim.x * blockDim.x) {
        const float pr = prior[p];
        float g = 0.0f;
        if (pr > 0.0f) {
            const float d = depth[p] - pr;
            s += fabsf(d);
            g = d > 0.0f ? gscale : (d < 0.0f ? -gscale : 0.0f);
        }
        if (dL) dL[p] = g;
    }
    const double t = block_sum_dbl(s, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(256) k_iso(const float *__restrict__ P, long long n, long long ld, float gscale,
                                              float *__restrict__ G, double *__restrict__ partials) {
    __shared__ double sm[8];
    double sum = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float s0 = expf(P[3 * ld + i]), s1 = expf(P[4 * ld + i]), s2 = expf(P[5 * ld + i]);
        const float m = (s0 + s1 + s2) * (1.0f / 3.0f);
        const float d0 = s0 - m, d1 = s1 - m, d2 = s2 - m;
        sum += (double)(fabsf(d0) + fabsf(d1) + fabsf(d2));
        if (G) {
            float gl[3] = {0.0f, 0.0f, 0.0f};
            iso_grad(P[3 * ld + i], P[4 * ld + i], P[5 * ld + i], gscale, gl);
            G[3 * ld + i] += gl[0];
            G[4 * ld + i] += gl[1];
            G[5 * ld + i] += gl[2];
        }
    }
    const double t = block_sum_dbl(sum, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(256) k_sum_final(const double *__restrict__ partials, int nb, double mul,
                                                    float *__restrict__ out) {
    __shared__ double sm[8];
    double a = 0.0;
    for (int i = threadIdx.x; i < nb; i += 256) a += partials[i];
    const double t = block_sum_dbl(a, sm);
    if (threadIdx.x == 0) *out = (float)(t * mul);
}

size_t reg_workspace_bytes() { return align_up(sizeof(double) * kRegBlocks, 256); }

cudaError_t launch_geo(const float *depth, const float *prior, long long npx, float weight, float *loss,
                       float *dL, void *ws, cudaStream_t s) {
    if (npx <= 0) return cudaSuccess;
    double *partials = (double *)ws;
    const int nb = (int)std::min<long long>(ceil_div(npx, 256), kRegBlocks);
    k_geo<<<nb, 256, 0, s>>>(depth, prior, npx, (float)(weight / (double)npx), dL, partials);
    k_sum_final<<<1, 256, 0, s>>>(partials, nb, weight / (double)npx, loss);
    return cudaGetLastError();
}

cudaError_t launch_iso(const float *P, long long n, long long ld, float weight, float *loss, float *G, void *ws,
                       cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    double *partials = (double *)ws;
    const int nb = (int)std::min<long long>(ceil_div(n, 256), kRegBlocks);
    k_iso<<<nb, 256, 0, s>>>(P, n, ld, (float)(weight / (double)n), G, partials);
    k_sum_final<<<1, 256, 0, s>>>(partials, nb, weight / (double)n, loss);
    return cudaGetLastError();
}

}  // namespace gs
