// prune.cu -- chunk scores and global densify / prune decisions from the
// per-Gaussian lifecycle accumulators (Supp. E.1, E.2; Sec. 3.3.2):
//   S_d = kappa / |V_c|, densify |= S_d > tau_d;
//   L = log(1 + gamma), S_p = (L - min L) / (max L - min L) over the active
//   Gaussians (|Omega| > 0), 0 elsewhere or when max = min;
//   prune_max = max(prune_max, S_p), prune = prune_max > tau_p.
#include "gs_internal.cuh"
#include "gs_kernels.h"

namespace gs {

// L >= 0, so the bit patterns order like the values; the minimum is kept as
// the maximum of (0x7fffffff - bits) so one zero-fill initialises both words.
__global__ void __launch_bounds__(256) k_prune_minmax(const float *__restrict__ acc, long long ld, long long n,
                                                       unsigned int *__restrict__ mm) {
    unsigned int mx = 0, mn = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (acc[0 * ld + i] > 0.0f) {
            const unsigned int b = __float_as_uint(log1pf(acc[2 * ld + i]));
            mx = max(mx, b);
            mn = max(mn, 0x7fffffffu - b);
        }
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = max(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&mm[0], mx);
        atomicMax(&mm[1], mn);
    }
}

__global__ void __launch_bounds__(256) k_prune_apply(const float *__restrict__ acc, long long ld, long long n,
                                                      float inv_views, float tau_d, float tau_p,
                                                      const unsigned int *__restrict__ mm, float *__restrict__ S_d,
                                                      float *__restrict__ S_p, float *__restrict__ prune_max,
                                                      unsigned char *__restrict__ densify,
                                                      unsigned char *__restrict__ prune, float n_views) {
    const float lmax = __uint_as_float(mm[0]);
    const float lmin = __uint_as_float(0x7fffffffu - mm[1]);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float sd = acc[1 * ld + i] / n_views;
        S_d[i] = sd;
        if (sd > tau_d) densify[i] = 1;
        float sp = 0.0f;
        if (acc[0 * ld + i] > 0.0f && lmax > lmin) sp = (log1pf(acc[2 * ld + i]) - lmin) / (lmax - lmin);
        S_p[i] = sp;
        const float pm = fmaxf(prune_max[i], sp);
        prune_max[i] = pm;
        prune[i] = pm > tau_p ? 1 : 0;
    }
    (void)inv_views;
}

size_t prune_workspace_bytes(long long) { return 256; }

void launch_prune(const float *acc, long long ld, long long n, int n_views, float tau_d, float tau_p, float *S_d,
                  float *S_p, float *prune_max, unsigned char *densify, unsigned char *prune, void *ws,
                  cudaStream_t s) {
    if (n <= 0) return;
    unsigned int *mm = (unsigned int *)ws;
    cudaMemsetAsync(mm, 0, 2 * sizeof(unsigned int), s);
    const int blocks = (int)std::min<long long>(ceil_div(n, 256), 148 * 8);
    k_prune_minmax<<<blocks, 256, 0, s>>>(acc, ld, n, mm);
    k_prune_apply<<<blocks, 256, 0, s>>>(acc, ld, n, 1.0f / n_views, tau_d, tau_p, mm, S_d, S_p, prune_max, densify,
                                         prune, (float)n_views);
}

}  // namespace gs
