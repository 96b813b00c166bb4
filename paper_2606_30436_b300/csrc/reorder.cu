// reorder.cu -- spatial order of the Gaussians' rows.
//
// Not a step of the paper's method but a layout of its parameter planes: the
// rows are put in the Morton (Z-)order of the Gaussians' means, so that the
// Gaussians a view sees sit near each other in every plane.  The projection,
// its backward and the compositing then read whole 32-byte sectors of visible
// Gaussians instead of sectors of which one visible Gaussian uses 4 bytes.
//
// Order (exactly, so that a host program reproduces it bit for bit):
//   box     lo_a = min over the means of axis a, hi_a = max (exact)
//   scale   1024 / max_a (hi_a - lo_a) in FP32 (0 when that extent is 0 or not finite)
//   cell    q_a = 1023 if t >= 1023, else (int) t if t > 0, else 0, with t = (m_a - lo_a) * scale
//           in FP32 (one rounding per operation)
//   code    bit b of q_x at bit 3b, of q_y at 3b + 1, of q_z at 3b + 2 (30 bits)
//   rows    sorted stably by code: equal codes keep their order
// Four steps: the box (a reduction with ordered-integer atomics), the codes,
// the stable LSD radix sort of the binning (four passes over 30 bits), and per
// plane set a gather into scratch followed by one copy back, so every buffer
// keeps its address (captured graphs stay valid).
#include <cfloat>

#include "gs_internal.cuh"
#include "gs_kernels.h"

namespace gs {

constexpr int kReorderThreads = 256;
constexpr int kReorderBlocks = 148 * 4;
constexpr int kMortonBits = 10;  // per axis

// float -> unsigned with the same order (negative floats reversed below the positive ones)
__device__ __forceinline__ unsigned ordered_bits(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_ordered_bits(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// the 10 low bits of x moved to bits 0, 3, 6, ..., 27 (the usual shift-and-mask spreading)
__device__ __forceinline__ uint32_t spread3(uint32_t x) {
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void k_reorder_init(unsigned *__restrict__ box, int *__restrict__ count, long long n) {
    if (threadIdx.x < 3) box[threadIdx.x] = 0xffffffffu;
    else if (threadIdx.x < 6) box[threadIdx.x] = 0u;
    else if (threadIdx.x == 6) *count = (int)n;
}

__global__ void __launch_bounds__(kReorderThreads) k_reorder_box(const float *__restrict__ P, long long n,
                                                                 long long ld, unsigned *__restrict__ box) {
    unsigned lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        #pragma unroll
        for (int a = 0; a < 3; ++a) {
            const unsigned k = ordered_bits(P[a * ld + i]);
            lo[a] = min(lo[a], k);
            hi[a] = max(hi[a], k);
        }
    }
    #pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = __reduce_min_sync(0xffffffffu, lo[a]);
        hi[a] = __reduce_max_sync(0xffffffffu, hi[a]);
    }
    if ((threadIdx.x & 31) == 0) {
        #pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(&box[a], lo[a]);
            atomicMax(&box[3 + a], hi[a]);
        }
    }
}

__global__ void __launch_bounds__(kReorderThreads) k_reorder_codes(const float *__restrict__ P, long long n,
                                                                   long long ld, const unsigned *__restrict__ box,
                                                                   uint32_t *__restrict__ key,
                                                                   uint32_t *__restrict__ val) {
    float lo[3], ext = 0.0f;
    #pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = from_ordered_bits(box[a]);
        ext = fmaxf(ext, __fsub_rn(from_ordered_bits(box[3 + a]), lo[a]));
    }
    const float scale = (ext > 0.0f && ext <= FLT_MAX) ? __fdiv_rn(1024.0f, ext) : 0.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        uint32_t code = 0;
        #pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float t = __fmul_rn(__fsub_rn(P[a * ld + i], lo[a]), scale);
            const int q = t >= (float)((1 << kMortonBits) - 1) ? (1 << kMortonBits) - 1 : (t > 0.0f ? (int)t : 0);
            code |= spread3((uint32_t)q) << a;
        }
        key[i] = code;
        val[i] = (uint32_t)i;
    }
}

// dst[p][i] = src[p][perm[i]] for the n rows, the padding rows [n, ld) copied as they are
__global__ void __launch_bounds__(kReorderThreads) k_reorder_gather(const float *__restrict__ src,
                                                                    float *__restrict__ dst, long long n, long long ld,
                                                                    const uint32_t *__restrict__ perm) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ld) return;
    const long long p = (long long)blockIdx.y * ld;
    dst[p + i] = src[p + (i < n ? (long long)perm[i] : i)];
}

struct ReorderWs {
    int *count;
    unsigned *box;
    uint32_t *k0, *v0, *k1, *v1, *perm;
    void *sort;
    float *scratch;
    size_t bytes;
};

static ReorderWs carve_reorder(void *base, long long n, long long ld, int max_planes) {
    ReorderWs w;
    size_t off = 0;
    char *b = (char *)base;
    auto take = [&](size_t bytes) {
        char *p = b ? b + off : nullptr;
        off = align_up(off + bytes, 256);
        return p;
    };
    w.count = (int *)take(sizeof(int));
    w.box = (unsigned *)take(6 * sizeof(unsigned));
    w.k0 = (uint32_t *)take(sizeof(uint32_t) * n);
    w.v0 = (uint32_t *)take(sizeof(uint32_t) * n);
    w.k1 = (uint32_t *)take(sizeof(uint32_t) * n);
    w.v1 = (uint32_t *)take(sizeof(uint32_t) * n);
    w.perm = (uint32_t *)take(sizeof(uint32_t) * n);
    w.sort = take(key_sort_scratch_bytes());
    w.scratch = (float *)take(sizeof(float) * (size_t)max_planes * (size_t)ld);
    w.bytes = off;
    return w;
}

size_t reorder_workspace_bytes(long long n, long long ld, int max_planes) {
    return carve_reorder(nullptr, n, ld, max_planes).bytes;
}

cudaError_t launch_reorder(float *P, long long n, long long ld, int planes, float *const *extra,
                           const int *extra_planes, int n_extra, int *perm, void *ws, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int maxp = planes;
    for (int e = 0; e < n_extra; ++e) maxp = max(maxp, extra_planes[e]);
    ReorderWs w = carve_reorder(ws, n, ld, maxp);
    uint32_t *order = perm ? (uint32_t *)perm : w.perm;
    k_reorder_init<<<1, 32, 0, s>>>(w.box, w.count, n);
    const int blocks = (int)min((long long)kReorderBlocks, ceil_div(n, (long long)kReorderThreads));
    k_reorder_box<<<blocks, kReorderThreads, 0, s>>>(P, n, ld, w.box);
    k_reorder_codes<<<blocks, kReorderThreads, 0, s>>>(P, n, ld, w.box, w.k0, w.v0);
    launch_key_sort(w.k0, w.v0, w.k1, w.v1, w.count, n, 3 * kMortonBits, w.sort, order, s);
    // every set gathered, then copied back; the parameters last (their means gave the order)
    for (int e = 0; e <= n_extra; ++e) {
        float *set = e < n_extra ? extra[e] : P;
        const int np = e < n_extra ? extra_planes[e] : planes;
        const dim3 grid((unsigned)ceil_div(ld, (long long)kReorderThreads), (unsigned)np);
        k_reorder_gather<<<grid, kReorderThreads, 0, s>>>(set, w.scratch, n, ld, order);
        const cudaError_t err = cudaMemcpyAsync(set, w.scratch, sizeof(float) * (size_t)np * (size_t)ld,
                                                cudaMemcpyDeviceToDevice, s);
        if (err != cudaSuccess) return err;
    }
    return cudaGetLastError();
}

}  // namespace gs
