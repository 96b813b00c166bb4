// adam.cu -- Adam (Kingma & Ba) with bias correction over every parameter
// plane, dense: all Gaussians move every step, as with torch.optim.Adam.  The
// parameter, gradient and both moment buffers share the plane-major layout, so
// the update is one flat float4 stream (28 bytes of HBM traffic per parameter).
#include "gs_internal.cuh"
#include "gs_kernels.h"

namespace gs {

struct AdamLr { float lr[6]; };

// The square root and the division of the update take the SFU's approximations (relative
// errors of a few 2^-23): the IEEE-rounded forms cost more issue slots than the 28 bytes of
// traffic per element leave at HBM speed.
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ int lr_group(long long plane) {
    // means, log-scales, quaternion, opacity, SH degree 0, SH degree >= 1
    return plane < 3 ? 0 : plane < 6 ? 1 : plane < 10 ? 2 : plane == 10 ? 3 : plane < 14 ? 4 : 5;
}

__global__ void __launch_bounds__(256) k_adam(float4 *__restrict__ p, const float4 *__restrict__ g,
                                               float4 *__restrict__ m, float4 *__restrict__ v, long long ld4,
                                               long long total4, AdamLr lr, float b1, float b2, float inv_bc1,
                                               float inv_sqrt_bc2, float eps, const long long *__restrict__ step_dev) {
    griddep_wait();
    if (step_dev) {  // bias corrections from the device step counter (graph replay)
        __shared__ float s_bc[2];
        if (threadIdx.x == 0) {
            adam_bias_inv(b1, b2, *step_dev, s_bc[0], s_bc[1]);
        }
        __syncthreads();
        inv_bc1 = s_bc[0];
        inv_sqrt_bc2 = s_bc[1];
    }
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < total4; i0 += 2 * stride) {
        float4 gg[2], mm[2], vv[2], pp[2];
        #pragma unroll
        for (int u = 0; u < 2; ++u) {
            const long long i = i0 + u * stride;
            if (i < total4) { gg[u] = g[i]; mm[u] = m[i]; vv[u] = v[i]; pp[u] = p[i]; }
        }
        #pragma unroll
        for (int u = 0; u < 2; ++u) {
            const long long i = i0 + u * stride;
            if (i >= total4) continue;
            const float a = lr.lr[lr_group(i / ld4)];
#define GS_ADAM_LANE(c)                                                         \
    mm[u].c = b1 * mm[u].c + (1.0f - b1) * gg[u].c;                             \
    vv[u].c = b2 * vv[u].c + (1.0f - b2) * gg[u].c * gg[u].c;                   \
    pp[u].c -= __fdividef(a * (mm[u].c * inv_bc1), sqrt_approx(vv[u].c) * inv_sqrt_bc2 + eps);
            GS_ADAM_LANE(x) GS_ADAM_LANE(y) GS_ADAM_LANE(z) GS_ADAM_LANE(w)
#undef GS_ADAM_LANE
            m[i] = mm[u];
            v[i] = vv[u];
            p[i] = pp[u];
        }
    }
}

// The same update where the gradient rows of Gaussians no view sees were not written:
// rows4[c] holds the marks of the four Gaussians of float4 column c.  A thread takes one
// column through kAdamPlanes planes, so the marks are read once for those planes and an
// all-zero mark skips the gradient's loads.  part selects the rows: 0 all (unmarked ones
// with a zero gradient), 1 the marked rows only (scalar stores where a column is mixed), so
// that it may run beside k_adam_unseen, which writes the others.
constexpr int kAdamPlanes = 8;

__device__ __forceinline__ void store_lanes(float4 *base, long long i, const float4 &val, uint32_t own) {
    if (own == 0x01010101u) {
        base[i] = val;
    } else {
        float *f = reinterpret_cast<float *>(base + i);
        if (own & 0xffu) f[0] = val.x;
        if (own & 0xff00u) f[1] = val.y;
        if (own & 0xff0000u) f[2] = val.z;
        if (own & 0xff000000u) f[3] = val.w;
    }
}

__global__ void __launch_bounds__(256) k_adam_rows(float4 *__restrict__ p, const float4 *__restrict__ g,
                                                    float4 *__restrict__ m, float4 *__restrict__ v, long long ld4,
                                                    int planes, AdamLr lr, float b1, float b2, float inv_bc1,
                                                    float inv_sqrt_bc2, float eps,
                                                    const long long *__restrict__ step_dev,
                                                    const uint32_t *__restrict__ rows4, int part) {
    griddep_wait();
    if (step_dev) {
        __shared__ float s_bc[2];
        if (threadIdx.x == 0) {
            adam_bias_inv(b1, b2, *step_dev, s_bc[0], s_bc[1]);
        }
        __syncthreads();
        inv_bc1 = s_bc[0];
        inv_sqrt_bc2 = s_bc[1];
    }
    const long long chunks = (planes + kAdamPlanes - 1) / kAdamPlanes;
    const long long items = chunks * ld4;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const long long chunk = it / ld4, c4 = it - chunk * ld4;
        const uint32_t r = rows4[c4];                          // gradient marks
        const uint32_t own = part == 1 ? r : 0x01010101u;  // the lanes this call writes
        if (own == 0u) continue;
        const int q0 = (int)chunk * kAdamPlanes, q1 = min(planes, q0 + kAdamPlanes);
        for (int q = q0; q < q1; q += 2) {
            float4 gg[2], mm[2], vv[2], pp[2];
            #pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (q + u >= q1) continue;
                const long long i = (long long)(q + u) * ld4 + c4;
                mm[u] = m[i]; vv[u] = v[i]; pp[u] = p[i];
                gg[u] = r ? g[i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (r != 0x01010101u) {
                    gg[u].x = (r & 0xffu) ? gg[u].x : 0.0f;
                    gg[u].y = (r & 0xff00u) ? gg[u].y : 0.0f;
                    gg[u].z = (r & 0xff0000u) ? gg[u].z : 0.0f;
                    gg[u].w = (r & 0xff000000u) ? gg[u].w : 0.0f;
                }
            }
            #pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (q + u >= q1) continue;
                const long long i = (long long)(q + u) * ld4 + c4;
                const float a = lr.lr[lr_group(q + u)];
#define GS_ADAM_LANE(c)                                                         \
    mm[u].c = b1 * mm[u].c + (1.0f - b1) * gg[u].c;                             \
    vv[u].c = b2 * vv[u].c + (1.0f - b2) * gg[u].c * gg[u].c;                   \
    pp[u].c -= __fdividef(a * (mm[u].c * inv_bc1), sqrt_approx(vv[u].c) * inv_sqrt_bc2 + eps);
                GS_ADAM_LANE(x) GS_ADAM_LANE(y) GS_ADAM_LANE(z) GS_ADAM_LANE(w)
#undef GS_ADAM_LANE
                store_lanes(m, i, mm[u], own);
                store_lanes(v, i, vv[u], own);
                store_lanes(p, i, pp[u], own);
            }
        }
    }
}

// Part 2 as a background kernel: one CTA of kBgThreads per SM, each thread a float4 column
// of four Gaussians through all planes, kBgU planes' loads in flight, with streaming cache
// hints: little of the SM and of L2 taken from the kernels it runs beside (swept: 64 to 256
// threads, one or two CTAs per SM, one to eight planes in flight).
constexpr int kBgThreads = 256;
constexpr int kBgU = 1;

__global__ void __launch_bounds__(kBgThreads, 1) k_adam_unseen(float4 *__restrict__ p, float4 *__restrict__ m,
                                                               float4 *__restrict__ v, long long ld4, int planes,
                                                               AdamLr lr, float b1, float b2, float inv_bc1,
                                                               float inv_sqrt_bc2, float eps,
                                                               const long long *__restrict__ step_dev,
                                                               const int4 *__restrict__ radius4, int n_views) {
    griddep_wait();
    if (step_dev) {
        __shared__ float s_bc[2];
        if (threadIdx.x == 0) {
            adam_bias_inv(b1, b2, *step_dev, s_bc[0], s_bc[1]);
        }
        __syncthreads();
        inv_bc1 = s_bc[0];
        inv_sqrt_bc2 = s_bc[1];
    }
    for (long long c4 = (long long)blockIdx.x * blockDim.x + threadIdx.x; c4 < ld4;
         c4 += (long long)gridDim.x * blockDim.x) {
        uint32_t seen = 0u;
        for (int vw = 0; vw < n_views; ++vw) {
            const int4 rad = radius4[vw * ld4 + c4];
            seen |= (rad.x > 0 ? 0x1u : 0u) | (rad.y > 0 ? 0x100u : 0u) | (rad.z > 0 ? 0x10000u : 0u) |
                    (rad.w > 0 ? 0x1000000u : 0u);
        }
        const uint32_t own = seen ^ 0x01010101u;
        if (own == 0u) continue;
        for (int q = 0; q < planes; q += kBgU) {
            float4 mm[kBgU], vv[kBgU], pp[kBgU];
            #pragma unroll
            for (int u = 0; u < kBgU; ++u) {
                if (q + u >= planes) continue;
                const long long i = (long long)(q + u) * ld4 + c4;
                mm[u] = __ldcs(m + i); vv[u] = __ldcs(v + i); pp[u] = __ldcs(p + i);
            }
            #pragma unroll
            for (int u = 0; u < kBgU; ++u) {
                if (q + u >= planes) continue;
                const long long i = (long long)(q + u) * ld4 + c4;
                const float a = lr.lr[lr_group(q + u)];
                const float4 gz = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                float4 gg[1] = {gz};
#define GS_ADAM_LANE(c)                                                         \
    mm[u].c = b1 * mm[u].c + (1.0f - b1) * gg[0].c;                             \
    vv[u].c = b2 * vv[u].c + (1.0f - b2) * gg[0].c * gg[0].c;                   \
    pp[u].c -= __fdividef(a * (mm[u].c * inv_bc1), sqrt_approx(vv[u].c) * inv_sqrt_bc2 + eps);
                GS_ADAM_LANE(x) GS_ADAM_LANE(y) GS_ADAM_LANE(z) GS_ADAM_LANE(w)
#undef GS_ADAM_LANE
                if (own == 0x01010101u) {
                    __stcs(m + i, mm[u]); __stcs(v + i, vv[u]); __stcs(p + i, pp[u]);
                } else {
                    store_lanes(m, i, mm[u], own);
                    store_lanes(v, i, vv[u], own);
                    store_lanes(p, i, pp[u], own);
                }
            }
        }
    }
}

void launch_adam(float *p, const float *g, float *m, float *v, long long ld, int planes, const float lr[6],
                 float beta1, float beta2, float eps, long long step, const long long *step_dev,
                 const uint8_t *rows, cudaStream_t s, int part, const int *radius, int n_views) {
    AdamLr L;
    for (int k = 0; k < 6; ++k) L.lr[k] = lr[k];
    const double st = step_dev ? 1.0 : (double)step;  // placeholder when the device counter is used
    const double bc1 = 1.0 - pow((double)beta1, st);
    const double bc2 = 1.0 - pow((double)beta2, st);
    const long long total4 = (long long)planes * ld / 4;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (part == 2) {
        const int blocks = (int)std::min<long long>(ceil_div(ld / 4, kBgThreads), (long long)sms);
        if (blocks <= 0) return;
        // the largest shared-memory split, as the sort and compositing kernels it runs beside
        // take: a CTA resident under another split keeps those kernels off its SM until it ends
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_adam_unseen, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            attr = true;
        }
        launch_pdl(k_adam_unseen, blocks, kBgThreads, 0, s, (float4 *)p, (float4 *)m, (float4 *)v, ld / 4, planes, L, beta1,
                                                    beta2, (float)(1.0 / bc1), (float)(1.0 / sqrt(bc2)), eps,
                                                    step_dev, (const int4 *)radius, n_views);
        return;
    }
    if (rows) {
        const long long items = (planes + kAdamPlanes - 1) / kAdamPlanes * (ld / 4);
        const int blocks = (int)std::min<long long>(ceil_div(items, 256), (long long)sms * 8);
        if (blocks <= 0) return;
        launch_pdl(k_adam_rows, blocks, 256, 0, s, (float4 *)p, (const float4 *)g, (float4 *)m, (float4 *)v, ld / 4, planes,
                                           L, beta1, beta2, (float)(1.0 / bc1), (float)(1.0 / sqrt(bc2)), eps,
                                           step_dev, (const uint32_t *)rows, part);
        return;
    }
    const long long want = ceil_div(total4, 256);
    const int blocks = (int)std::min<long long>(want, (long long)sms * 8);
    if (blocks <= 0) return;
    launch_pdl(k_adam, blocks, 256, 0, s, (float4 *)p, (const float4 *)g, (float4 *)m, (float4 *)v, ld / 4, total4, L, beta1,
                                  beta2, (float)(1.0 / bc1), (float)(1.0 / sqrt(bc2)), eps, step_dev);
}

}  // namespace gs
