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
    if (step_dev) {  // bias corrections from the device step counter (graph replay)
        __shared__ float s_bc[2];
        if (threadIdx.x == 0) {
            const double t = (double)*step_dev;
            s_bc[0] = (float)(1.0 / (1.0 - pow((double)b1, t)));
            s_bc[1] = (float)(1.0 / sqrt(1.0 - pow((double)b2, t)));
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
// all-zero mark skips the gradient's loads.
constexpr int kAdamPlanes = 8;

__global__ void __launch_bounds__(256) k_adam_rows(float4 *__restrict__ p, const float4 *__restrict__ g,
                                                    float4 *__restrict__ m, float4 *__restrict__ v, long long ld4,
                                                    int planes, AdamLr lr, float b1, float b2, float inv_bc1,
                                                    float inv_sqrt_bc2, float eps,
                                                    const long long *__restrict__ step_dev,
                                                    const uint32_t *__restrict__ rows4) {
    if (step_dev) {
        __shared__ float s_bc[2];
        if (threadIdx.x == 0) {
            const double t = (double)*step_dev;
            s_bc[0] = (float)(1.0 / (1.0 - pow((double)b1, t)));
            s_bc[1] = (float)(1.0 / sqrt(1.0 - pow((double)b2, t)));
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
        const uint32_t r = rows4[c4];
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
                m[i] = mm[u];
                v[i] = vv[u];
                p[i] = pp[u];
            }
        }
    }
}

void launch_adam(float *p, const float *g, float *m, float *v, long long ld, int planes, const float lr[6],
                 float beta1, float beta2, float eps, long long step, const long long *step_dev,
                 const uint8_t *rows, cudaStream_t s) {
    AdamLr L;
    for (int k = 0; k < 6; ++k) L.lr[k] = lr[k];
    const double st = step_dev ? 1.0 : (double)step;  // placeholder when the device counter is used
    const double bc1 = 1.0 - pow((double)beta1, st);
    const double bc2 = 1.0 - pow((double)beta2, st);
    const long long total4 = (long long)planes * ld / 4;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (rows) {
        const long long items = (planes + kAdamPlanes - 1) / kAdamPlanes * (ld / 4);
        const int blocks = (int)std::min<long long>(ceil_div(items, 256), (long long)sms * 8);
        if (blocks <= 0) return;
        k_adam_rows<<<blocks, 256, 0, s>>>((float4 *)p, (const float4 *)g, (float4 *)m, (float4 *)v, ld / 4, planes,
                                           L, beta1, beta2, (float)(1.0 / bc1), (float)(1.0 / sqrt(bc2)), eps,
                                           step_dev, (const uint32_t *)rows);
        return;
    }
    const long long want = ceil_div(total4, 256);
    const int blocks = (int)std::min<long long>(want, (long long)sms * 8);
    if (blocks <= 0) return;
    k_adam<<<blocks, 256, 0, s>>>((float4 *)p, (const float4 *)g, (float4 *)m, (float4 *)v, ld / 4, total4, L, beta1,
                                  beta2, (float)(1.0 / bc1), (float)(1.0 / sqrt(bc2)), eps, step_dev);
}

}  // namespace gs
