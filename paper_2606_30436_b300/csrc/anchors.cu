// anchors.cu -- Scaffold-GS anchors (Supp. D.1 decoding, Supp. D.3 LoD
// mask): each anchor's decoder turns (feature, view direction, log(1 +
// distance)) into its K = 10 Gaussians, written as SH-degree-0 Gaussians for
// the rasteriser; the backward takes the rasteriser's parameter gradients back
// to the anchors and the decoder's weights; a flat Adam updates both.
//
// k_anchor_decode: thread per anchor, the decoder's weights (11,468 floats)
// in shared memory and read as broadcasts; hidden layer in registers; slot
// (k, i) of the output is column k ld + i of every plane (coalesced per k).
// Dropped Gaussians (outside the level's distance band, opacity <= 0) get a
// placeholder whose opacity logit (-30) the projection culls.
// k_anchor_decode_bwd: 128-anchor tiles, thread per anchor.  The inputs, the
// hidden activations and dL/dz of the tile are staged in shared memory
// ([row][129]: a column read by a warp touches 32 banks); each thread then
// owns 70 entries of dW2 (35 outputs of its warp x 2 hidden units of its
// lane, so a row of the tile costs 37 loads for 70 FMAs) and 18 of dW1, sums
// them over the tile's anchors in registers across its tiles (one FP32
// atomic per weight per CTA at the end), and takes its own anchor's
// dL/dh = W2^T dz and dL/df = W1^T dL/dpre.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "gs_internal.cuh"
#include "gs_kernels.h"

namespace gs {

namespace {

constexpr int kAK = GS_ANCHOR_K, kAF = GS_ANCHOR_FEAT, kAIn = kAF + 4, kAH = 64, kAOut = 14 * kAK;
constexpr int kAW1 = 0, kAB1 = kAW1 + kAH * kAIn, kAW2 = kAB1 + kAH, kAB2 = kAW2 + kAOut * kAH,
              kANW = kAB2 + kAOut;
static_assert(kANW == GS_ANCHOR_WEIGHTS, "decoder weight count");
static_assert(kAIn % 4 == 0 && kAH % 4 == 0 && kAW2 % 4 == 0, "weight rows on 16-byte boundaries");
constexpr int kPlaneLogL = kAF, kPlaneOffs = kAF + 3;
static_assert(kPlaneOffs + 3 * kAK == GS_ANCHOR_PLANES, "anchor planes");
constexpr float kY00 = 0.28209479177387814f;
constexpr float kDeadLogit = -30.0f;
constexpr int kBT = 128, kLdS = kBT + 1;  // backward tile and its padded shared row

__device__ __forceinline__ float sigmoidf(float z) { return 1.0f / (1.0f + expf(-z)); }

// log(sigmoid(z)) without overflow for either sign
__device__ __forceinline__ float log_sigmoidf(float z) {
    return z >= 0.0f ? -log1pf(expf(-z)) : z - log1pf(expf(z));
}

// Decoder input of anchor i (feature, unit direction from the camera, log(1 + d)); returns d.
__device__ __forceinline__ float anchor_input(const float *__restrict__ A, const float *__restrict__ pos, long long ld,
                                              long long i, const AnchorView &v, float *x) {
    const float dx = pos[i] - v.c[0], dy = pos[ld + i] - v.c[1], dz = pos[2 * ld + i] - v.c[2];
    const float d = sqrtf(dx * dx + dy * dy + dz * dz);
    #pragma unroll
    for (int c = 0; c < kAF; ++c) x[c] = A[c * ld + i];
    x[kAF] = dx / d;
    x[kAF + 1] = dy / d;
    x[kAF + 2] = dz / d;
    x[kAF + 3] = log1pf(d);
    return d;
}

__device__ __forceinline__ bool band_active(const AnchorView &v, int l, float d) {
    return l >= 0 && l < v.levels && d >= v.lo[l] && d < v.hi[l];
}

__device__ __forceinline__ void write_dead(float *__restrict__ G, long long gld, long long col, const float *p,
                                           const float *L) {
    #pragma unroll
    for (int c = 0; c < 3; ++c) {
        G[c * gld + col] = p[c];
        G[(3 + c) * gld + col] = L[c];
    }
    G[6 * gld + col] = 1.0f;
    G[7 * gld + col] = 0.0f;
    G[8 * gld + col] = 0.0f;
    G[9 * gld + col] = 0.0f;
    G[10 * gld + col] = kDeadLogit;
    G[11 * gld + col] = 0.0f;
    G[12 * gld + col] = 0.0f;
    G[13 * gld + col] = 0.0f;
}

__global__ void __launch_bounds__(256) k_anchor_decode(const float *__restrict__ A, const float *__restrict__ pos,
                                                       const int *__restrict__ level, long long n, long long ld,
                                                       const float *__restrict__ w, const __grid_constant__ AnchorView v,
                                                       float *__restrict__ G, long long gld) {
    __shared__ __align__(16) float sw[kANW];
    for (int j = threadIdx.x; j < kANW; j += blockDim.x) sw[j] = w[j];
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ld) return;
    float p[3] = {0.0f, 0.0f, 0.0f}, L[3] = {0.0f, 0.0f, 0.0f};
    bool M = false;
    float h[kAH];
    if (i < n) {
        float x[kAIn];
        const float d = anchor_input(A, pos, ld, i, v, x);
        #pragma unroll
        for (int c = 0; c < 3; ++c) {
            p[c] = pos[c * ld + i];
            L[c] = A[(kPlaneLogL + c) * ld + i];
        }
        M = band_active(v, level[i], d);
        if (M) {
            // weight rows read as float4 broadcasts (rows start on 16-byte boundaries)
            #pragma unroll
            for (int o = 0; o < kAH; ++o) {
                const float4 *w4 = reinterpret_cast<const float4 *>(sw + kAW1 + o * kAIn);
                float s = sw[kAB1 + o];
                #pragma unroll
                for (int c = 0; c < kAIn / 4; ++c) {
                    const float4 q = w4[c];
                    s += q.x * x[4 * c] + q.y * x[4 * c + 1] + q.z * x[4 * c + 2] + q.w * x[4 * c + 3];
                }
                h[o] = fmaxf(s, 0.0f);
            }
        }
    }
    for (int k = 0; k < kAK; ++k) {
        const long long col = k * ld + i;
        if (!M) {
            write_dead(G, gld, col, p, L);
            continue;
        }
        float z[14];
        #pragma unroll
        for (int j = 0; j < 14; ++j) {
            const int o = 14 * k + j;
            const float4 *w4 = reinterpret_cast<const float4 *>(sw + kAW2 + o * kAH);
            float s = sw[kAB2 + o];
            #pragma unroll
            for (int c = 0; c < kAH / 4; ++c) {
                const float4 q = w4[c];
                s += q.x * h[4 * c] + q.y * h[4 * c + 1] + q.z * h[4 * c + 2] + q.w * h[4 * c + 3];
            }
            z[j] = s;
        }
        const float a = tanhf(z[3]);
        if (!(a > 0.0f)) {
            write_dead(G, gld, col, p, L);
            continue;
        }
        #pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float l = expf(L[c]);
            G[c * gld + col] = p[c] + (A[(kPlaneOffs + 3 * k + c) * ld + i] + z[11 + c]) * l;  // mean
            G[(3 + c) * gld + col] = L[c] + log_sigmoidf(z[8 + c]);                          // log(l ds)
            G[(11 + c) * gld + col] = (sigmoidf(z[c]) - 0.5f) / kY00;                          // colour
        }
        G[6 * gld + col] = 1.0f + z[4];
        G[7 * gld + col] = z[5];
        G[8 * gld + col] = z[6];
        G[9 * gld + col] = z[7];
        G[10 * gld + col] = logf(a) - log1pf(-a);
    }
}

struct BwdSmem {
    float w[kANW];
    float xs[kAIn][kLdS];
    float hs[kAH][kLdS];   // hidden activations, then dL/d(pre-activation)
    float dz[kAOut][kLdS];
};

__global__ void __launch_bounds__(kBT) k_anchor_decode_bwd(const float *__restrict__ A, const float *__restrict__ pos,
                                                           const int *__restrict__ level, long long n, long long ld,
                                                           const float *__restrict__ w,
                                                           const __grid_constant__ AnchorView v,
                                                           const float *__restrict__ GG, long long gld,
                                                           float *__restrict__ gA, float *__restrict__ gw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem &s = *reinterpret_cast<BwdSmem *>(smem_raw);
    const int t = threadIdx.x;
    for (int j = t; j < kANW; j += kBT) s.w[j] = w[j];
    constexpr int kE2 = kAOut * kAH / kBT, kE1 = kAH * kAIn / kBT;  // 70, 18 entries per thread
    static_assert(kE2 * kBT == kAOut * kAH && kE1 * kBT == kAH * kAIn, "weight entries per thread");
    // dW2 entries of this thread: outputs kO2 * warp + j (j < kO2), hidden units lane and lane + 32
    constexpr int kO2 = kAOut / (kBT / 32);  // 35
    static_assert(kO2 * (kBT / 32) == kAOut && 2 * kO2 == kE2 && kAH == 64, "dW2 blocking");
    const int warp = t >> 5, lane = t & 31;
    float aW2[kE2], aW1[kE1], aB2[2] = {0.0f, 0.0f}, aB1 = 0.0f;
    #pragma unroll
    for (int j = 0; j < kE2; ++j) aW2[j] = 0.0f;
    #pragma unroll
    for (int j = 0; j < kE1; ++j) aW1[j] = 0.0f;
    __syncthreads();
    const long long tiles = ceil_div(n, (long long)kBT);
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const long long i = tile * kBT + t;
        const bool valid = i < n;
        bool M = false;
        float L[3] = {0.0f, 0.0f, 0.0f};
        {
            float x[kAIn];
            float d = 0.0f;
            if (valid) {
                d = anchor_input(A, pos, ld, i, v, x);
                M = band_active(v, level[i], d);
                #pragma unroll
                for (int c = 0; c < 3; ++c) L[c] = A[(kPlaneLogL + c) * ld + i];
            } else {
                #pragma unroll
                for (int c = 0; c < kAIn; ++c) x[c] = 0.0f;
            }
            #pragma unroll
            for (int c = 0; c < kAIn; ++c) s.xs[c][t] = x[c];
            #pragma unroll
            for (int o = 0; o < kAH; ++o) {
                float a = s.w[kAB1 + o];
                #pragma unroll
                for (int c = 0; c < kAIn; ++c) a += s.w[kAW1 + o * kAIn + c] * x[c];
                s.hs[o][t] = M ? fmaxf(a, 0.0f) : 0.0f;
            }
        }
        // dL/dz of the kept Gaussians; the anchor's own offset and log-scale gradients
        float gL[3] = {0.0f, 0.0f, 0.0f};
        for (int k = 0; k < kAK; ++k) {
            float dz[14];
            #pragma unroll
            for (int j = 0; j < 14; ++j) dz[j] = 0.0f;
            float gO[3] = {0.0f, 0.0f, 0.0f};
            if (M) {
                float z[14];
                #pragma unroll
                for (int j = 0; j < 14; ++j) {
                    const int o = 14 * k + j;
                    float a = s.w[kAB2 + o];
                    #pragma unroll 16
                    for (int c = 0; c < kAH; ++c) a += s.w[kAW2 + o * kAH + c] * s.hs[c][t];
                    z[j] = a;
                }
                const float a = tanhf(z[3]);
                if (a > 0.0f) {
                    const long long col = k * ld + i;
                    float g[14];
                    #pragma unroll
                    for (int j = 0; j < 14; ++j) g[j] = GG[j * gld + col];
                    #pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float l = expf(L[c]);
                        const float O = A[(kPlaneOffs + 3 * k + c) * ld + i] + z[11 + c];
                        dz[11 + c] = g[c] * l;
                        gO[c] = g[c] * l;
                        gL[c] += g[c] * O * l + g[3 + c];
                        dz[8 + c] = g[3 + c] * (1.0f - sigmoidf(z[8 + c]));
                        const float sc = sigmoidf(z[c]);
                        dz[c] = g[11 + c] * sc * (1.0f - sc) / kY00;
                    }
                    #pragma unroll
                    for (int c = 0; c < 4; ++c) dz[4 + c] = g[6 + c];
                    dz[3] = g[10] * (1.0f + a) / a;  // d logit(tanh z) / dz
                }
            }
            #pragma unroll
            for (int j = 0; j < 14; ++j) s.dz[14 * k + j][t] = dz[j];
            if (valid) {
                #pragma unroll
                for (int c = 0; c < 3; ++c) gA[(kPlaneOffs + 3 * k + c) * ld + i] = gO[c];
            }
        }
        if (valid) {
            #pragma unroll
            for (int c = 0; c < 3; ++c) gA[(kPlaneLogL + c) * ld + i] = gL[c];
        }
        __syncthreads();
        // dW2, db2 over the tile's anchors: per row r, 35 broadcast loads of dz and two of h
        // feed 70 accumulators
        for (int r = 0; r < kBT; ++r) {
            const float h0 = s.hs[lane][r], h1 = s.hs[lane + 32][r];
            #pragma unroll
            for (int j = 0; j < kO2; ++j) {
                const float g = s.dz[kO2 * warp + j][r];
                aW2[2 * j] += g * h0;
                aW2[2 * j + 1] += g * h1;
            }
        }
        #pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int o = t + kBT * q;
            if (o < kAOut) {
                float a = 0.0f;
                for (int r = 0; r < kBT; ++r) a += s.dz[o][r];
                aB2[q] += a;
            }
        }
        // the anchor's dL/dh = W2^T dz through the ReLU
        float dp[kAH];
        #pragma unroll
        for (int c = 0; c < kAH; ++c) dp[c] = 0.0f;
        for (int o = 0; o < kAOut; ++o) {
            const float g = s.dz[o][t];
            const float4 *w4 = reinterpret_cast<const float4 *>(s.w + kAW2 + o * kAH);
            #pragma unroll
            for (int c = 0; c < kAH / 4; ++c) {
                const float4 q = w4[c];
                dp[4 * c] += q.x * g;
                dp[4 * c + 1] += q.y * g;
                dp[4 * c + 2] += q.z * g;
                dp[4 * c + 3] += q.w * g;
            }
        }
        #pragma unroll
        for (int c = 0; c < kAH; ++c) dp[c] = s.hs[c][t] > 0.0f ? dp[c] : 0.0f;
        __syncthreads();  // every thread has read the activations
        #pragma unroll
        for (int c = 0; c < kAH; ++c) s.hs[c][t] = dp[c];
        __syncthreads();
        // dW1, db1 over the tile's anchors; the anchor's feature gradient
        #pragma unroll
        for (int j = 0; j < kE1; ++j) {
            const int e = t + kBT * j, o = e / kAIn, c = e % kAIn;
            float a = 0.0f;
            #pragma unroll 8
            for (int r = 0; r < kBT; ++r) a += s.hs[o][r] * s.xs[c][r];
            aW1[j] += a;
        }
        if (t < kAH) {
            float a = 0.0f;
            for (int r = 0; r < kBT; ++r) a += s.hs[t][r];
            aB1 += a;
        }
        if (valid) {
            for (int c = 0; c < kAF; ++c) {
                float a = 0.0f;
                #pragma unroll
                for (int o = 0; o < kAH; ++o) a += s.w[kAW1 + o * kAIn + c] * dp[o];
                gA[c * ld + i] = a;
            }
        }
        __syncthreads();  // the tile's shared arrays are rewritten next
    }
    #pragma unroll
    for (int j = 0; j < kO2; ++j) {
        const int o = kO2 * warp + j;
        atomicAdd(&gw[kAW2 + o * kAH + lane], aW2[2 * j]);
        atomicAdd(&gw[kAW2 + o * kAH + lane + 32], aW2[2 * j + 1]);
    }
    #pragma unroll
    for (int j = 0; j < kE1; ++j) atomicAdd(&gw[kAW1 + t + kBT * j], aW1[j]);
    #pragma unroll
    for (int q = 0; q < 2; ++q)
        if (t + kBT * q < kAOut) atomicAdd(&gw[kAB2 + t + kBT * q], aB2[q]);
    if (t < kAH) atomicAdd(&gw[kAB1 + t], aB1);
}

__global__ void k_adam_flat(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long n, float lr, float b1, float b2, float eps, float bc1,
                            float bc2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi, vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

int sm_count_anchor() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace

cudaError_t launch_anchor_decode(const float *A, const float *pos, const int *level, long long n, long long ld,
                                 const float *w, const AnchorView &v, float *G, long long gld, cudaStream_t s) {
    if (ld <= 0) return cudaSuccess;
    k_anchor_decode<<<(unsigned)ceil_div(ld, 256ll), 256, 0, s>>>(A, pos, level, n, ld, w, v, G, gld);
    return cudaGetLastError();
}

cudaError_t launch_anchor_decode_bwd(const float *A, const float *pos, const int *level, long long n, long long ld,
                                     const float *w, const AnchorView &v, const float *GG, long long gld, float *gA,
                                     float *gw, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(gA, 0, sizeof(float) * GS_ANCHOR_PLANES * (size_t)ld, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(gw, 0, sizeof(float) * kANW, s);
    if (e != cudaSuccess || n <= 0) return e;
    const size_t smem = sizeof(BwdSmem);
    static bool attr = false;
    if (!attr) {
        e = cudaFuncSetAttribute(k_anchor_decode_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long grid = std::min<long long>(ceil_div(n, (long long)kBT), (long long)sm_count_anchor());
    k_anchor_decode_bwd<<<(unsigned)grid, kBT, smem, s>>>(A, pos, level, n, ld, w, v, GG, gld, gA, gw);
    return cudaGetLastError();
}

cudaError_t launch_adam_flat(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                             float eps, long long step, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const float bc1 = (float)(1.0 - std::pow((double)b1, (double)step));
    const float bc2 = (float)(1.0 - std::pow((double)b2, (double)step));
    const long long blocks = std::min<long long>(ceil_div(n, 256ll), 4096ll);
    k_adam_flat<<<(unsigned)blocks, 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2);
    return cudaGetLastError();
}

}  // namespace gs
