// mlp.cu -- learned prune / densify predictor: per-Gaussian features, an MLP
// 16 -> 64 -> 64 -> 2 (ReLU, sigmoid outputs: densify, prune) on the 5th
// generation tensor cores, and its training step on labels from the plain
// criterion of Supp. E (S_d > tau_d, S_p > tau_p).
//
// Tile = 128 Gaussians = the M of one tcgen05.mma; thread t of the CTA owns
// row t (TMEM lane t).  Layer 1 (K = 16) and layer 2 (K = 64, four K = 16
// steps) and, in training, the data gradient dh1 = dh2 W2 (K = 64) run as
// tcgen05.mma.kind::f16 with BF16 operands in shared memory (K-major, no
// swizzle: 8x8 core matrices of 128 bytes, leading offset = the next core
// matrix along K, stride offset = the next 8-row group) and FP32 accumulators
// in TMEM, read back with tcgen05.ld.  The hidden layers' weight gradients
// are tcgen05 contractions over the tile's rows whose operands are the same
// tiles read MN-major (the transpose bits of the instruction descriptor).
// The 64 -> 2 head, the BCE gradient and the output layer's weight gradient
// run in FP32 on CUDA cores.
// Every mbarrier wait is bounded; on a timeout the kernel flags the status
// word, stops issuing, and still frees its TMEM.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>

#include <cuda_bf16.h>

#include "gs_internal.cuh"
#include "gs_kernels.h"
#include "tcgen05.cuh"

namespace gs {

constexpr int kIn = 16, kH = 64, kOut = 2, kM = 128;
constexpr int kW1 = 0, kB1 = kW1 + kH * kIn, kW2 = kB1 + kH, kB2 = kW2 + kH * kH, kW3 = kB2 + kH,
              kB3 = kW3 + kOut * kH, kNW = kB3 + kOut;
constexpr int kRing = 8;            // blend-weight history (views)
constexpr int kTmemCols = 128;      // D1 in columns [0, 64), D2 in [64, 128)

// KX and KH: core matrices per 8-row group of x and h1 (2 and 8 for the
// forward; wider in training, where the extra columns hold the constant 1 of
// the bias gradient and zero padding).
template <int KX, int KH>
struct MlpSmemT {
    static constexpr int kx = KX, kh = KH;
    alignas(128) __nv_bfloat16 w1[kH * kIn];    // B of layer 1: [n = out][k = in]
    alignas(128) __nv_bfloat16 w2[kH * kH];     // B of layer 2: [n = out][k = in]
    alignas(128) __nv_bfloat16 x[kM * 8 * KX];  // A of layer 1: [m = row][k = in]
    alignas(128) __nv_bfloat16 h1[kM * 8 * KH]; // A of layer 2: [m = row][k = in]
    float b1[kH], b2[kH], w3[kOut * kH], b3[kOut];
    uint64_t mbar;
    uint32_t tmem;
};
using MlpSmem = MlpSmemT<kIn / 8, kH / 8>;

// Loads the weights into shared memory (BF16 operands, FP32 rest), allocates
// TMEM and initialises the mbarrier.
template <class S>
__device__ void mlp_setup(S &s, const float *__restrict__ w, uint32_t cols = kTmemCols) {
    for (int i = threadIdx.x; i < kH * kIn; i += blockDim.x) {
        const int o = i / kIn, c = i % kIn;
        s.w1[cm_off(o, c, kIn / 8)] = __float2bfloat16_rn(w[kW1 + i]);
    }
    for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) {
        const int o = i / kH, c = i % kH;
        s.w2[cm_off(o, c, kH / 8)] = __float2bfloat16_rn(w[kW2 + i]);
    }
    for (int i = threadIdx.x; i < kH; i += blockDim.x) { s.b1[i] = w[kB1 + i]; s.b2[i] = w[kB2 + i]; }
    for (int i = threadIdx.x; i < kOut * kH; i += blockDim.x) s.w3[i] = w[kW3 + i];
    if (threadIdx.x < kOut) s.b3[threadIdx.x] = w[kB3 + threadIdx.x];
    tmem_alloc(&s.tmem, cols);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&s.mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
}

// After a timed-out wait no further MMA is issued; the last one committed
// (parity phase ^ 1) gets one more bounded wait before its TMEM is freed.
template <class S>
__device__ void mlp_finish(S &s, bool ok, uint32_t phase, int *status, uint32_t cols = kTmemCols) {
    if (!ok) {
        mbar_wait(&s.mbar, phase ^ 1u);
        if (threadIdx.x == 0 && status) atomicOr(status, 1 << GS_ERR_TIMEOUT);
    }
    tmem_free(s.tmem, cols);
}

// One tile's forward through layer 2.  The thread's features are already in
// s.x; on return h2 (64 FP32, after ReLU) and h1 (64 FP32, after ReLU) hold
// the thread's row.  Returns false on a wait timeout.
template <class S>
__device__ bool mlp_tile_forward(S &s, uint32_t &phase, float *h1, float *h2, long long polls = kSpin) {
    const uint32_t tmem = s.tmem;
    asm volatile("fence.proxy.async.shared::cta;");  // s.x written by threads, read by the tensor core
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        // layer 1: D1[128 x 64] = X[128 x 16] W1^T, one K = 16 step
        mma_bf16(tmem, smem_desc(smem_addr(s.x), 128, S::kx * 128), smem_desc(smem_addr(s.w1), 128, 256),
                 idesc_bf16(kM, kH), false);
        mma_commit(&s.mbar);
    }
    bool ok = mbar_wait(&s.mbar, phase, polls);
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        tmem_row64(tmem, 0, h1);
        #pragma unroll
        for (int c = 0; c < kH; ++c) h1[c] = fmaxf(h1[c] + s.b1[c], 0.0f);
        #pragma unroll
        for (int c0 = 0; c0 < kH; c0 += 8) store_row8(s.h1, threadIdx.x, c0, S::kh, h1 + c0);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    ok = __syncthreads_and(ok);
    if (ok && threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        // layer 2: D2[128 x 64] = H1[128 x 64] W2^T, four K = 16 steps of two core matrices each
        #pragma unroll
        for (int kb = 0; kb < kH / 16; ++kb)
            mma_bf16(tmem + 64, smem_desc(smem_addr(s.h1) + kb * 256, 128, S::kh * 128),
                     smem_desc(smem_addr(s.w2) + kb * 256, 128, 1024), idesc_bf16(kM, kH), kb > 0);
        mma_commit(&s.mbar);
    }
    if (ok) {
        ok = mbar_wait(&s.mbar, phase, polls);
        phase ^= 1u;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        tmem_row64(tmem, 64, h2);
        #pragma unroll
        for (int c = 0; c < kH; ++c) h2[c] = fmaxf(h2[c] + s.b2[c], 0.0f);
    }
    return ok;
}

__global__ void __launch_bounds__(kM, 4) k_mlp_forward(const float *__restrict__ feat, long long n, long long ld,
                                                     const float *__restrict__ w, float *__restrict__ prob,
                                                     uint8_t *__restrict__ densify, uint8_t *__restrict__ prune,
                                                     int *__restrict__ status, long long polls) {
    __shared__ __align__(1024) MlpSmem s;
    mlp_setup(s, w);
    uint32_t phase = 0;
    bool ok = true;
    const long long tiles = ceil_div(n, (long long)kM);
    // the next tile's inputs are loaded into registers while this tile's MMAs run
    float xn[kIn];
    auto load = [&](long long t) {
        const long long row = t * kM + threadIdx.x;
        #pragma unroll
        for (int c = 0; c < kIn; ++c) xn[c] = row < n ? feat[c * ld + row] : 0.0f;
    };
    if ((long long)blockIdx.x < tiles) load(blockIdx.x);
    for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        const long long row = t * kM + threadIdx.x;
        const bool valid = row < n;
        store_row8(s.x, threadIdx.x, 0, kIn / 8, xn);
        store_row8(s.x, threadIdx.x, 8, kIn / 8, xn + 8);
        if (t + gridDim.x < tiles) load(t + gridDim.x);
        float h1[kH], h2[kH];
        ok = mlp_tile_forward(s, phase, h1, h2, polls);
        if (ok && valid) {
            #pragma unroll
            for (int k = 0; k < kOut; ++k) {
                float z = s.b3[k];
                #pragma unroll
                for (int c = 0; c < kH; ++c) z += s.w3[k * kH + c] * h2[c];
                if (prob) prob[k * ld + row] = 1.0f / (1.0f + expf(-z));
                uint8_t *dec = k == 0 ? densify : prune;
                if (dec) dec[row] = z > 0.0f ? 1 : 0;  // sigmoid(z) > 1/2
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        ok = __syncthreads_and(ok);
    }
    mlp_finish(s, ok, phase, status);
}

// Training step: mean BCE over the n rows and both outputs, gradient of every
// weight accumulated into grads (FP32 atomics, one set per CTA).  Per tile:
// the forward (layers 1 and 2 on the tensor cores), the head and dL/dh2 in
// FP32, then three tcgen05 contractions with BF16 operands and FP32
// accumulators in TMEM:
//   dh1 (before the ReLU mask) = dh2 W2                          [128 x 64],
//   dW2 | db2 += dh2^T [h1 | 1]   over the tile's rows (K = 128)  [64 x 80],
//   dW1 | db1 += dh1^T [x | 1]    over the tile's rows            [64 x 32].
// dh2 and dh1 are stored once, [row][out] (A of the data gradient K-major, A
// of the weight sums MN-major); h1 and x are the forward's own operands,
// stored with a constant-1 column (the bias) and zero padding and read
// MN-major as the weight sums' B.  dh2 and dh1 enter as dL/dh / scale (O(1)
// values), the sums are rescaled at the end.  The weight sums use M = 128 of
// which the first 64 rows are the layer's outputs (rows 64-127 of D are never
// read; their A rows read whatever shared memory follows).  dW3 and db3 stay
// in FP32 on CUDA cores, from transposed copies of h2 and dL/dz.
constexpr uint32_t kTrainCols = 256;
constexpr int kColW2 = 128, kN2 = 80;  // dW2 | db2 accumulator: 64 weights, the bias, zero padding
constexpr int kColW1 = 208, kN1 = 32;  // dW1 | db1 accumulator: 16 weights, the bias, zero padding
constexpr int kLdH2 = kM + 4;          // padded row of the transposed h2 (16-byte aligned, conflict-free)
using MlpTrainF = MlpSmemT<kN1 / 8, kN2 / 8>;

struct MlpTrainSmem {
    MlpTrainF f;
    alignas(128) __nv_bfloat16 w2t[kH * kH];  // B of the data gradient: [n = in][k = out] = W2^T
    alignas(128) __nv_bfloat16 dh[kM * kH];   // [row][out]: dh2 / scale, then dh1 / scale
    alignas(16) float h2t[kH][kLdH2];         // FP32 h2, [out][row]
    alignas(16) float dzt[kOut][kM];          // dL/dz, [output][row]
    float red[kM / 32];
};

// Byte strides of the MN-major reads: dh as [m = out][k = row] has 8-out groups
// 128 B apart and 8-row groups kH / 8 * 128 B apart; h1 and x as [n = in][k = row]
// likewise with kN2 / 8 and kN1 / 8 groups per row group.
constexpr uint32_t kDhK = kH / 8 * 128, kH1K = kN2 / 8 * 128, kXK = kN1 / 8 * 128;
// Every descriptor read stays inside the CTA's shared memory whichever of the
// two strides the hardware takes as the K one: the largest byte reached from
// an operand's start is (last K step) + 15 or 9 or 3 groups x the larger stride
// + one group x the other + 127.
static_assert(offsetof(MlpTrainSmem, dh) + 7 * 2 * kDhK + 15 * kDhK + 128 + 127 < sizeof(MlpTrainSmem), "dh read");
static_assert(offsetof(MlpTrainSmem, f) + offsetof(MlpTrainF, h1) + 7 * 2 * kH1K + 9 * kH1K + 128 + 127 <
                  sizeof(MlpTrainSmem), "h1 read");
static_assert(offsetof(MlpTrainF, x) + 7 * 2 * kXK + 3 * kXK + 128 + 127 < sizeof(MlpTrainSmem), "x read");
static_assert(offsetof(MlpTrainSmem, w2t) % 128 == 0 && offsetof(MlpTrainSmem, dh) % 128 == 0 &&
                  offsetof(MlpTrainF, x) % 128 == 0 && offsetof(MlpTrainF, h1) % 128 == 0,
              "tensor-core operands must be 16-byte aligned");
static_assert(2 * (sizeof(MlpTrainSmem) + 1024) <= 228 * 1024, "two training CTAs per SM");
static_assert(kColW1 + kN1 <= (int)kTrainCols && kColW2 + kN2 <= kColW1, "TMEM columns");

__global__ void __launch_bounds__(kM, 2) k_mlp_train(const float *__restrict__ feat, const uint8_t *__restrict__ y_densify,
                                                      const uint8_t *__restrict__ y_prune, long long n, long long ld,
                                                      const float *__restrict__ w, float *__restrict__ grad,
                                                      float *__restrict__ loss, int *__restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    MlpTrainSmem &s = *reinterpret_cast<MlpTrainSmem *>(smem_raw);
    mlp_setup(s.f, w, kTrainCols);
    const int t = threadIdx.x;
    for (int i = t; i < kH * kH; i += blockDim.x) {
        const int o = i / kH, c = i % kH;  // W2[o][c] -> B[n = c][k = o]
        s.w2t[cm_off(c, o, kH / 8)] = __float2bfloat16_rn(w[kW2 + i]);
    }
    {
        // the constant columns of x and h1: 1 (the bias gradient), then zeros
        const float one[8] = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, zero[8] = {};
        store_row8(s.f.x, t, kIn, kN1 / 8, one);
        store_row8(s.f.x, t, kIn + 8, kN1 / 8, zero);
        store_row8(s.f.h1, t, kH, kN2 / 8, one);
        store_row8(s.f.h1, t, kH + 8, kN2 / 8, zero);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();

    const float scale = 1.0f / (float)(n * kOut);
    const uint32_t tmem = s.f.tmem;
    float gw3 = 0.f, gb3 = 0.f;  // W3 (k, c) = (t / 64, t % 64); b3 for t < 2
    double lsum = 0.0;
    uint32_t phase = 0;
    bool ok = true, first = true;
    const long long tiles = ceil_div(n, (long long)kM);
    // the next tile's inputs are loaded into registers while this tile's MMAs run
    float xn[kIn];
    auto load = [&](long long tl) {
        const long long row = tl * kM + t;
        #pragma unroll
        for (int c = 0; c < kIn; ++c) xn[c] = row < n ? feat[c * ld + row] : 0.0f;
    };
    if ((long long)blockIdx.x < tiles) load(blockIdx.x);
    for (long long tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const long long row = tile * kM + t;
        const bool valid = row < n;
        const float yd = valid && y_densify[row] ? 1.0f : 0.0f, yp = valid && y_prune[row] ? 1.0f : 0.0f;
        store_row8(s.f.x, t, 0, kN1 / 8, xn);
        store_row8(s.f.x, t, 8, kN1 / 8, xn + 8);
        if (tile + gridDim.x < tiles) load(tile + gridDim.x);
        float h2[kH];
        {
            float h1[kH];
            ok = mlp_tile_forward(s.f, phase, h1, h2);
        }
        // head, BCE and (p - y) (FP32, this thread's row)
        float r[kOut] = {0.f, 0.f};
        if (ok && valid) {
            #pragma unroll
            for (int k = 0; k < kOut; ++k) {
                float z = s.f.b3[k];
                #pragma unroll
                for (int c = 0; c < kH; ++c) z += s.f.w3[k * kH + c] * h2[c];
                const float p = 1.0f / (1.0f + expf(-z));
                const float y = k == 0 ? yd : yp;
                // BCE from the logit: log(1 + e^z) - y z, stable for either sign of z
                lsum += (double)(fmaxf(z, 0.0f) - y * z + log1pf(expf(-fabsf(z))));
                r[k] = p - y;
            }
        }
        // dL/dh2 / scale = [h2 > 0] (p - y) W3, rounded to BF16, [row][out]
        #pragma unroll
        for (int c0 = 0; c0 < kH; c0 += 8) {
            float d[8];
            #pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = c0 + j;
                d[j] = h2[c] > 0.0f ? r[0] * s.f.w3[c] + r[1] * s.f.w3[kH + c] : 0.0f;
            }
            store_row8(s.dh, t, c0, kH / 8, d);
        }
        #pragma unroll
        for (int c = 0; c < kH; ++c) s.h2t[c][t] = h2[c];
        s.dzt[0][t] = r[0] * scale;
        s.dzt[1][t] = r[1] * scale;
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        ok = __syncthreads_and(ok);
        if (ok && t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            // dh1 / scale (before the ReLU mask) = (dh2 / scale) W2 -> TMEM columns [0, 64)
            #pragma unroll
            for (int kb = 0; kb < kH / 16; ++kb)
                mma_bf16(tmem, smem_desc(smem_addr(s.dh) + kb * 256, 128, kDhK),
                         smem_desc(smem_addr(s.w2t) + kb * 256, 128, 1024), idesc_bf16(kM, kH), kb > 0);
            // dW2 | db2 += (dh2 / scale)^T [h1 | 1] over the tile's rows, 16 rows per step
            #pragma unroll
            for (int kb = 0; kb < kM / 16; ++kb)
                mma_bf16(tmem + kColW2, smem_desc_mn(smem_addr(s.dh) + kb * 2 * kDhK, kDhK, 128),
                         smem_desc_mn(smem_addr(s.f.h1) + kb * 2 * kH1K, kH1K, 128), idesc_bf16_mn(kM, kN2),
                         !first || kb > 0);
            mma_commit(&s.f.mbar);
        }
        // the output layer's gradient on CUDA cores while the tensor core works
        if (ok) {
            const float4 *hz = reinterpret_cast<const float4 *>(s.h2t[t % kH]);
            const float4 *dq = reinterpret_cast<const float4 *>(s.dzt[t / kH]);
            #pragma unroll 8
            for (int q = 0; q < kM / 4; ++q) {
                const float4 a = dq[q], b = hz[q];
                gw3 += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
            }
            if (t < kOut) {
                const float4 *dz = reinterpret_cast<const float4 *>(s.dzt[t]);
                #pragma unroll 8
                for (int q = 0; q < kM / 4; ++q) {
                    const float4 a = dz[q];
                    gb3 += (a.x + a.y) + (a.z + a.w);
                }
            }
        }
        if (ok) {
            ok = mbar_wait(&s.f.mbar, phase);
            phase ^= 1u;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (ok) {
            // dh1 / scale = [h1 > 0] (dh1 before the mask), over dh2 (its MMAs are done)
            float d1[kH];
            tmem_row64(tmem, 0, d1);
            #pragma unroll
            for (int c0 = 0; c0 < kH; c0 += 8) {
                const uint4 hv = *reinterpret_cast<const uint4 *>(s.f.h1 + cm_off(t, c0, kN2 / 8));
                const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
                #pragma unroll
                for (int j = 0; j < 8; ++j) {
                    // h1 >= 0 after the ReLU: a BF16 with any magnitude bit set is positive
                    const bool on = ((hw[j >> 1] >> (16 * (j & 1))) & 0x7fffu) != 0u;
                    d1[c0 + j] = on ? d1[c0 + j] : 0.0f;
                }
                store_row8(s.dh, t, c0, kH / 8, d1 + c0);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        ok = __syncthreads_and(ok);
        if (ok && t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            // dW1 | db1 += (dh1 / scale)^T [x | 1] over the tile's rows
            #pragma unroll
            for (int kb = 0; kb < kM / 16; ++kb)
                mma_bf16(tmem + kColW1, smem_desc_mn(smem_addr(s.dh) + kb * 2 * kDhK, kDhK, 128),
                         smem_desc_mn(smem_addr(s.f.x) + kb * 2 * kXK, kXK, 128), idesc_bf16_mn(kM, kN1),
                         !first || kb > 0);
            mma_commit(&s.f.mbar);
        }
        if (ok) {
            ok = mbar_wait(&s.f.mbar, phase);
            phase ^= 1u;
        }
        first = false;
        asm volatile("tcgen05.fence::before_thread_sync;");
        ok = __syncthreads_and(ok);
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok && !first) {
        // the weight sums: rows (TMEM lanes) 0-63 hold the layer's outputs (warps 0 and 1)
        float v[kN2];
        const uint32_t lane_base = (uint32_t)((t >> 5) * 32) << 16;
        #pragma unroll
        for (int c = 0; c < kN2; c += 16) tmem_ld16(tmem + lane_base + (uint32_t)(kColW2 + c), v + c);
        float u[kN1];
        #pragma unroll
        for (int c = 0; c < kN1; c += 16) tmem_ld16(tmem + lane_base + (uint32_t)(kColW1 + c), u + c);
        if (t < kH) {
            #pragma unroll
            for (int c = 0; c < kH; ++c) atomicAdd(&grad[kW2 + t * kH + c], v[c] * scale);
            atomicAdd(&grad[kB2 + t], v[kH] * scale);
            #pragma unroll
            for (int c = 0; c < kIn; ++c) atomicAdd(&grad[kW1 + t * kIn + c], u[c] * scale);
            atomicAdd(&grad[kB1 + t], u[kIn] * scale);
        }
    }
    if (ok) {
        atomicAdd(&grad[kW3 + t], gw3);
        if (t < kOut) atomicAdd(&grad[kB3 + t], gb3);
        // BCE partial: warp sums, then one atomic per CTA
        float lv = (float)lsum;
        #pragma unroll
        for (int off = 16; off > 0; off >>= 1) lv += __shfl_xor_sync(0xffffffffu, lv, off);
        if ((t & 31) == 0) s.red[t >> 5] = lv;
    }
    __syncthreads();
    if (ok && t == 0) {
        float a = 0.f;
        for (int i = 0; i < kM / 32; ++i) a += s.red[i];
        atomicAdd(loss, a * scale);
    }
    mlp_finish(s.f, ok, phase, status, kTrainCols);
}

// Per-Gaussian inputs of the predictor (planes of ld), from the parameters,
// the lifecycle accumulators and the ring of per-view maximum blend weights:
//  0 opacity sigmoid(logit)       1-3 log-scales
//  4 log(1 + views seen)          5 log(1 + 1e4 * accumulated ||dL/d(u,v)||)
//  6-13 max T*alpha of the last 8 views, most recent first (ring slot head, head-1, ...)
//  14 log(1 + distance from the mean to the camera centre)
//  15 log(1 + mean |Omega_v| over the views seen)
__global__ void __launch_bounds__(256) k_mlp_features(const float *__restrict__ P, long long n, long long ld,
                                                       const float *__restrict__ st, long long sld,
                                                       const float *__restrict__ ring, int head, float cx, float cy,
                                                       float cz, float *__restrict__ feat) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const float views = st[5 * sld + g];
    const float dx = P[0 * ld + g] - cx, dy = P[1 * ld + g] - cy, dz = P[2 * ld + g] - cz;
    feat[0 * ld + g] = 1.0f / (1.0f + expf(-P[10 * ld + g]));
    feat[1 * ld + g] = P[3 * ld + g];
    feat[2 * ld + g] = P[4 * ld + g];
    feat[3 * ld + g] = P[5 * ld + g];
    feat[4 * ld + g] = log1pf(views);
    feat[5 * ld + g] = log1pf(1.0e4f * st[4 * sld + g]);
    #pragma unroll
    for (int j = 0; j < kRing; ++j) feat[(6 + j) * ld + g] = ring[(long long)((head - j + kRing) % kRing) * ld + g];
    feat[14 * ld + g] = log1pf(sqrtf(dx * dx + dy * dy + dz * dz));
    feat[15 * ld + g] = log1pf(st[0 * sld + g] / fmaxf(views, 1.0f));
}

// ring[slot] = max T*alpha accumulated since the last push; the accumulator restarts at 0.
__global__ void __launch_bounds__(256) k_mlp_push_blend(float *__restrict__ st, long long sld, long long n,
                                                         float *__restrict__ ring, long long ld, int slot) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    ring[(long long)slot * ld + g] = st[3 * sld + g];
    st[3 * sld + g] = 0.0f;
}

__global__ void __launch_bounds__(256) k_mlp_adam(float *__restrict__ w, const float *__restrict__ g,
                                                   float *__restrict__ m, float *__restrict__ v, float lr, float b1,
                                                   float b2, float eps, float inv_bc1, float inv_sqrt_bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNW) return;
    const float gg = g[i];
    const float mm = b1 * m[i] + (1.0f - b1) * gg, vv = b2 * v[i] + (1.0f - b2) * gg * gg;
    m[i] = mm;
    v[i] = vv;
    w[i] -= lr * (mm * inv_bc1) / (sqrtf(vv) * inv_sqrt_bc2 + eps);
}

int mlp_num_weights() { return kNW; }

static int sm_count() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

cudaError_t launch_mlp_forward(const float *feat, long long n, long long ld, const float *w, float *prob,
                               uint8_t *densify, uint8_t *prune, int *status, long long max_polls, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    // four CTAs per SM fill the SM's 512 TMEM columns (128 each)
    const long long grid = std::min<long long>(ceil_div(n, (long long)kM), 4ll * sm_count());
    k_mlp_forward<<<(unsigned)grid, kM, 0, s>>>(feat, n, ld, w, prob, densify, prune, status,
                                                max_polls < 0 ? kSpin : max_polls);
    return cudaGetLastError();
}

cudaError_t launch_mlp_train(const float *feat, const uint8_t *y_densify, const uint8_t *y_prune, long long n,
                             long long ld, const float *w, float *grad, float *loss, int *status, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = sizeof(MlpTrainSmem) + 1024;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * kNW, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    // two CTAs per SM (shared memory and TMEM: 2 x 256 columns)
    const long long grid = std::min<long long>(ceil_div(n, (long long)kM), 2ll * sm_count());
    k_mlp_train<<<(unsigned)grid, kM, smem, s>>>(feat, y_densify, y_prune, n, ld, w, grad, loss, status);
    return cudaGetLastError();
}

cudaError_t launch_mlp_features(const float *P, long long n, long long ld, const float *stats, long long sld,
                                const float *ring, int head, const float cam[3], float *feat, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_mlp_features<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(P, n, ld, stats, sld, ring, head, cam[0], cam[1], cam[2],
                                                               feat);
    return cudaGetLastError();
}

cudaError_t launch_mlp_push_blend(float *stats, long long sld, long long n, float *ring, long long ld, int slot,
                                  cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_mlp_push_blend<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(stats, sld, n, ring, ld, slot);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float *w, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                            long long step, cudaStream_t s) {
    const double bc1 = 1.0 - pow((double)b1, (double)step), bc2 = 1.0 - pow((double)b2, (double)step);
    k_mlp_adam<<<(unsigned)ceil_div(kNW, 256), 256, 0, s>>>(w, g, m, v, lr, b1, b2, eps, (float)(1.0 / bc1),
                                                             (float)(1.0 / sqrt(bc2)));
    return cudaGetLastError();
}

}  // namespace gs
