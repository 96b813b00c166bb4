// anchors.cu -- Scaffold-GS anchors (Supp. D.1 decoding, Supp. D.3 LoD
// mask): each anchor's decoder turns (feature, view direction, log(1 +
// distance)) into its K = 10 Gaussians, written as SH-degree-0 Gaussians for
// the rasteriser; the backward takes the rasteriser's parameter gradients back
// to the anchors and the decoder's weights; a flat Adam updates both.
//
// Both directions run the decoder's two layers on the 5th-generation tensor
// cores (BF16 operands in shared memory, FP32 sums in tensor memory), one
// 128-anchor tile per MMA; the per-Gaussian activations, the decoded
// parameters and dL/dz are FP32 on CUDA cores, one thread per anchor row.
// Slot (k, i) of the output is column k ld + i of every plane (coalesced per
// k).  Dropped Gaussians (outside the level's distance band, opacity <= 0) get
// a placeholder whose opacity logit (-30) the projection culls.  Every
// mbarrier wait is bounded; on a timeout a kernel flags the status word,
// stops issuing and still frees its tensor memory.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>

#include "gs_internal.cuh"
#include "gs_kernels.h"
#include "tcgen05.cuh"

namespace gs {

namespace {

constexpr int kAK = GS_ANCHOR_K, kAF = GS_ANCHOR_FEAT, kAIn = kAF + 4, kAH = 64, kAOut = 14 * kAK;
constexpr int kAW1 = 0, kAB1 = kAW1 + kAH * kAIn, kAW2 = kAB1 + kAH, kAB2 = kAW2 + kAOut * kAH,
              kANW = kAB2 + kAOut;
static_assert(kANW == GS_ANCHOR_WEIGHTS, "decoder weight count");
static_assert(kAIn % 4 == 0 && kAH % 4 == 0 && kAW2 % 4 == 0, "weight rows on 16-byte boundaries");
constexpr int kPlaneLogL = kAF, kPlaneOffs = kAF + 3;
static_assert(kPlaneOffs + 3 * kAK == GS_ANCHOR_PLANES, "anchor planes");
constexpr float kY00 = 0.28209479177387814f, kInvY00 = 1.0f / kY00;
constexpr float kDeadLogit = -30.0f;

// sigmoid and log(sigmoid) from the hardware exp2 / log2 approximations (__expf, __logf: a few
// units in the last place, well inside the decoded parameters' FP32 tolerance); the limits hold
// for either sign (1 / inf = 0; log(1 + e^-|z|) never overflows)
__device__ __forceinline__ float sigmoidf(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }

__device__ __forceinline__ float log_sigmoidf(float z) { return fminf(z, 0.0f) - __logf(1.0f + __expf(-fabsf(z))); }

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

// ---------------------------------------------------------------------------
// Tensor-core decoder.  A tile is 128 anchors = the M of one tcgen05.mma.
// Two threads own each anchor row r (threads r and r + 128, i.e. warps w and
// w + 4, which read the same TMEM lanes 32 (w % 4) ..): each takes half of
// the row's columns or Gaussian slots in every per-row phase.  Operands are
// BF16 in shared memory (K-major, no swizzle: 8x8 core matrices of 128
// bytes), sums FP32 in TMEM; the biases are added in FP32 when a row is read
// back.  The 140 outputs sit in 16-column slots (Gaussian k at columns 16 k ..
// 16 k + 13, two zero columns), so one 16-column TMEM load holds one
// Gaussian.  Opacity: a = tanh(z) > 0 iff z > 0, and logit(tanh z) =
// log(expm1(2 z) / 2).
// ---------------------------------------------------------------------------
constexpr int kM = 128;                   // anchors per tile
constexpr int kThreads = 2 * kM;          // two threads per anchor row
constexpr int kHS = kAK / 2, kHF = kAF / 2, kHH = kAH / 2;  // slots, features, hidden units per half
constexpr int kSlot = 16, kOutP = kSlot * kAK;  // padded outputs (160)
constexpr int kXC = 48, kXG = kXC / 8;    // x: 36 inputs, the constant 1 (column 36), zeros
constexpr int kHC = 80, kHG = kHC / 8;    // backward h: 64 activations, the constant 1 (column 64), zeros
constexpr int kOG = kOutP / 8;            // core matrices along the padded outputs
static_assert(kAIn < kXC && kOutP <= 256 && kOutP % 16 == 0 && 2 * kHS == kAK && kHF == 16 && kHH == 32,
              "tile shapes");

// TMEM lane base of the calling warp (warps w and w + 4 share lanes 32 (w % 4) ..).
__device__ __forceinline__ uint32_t lane_base() { return (uint32_t)(((threadIdx.x >> 5) & 3) * 32) << 16; }

struct DecWeights {
    alignas(128) __nv_bfloat16 w1[kAH * kXC];    // B of layer 1: [n = o][k = c], c >= 36 zero
    alignas(128) __nv_bfloat16 w2[kOutP * kAH];  // B of layer 2: [n = 16 k + j][k = c], j >= 14 zero
    float b1[kAH], b2[kOutP];                     // FP32 biases
};

// Eight consecutive FP32 weights (16-byte aligned) or zeros.
__device__ __forceinline__ void load8(const float *__restrict__ src, bool lo, bool hi, float *v) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 a = lo ? __ldg(reinterpret_cast<const float4 *>(src)) : z;
    const float4 b = hi ? __ldg(reinterpret_cast<const float4 *>(src) + 1) : z;
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// The BF16 operand images of W1 and W2 and the FP32 biases, from 16-byte loads (every row of
// W1 (36 floats) and W2 (64) starts on a 16-byte boundary).
__device__ void stage_weights(DecWeights &s, const float *__restrict__ w) {
    #pragma unroll
    for (int r = 0; r < (kAH * kXG + kThreads - 1) / kThreads; ++r) {
        const int u = threadIdx.x + kThreads * r;
        if (u < kAH * kXG) {
            const int o = u / kXG, c0 = 8 * (u % kXG);
            float v[8];
            load8(w + kAW1 + o * kAIn + c0, c0 + 4 <= kAIn, c0 + 8 <= kAIn, v);
            store_row8(s.w1, o, c0, kXG, v);
        }
    }
    static_assert(kOutP * (kAH / 8) % kThreads == 0, "W2 chunks per thread");
    #pragma unroll
    for (int r = 0; r < kOutP * (kAH / 8) / kThreads; ++r) {
        const int u = threadIdx.x + kThreads * r;
        const int q = u / (kAH / 8), c0 = 8 * (u % (kAH / 8)), k = q / kSlot, j = q % kSlot;
        float v[8];
        load8(w + kAW2 + (14 * k + j) * kAH + c0, j < 14, j < 14, v);
        store_row8(s.w2, q, c0, kAH / 8, v);
    }
    for (int i = threadIdx.x; i < kAH; i += kThreads) s.b1[i] = w[kAB1 + i];
    for (int i = threadIdx.x; i < kOutP; i += kThreads) {
        const int k = i / kSlot, j = i % kSlot;
        s.b2[i] = j < 14 ? w[kAB2 + 14 * k + j] : 0.0f;
    }
}

// TMEM allocation and the mbarrier; every thread sees both on return.
__device__ void tc_begin(uint64_t *mbar, uint32_t *slot, uint32_t cols) {
    tmem_alloc(slot, cols);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
}

// After a timed-out wait nothing more is issued; the product committed last
// (parity phase ^ 1) gets one more bounded wait before the TMEM is freed.
__device__ void tc_end(uint64_t *mbar, uint32_t tmem, uint32_t cols, bool ok, uint32_t phase, int *status) {
    if (!ok) {
        mbar_wait(mbar, phase ^ 1u);
        if (threadIdx.x == 0 && status) atomicOr(status, 1 << GS_ERR_TIMEOUT);
    }
    tmem_free(tmem, cols);
}

// Wait for the MMAs thread 0 committed (warp-uniform result).
__device__ __forceinline__ bool tc_wait(uint64_t *mbar, uint32_t &phase, long long polls) {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(mbar, phase, polls));
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;");
    return ok;
}

// Thread-written operands visible to the tensor core, TMEM reads finished, then a CTA barrier.
__device__ __forceinline__ bool tc_sync(bool ok) {
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    return __syncthreads_and(ok);
}

// This half's loads of one anchor's inputs (issued a tile ahead): its 16 features, the
// position, the log-scales and the level.
struct AnchorIn {
    float f[kHF], p[3], L[3];
    int lv;
};

__device__ __forceinline__ void load_anchor(AnchorIn &in, const float *__restrict__ A, const float *__restrict__ pos,
                                            const int *__restrict__ level, long long n, long long ld, long long i,
                                            int half) {
    const bool valid = i < n;
    #pragma unroll
    for (int c = 0; c < kHF; ++c) in.f[c] = valid ? A[(kHF * half + c) * ld + i] : 0.0f;
    #pragma unroll
    for (int c = 0; c < 3; ++c) {
        in.p[c] = valid ? pos[c * ld + i] : 0.0f;
        in.L[c] = valid ? A[(kPlaneLogL + c) * ld + i] : 0.0f;
    }
    in.lv = valid ? level[i] : -1;
}

// This half's columns of the tile row of x as the tensor core reads it: (feature,
// direction, log(1 + d)) of an active anchor (zeros otherwise), the constant 1, zeros.
// Half 0 writes columns 0-15, half 1 columns 16-47.  Returns whether the anchor is active.
__device__ __forceinline__ bool stage_x(__nv_bfloat16 *xs, int row, int half, const AnchorIn &in,
                                        const AnchorView &v) {
    const float dx = in.p[0] - v.c[0], dy = in.p[1] - v.c[1], dz = in.p[2] - v.c[2];
    const float d = sqrtf(dx * dx + dy * dy + dz * dz);
    const bool M = band_active(v, in.lv, d);
    float x[8];
    #pragma unroll
    for (int c0 = 0; c0 < kHF; c0 += 8) {
        #pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = M ? in.f[c0 + j] : 0.0f;
        store_row8(xs, row, kHF * half + c0, kXG, x);
    }
    if (half) {
        const float r = 1.0f / d;
        x[0] = M ? dx * r : 0.0f;
        x[1] = M ? dy * r : 0.0f;
        x[2] = M ? dz * r : 0.0f;
        x[3] = M ? log1pf(d) : 0.0f;
        x[4] = 1.0f;
        x[5] = x[6] = x[7] = 0.0f;
        store_row8(xs, row, kAF, kXG, x);
        #pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = 0.0f;
        store_row8(xs, row, kAF + 8, kXG, x);
    }
    return M;
}

// Layer 1: D = X W1^T, three K = 16 steps.
__device__ __forceinline__ void issue_layer1(uint32_t tmem, const __nv_bfloat16 *xs, const DecWeights &wt) {
    #pragma unroll
    for (int kb = 0; kb < kXC / 16; ++kb)
        mma_bf16(tmem, smem_desc(smem_addr(xs) + kb * 256, 128, kXG * 128),
                 smem_desc(smem_addr(wt.w1) + kb * 256, 128, kXG * 128), idesc_bf16(kM, kAH), kb > 0);
}

// Layer 2: D = H W2^T (N = 160 padded outputs), four K = 16 steps over the 64 activations.
__device__ __forceinline__ void issue_layer2(uint32_t tmem, const __nv_bfloat16 *hs, int hg, const DecWeights &wt) {
    #pragma unroll
    for (int kb = 0; kb < kAH / 16; ++kb)
        mma_bf16(tmem, smem_desc(smem_addr(hs) + kb * 256, 128, hg * 128),
                 smem_desc(smem_addr(wt.w2) + kb * 256, 128, (kAH / 8) * 128), idesc_bf16(kM, kOutP), kb > 0);
}

// Slot k's 14 outputs (plus two zero columns) of this thread's row, biases added; taddr =
// the TMEM base + this warp's lane base + the outputs' first column.
__device__ __forceinline__ void read_slot(uint32_t taddr, const DecWeights &wt, int k, float *z) {
    tmem_ld16(taddr + (uint32_t)(kSlot * k), z);
    #pragma unroll
    for (int j = 0; j < 14; ++j) z[j] += wt.b2[kSlot * k + j];
}

// The row's hidden pre-activations of this half (columns 32 half .. + 31), bias added.
__device__ __forceinline__ void read_hidden(uint32_t taddr, const DecWeights &wt, int half, float *pre) {
    tmem_ld16(taddr + (uint32_t)(kHH * half), pre);
    tmem_ld16(taddr + (uint32_t)(kHH * half + 16), pre + 16);
    #pragma unroll
    for (int c = 0; c < kHH; ++c) pre[c] += wt.b1[kHH * half + c];
}

struct DecSmem {
    DecWeights wt;
    alignas(128) __nv_bfloat16 x[kM * kXC];  // A of layer 1: [row][c]
    alignas(128) __nv_bfloat16 h[kM * kAH];  // A of layer 2: [row][c]
    uint64_t mbar;
    uint32_t tmem;
};
constexpr uint32_t kDecCols = 256;  // layer 1 in [0, 64), layer 2 in [64, 224)
constexpr int kDecZ = 64;
static_assert(kDecZ + kOutP <= (int)kDecCols, "decode TMEM columns");
static_assert(2 * (sizeof(DecSmem) + 1024) <= 228 * 1024, "two decode CTAs per SM");

__global__ void __launch_bounds__(kThreads, 2) k_anchor_decode(const float *__restrict__ A,
                                                                const float *__restrict__ pos,
                                                                const int *__restrict__ level, long long n,
                                                                long long ld, const float *__restrict__ w,
                                                                const __grid_constant__ AnchorView v,
                                                                float *__restrict__ G, long long gld,
                                                                int *__restrict__ status, long long polls) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    DecSmem &s = *reinterpret_cast<DecSmem *>(smem_raw);
    stage_weights(s.wt, w);
    tc_begin(&s.mbar, &s.tmem, kDecCols);
    const int t = threadIdx.x, row = t & (kM - 1), half = t >> 7;
    const uint32_t tmem = s.tmem, lb = lane_base();
    uint32_t phase = 0;
    bool ok = true;
    const long long tiles = ceil_div(ld, (long long)kM);
    AnchorIn in;
    if ((long long)blockIdx.x < tiles) load_anchor(in, A, pos, level, n, ld, (long long)blockIdx.x * kM + row, half);
    for (long long tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const long long i = tile * kM + row;
        const bool M = stage_x(s.x, row, half, in, v);
        float p[3], L[3], l[3], off[3 * kHS];
        #pragma unroll
        for (int c = 0; c < 3; ++c) { p[c] = in.p[c]; L[c] = in.L[c]; }
        if (tile + gridDim.x < tiles) load_anchor(in, A, pos, level, n, ld, (tile + gridDim.x) * kM + row, half);
        // this half's offsets arrive while the two layers run
        #pragma unroll
        for (int c = 0; c < 3 * kHS; ++c) off[c] = M ? A[(kPlaneOffs + 3 * kHS * half + c) * ld + i] : 0.0f;
        #pragma unroll
        for (int c = 0; c < 3; ++c) l[c] = expf(L[c]);
        ok = tc_sync(ok);
        if (ok && t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            issue_layer1(tmem, s.x, s.wt);
            mma_commit(&s.mbar);
        }
        if (ok) ok = tc_wait(&s.mbar, phase, polls);
        if (ok) {
            float hv[kHH];
            read_hidden(tmem + lb, s.wt, half, hv);
            #pragma unroll
            for (int c = 0; c < kHH; ++c) hv[c] = fmaxf(hv[c], 0.0f);
            #pragma unroll
            for (int c0 = 0; c0 < kHH; c0 += 8) store_row8(s.h, row, kHH * half + c0, kAH / 8, hv + c0);
        }
        ok = tc_sync(ok);
        if (ok && t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            issue_layer2(tmem + kDecZ, s.h, kAH / 8, s.wt);
            mma_commit(&s.mbar);
        }
        if (ok) ok = tc_wait(&s.mbar, phase, polls);
        if (ok) {
            #pragma unroll
            for (int kk = 0; kk < kHS; ++kk) {
                const int k = kHS * half + kk;
                float z[16];
                read_slot(tmem + lb + kDecZ, s.wt, k, z);
                if (i >= ld) continue;
                const long long col = k * ld + i;
                if (!M || !(z[3] > 0.0f)) {
                    write_dead(G, gld, col, p, L);
                    continue;
                }
                #pragma unroll
                for (int c = 0; c < 3; ++c) {
                    G[c * gld + col] = p[c] + (off[3 * kk + c] + z[11 + c]) * l[c];  // mean
                    G[(3 + c) * gld + col] = L[c] + log_sigmoidf(z[8 + c]);          // log(l ds)
                    G[(11 + c) * gld + col] = (sigmoidf(z[c]) - 0.5f) * kInvY00;       // colour
                }
                G[6 * gld + col] = 1.0f + z[4];
                G[7 * gld + col] = z[5];
                G[8 * gld + col] = z[6];
                G[9 * gld + col] = z[7];
                G[10 * gld + col] = logf(0.5f * expm1f(2.0f * z[3]));  // logit(tanh z)
            }
        }
    }
    tc_end(&s.mbar, tmem, kDecCols, ok, phase, status);
}

// Backward.  Per tile, after the forward's two layers (the activations h kept
// in shared memory with a constant-1 column, their ReLU mask in registers):
//   dz [row][160] from the decoded Gaussians' gradients (FP32 on CUDA cores,
//     with the anchors' offset and log-scale gradients), stored BF16;
//   dh = dz W2                      [128 x 64]  (K = 160),
//   dW2 | db2 += [h | 1]^T dz        over the tile's rows, [80 x 160] kept in TMEM;
//   dp = [pre > 0] dh, stored BF16;
//   df = dp W1 (feature columns)    [128 x 32]  (K = 64),
//   dW1 | db1 += dp^T [x | 1]        over the tile's rows, [64 x 48] kept in TMEM.
// The weight sums use M = 128 with the first 65 (64) rows meaningful: the
// remaining rows of D are never read, and their A rows read whatever shared
// memory follows the operand.  The weight sums leave TMEM once, at the end,
// as one FP32 atomic per weight per CTA.
struct BwdSmem {
    alignas(128) __nv_bfloat16 dz[kM * kOutP];  // [row][16 k + j]: dL/dz (A of dh K-major, B of dW2 MN-major)
    alignas(128) __nv_bfloat16 h[kM * kHC];     // [row][c]: h, 1, zeros (A of layer 2, A of dW2 MN-major)
    alignas(128) __nv_bfloat16 dp[kM * kAH];    // [row][o]: dL/dpre (A of df K-major, A of dW1 MN-major)
    alignas(128) __nv_bfloat16 x[kM * kXC];     // [row][c]: x, 1, zeros (A of layer 1, B of dW1 MN-major)
    alignas(128) __nv_bfloat16 w2t[kAH * kOutP];  // B of dh: [n = c][k = 16 k + j] = W2^T
    alignas(128) __nv_bfloat16 w1t[kAF * kAH];    // B of df: [n = feature c][k = o] = W1^T
    DecWeights wt;
    float gLx[3][kM];  // half 1's share of the log-scale gradients
    uint64_t mbar;
    uint32_t tmem;
};
// TMEM columns: pre then dh in [0, 64); z then df in [64, 224); dW2 | db2 in
// [224, 384); dW1 | db1 in [384, 432).
constexpr uint32_t kBwdCols = 512;
constexpr int kColZ = 64, kColDF = 64, kColW2 = 224, kColW1 = 384;
static_assert(kColZ + kOutP <= kColW2 && kColW2 + kOutP <= kColW1 && kColW1 + kXC <= (int)kBwdCols, "TMEM columns");
// Byte strides of the MN-major reads (8-row groups of the K-major arrays).
constexpr uint32_t kDzK = kOG * 128, kHK = kHG * 128, kDpK = (kAH / 8) * 128, kXK = kXG * 128;
// Every descriptor read stays inside the CTA's shared memory whichever of the
// two strides the hardware takes as the K one: the largest byte reached from
// an operand's start is (last K step) + (groups - 1) x the larger stride +
// one group x the other + 127.
static_assert(offsetof(BwdSmem, dz) + 7 * 2 * kDzK + (kOG - 1) * kDzK + 128 + 127 < sizeof(BwdSmem), "dz read");
static_assert(offsetof(BwdSmem, h) + 7 * 2 * kHK + 15 * kHK + 128 + 127 < sizeof(BwdSmem), "h read");
static_assert(offsetof(BwdSmem, dp) + 7 * 2 * kDpK + 15 * kDpK + 128 + 127 < sizeof(BwdSmem), "dp read");
static_assert(offsetof(BwdSmem, x) + 7 * 2 * kXK + (kXG - 1) * kXK + 128 + 127 < sizeof(BwdSmem), "x read");
static_assert(sizeof(BwdSmem) + 1024 <= 227 * 1024, "backward shared memory");

__global__ void __launch_bounds__(kThreads, 1) k_anchor_decode_bwd(const float *__restrict__ A,
                                                                    const float *__restrict__ pos,
                                                                    const int *__restrict__ level, long long n,
                                                                    long long ld, const float *__restrict__ w,
                                                                    const __grid_constant__ AnchorView v,
                                                                    const float *__restrict__ GG, long long gld,
                                                                    float *__restrict__ gA, float *__restrict__ gw,
                                                                    int *__restrict__ status, long long polls) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    BwdSmem &s = *reinterpret_cast<BwdSmem *>(smem_raw);
    stage_weights(s.wt, w);
    const int t = threadIdx.x, row = t & (kM - 1), half = t >> 7;
    {
        // the transposed images from FP32 copies of W2 and W1 in the (not yet used) dz and h arrays
        float *w2f = reinterpret_cast<float *>(s.dz), *w1f = reinterpret_cast<float *>(s.h);
        static_assert(sizeof(float) * kAOut * kAH <= sizeof(s.dz) && sizeof(float) * kAH * kAIn <= sizeof(s.h),
                      "weight scratch");
        for (int u = t; u < kAOut * kAH / 4; u += kThreads)
            reinterpret_cast<float4 *>(w2f)[u] = __ldg(reinterpret_cast<const float4 *>(w + kAW2) + u);
        for (int u = t; u < kAH * kAIn / 4; u += kThreads)
            reinterpret_cast<float4 *>(w1f)[u] = __ldg(reinterpret_cast<const float4 *>(w + kAW1) + u);
        __syncthreads();
        for (int u = t; u < kAH * kOG; u += kThreads) {
            const int c = u % kAH, q0 = 8 * (u / kAH);  // a warp reads 32 consecutive columns c
            float vv[8];
            #pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                const int k = (q0 + jj) / kSlot, j = (q0 + jj) % kSlot;
                vv[jj] = j < 14 ? w2f[(14 * k + j) * kAH + c] : 0.0f;
            }
            store_row8(s.w2t, c, q0, kOG, vv);
        }
        for (int u = t; u < kAF * (kAH / 8); u += kThreads) {
            const int c = u % kAF, o0 = 8 * (u / kAF);
            float vv[8];
            #pragma unroll
            for (int jj = 0; jj < 8; ++jj) vv[jj] = w1f[(o0 + jj) * kAIn + c];
            store_row8(s.w1t, c, o0, kAH / 8, vv);
        }
        __syncthreads();  // the scratch is read before h's constant columns overwrite it
        // h's constant columns: 1 (the bias gradient; half 0), then zeros (half 1)
        const float one[8] = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, zero[8] = {};
        store_row8(s.h, row, kAH + 8 * half, kHG, half ? zero : one);
    }
    tc_begin(&s.mbar, &s.tmem, kBwdCols);
    const uint32_t tmem = s.tmem, lb = lane_base();
    uint32_t phase = 0;
    bool ok = true, first = true;
    const long long tiles = ceil_div(n, (long long)kM);
    AnchorIn in;
    if ((long long)blockIdx.x < tiles) load_anchor(in, A, pos, level, n, ld, (long long)blockIdx.x * kM + row, half);
    for (long long tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const long long i = tile * kM + row;
        const bool valid = i < n;
        const bool M = stage_x(s.x, row, half, in, v);
        float l[3], off[3 * kHS];
        #pragma unroll
        for (int c = 0; c < 3; ++c) l[c] = in.L[c];
        if (tile + gridDim.x < tiles) load_anchor(in, A, pos, level, n, ld, (tile + gridDim.x) * kM + row, half);
        // this half's offsets and the incoming gradients of its Gaussians arrive while the two
        // layers run (70 loads in flight per thread)
        #pragma unroll
        for (int c = 0; c < 3 * kHS; ++c) off[c] = M ? A[(kPlaneOffs + 3 * kHS * half + c) * ld + i] : 0.0f;
        float gin[kHS][14];
        #pragma unroll
        for (int kk = 0; kk < kHS; ++kk) {
            #pragma unroll
            for (int j = 0; j < 14; ++j) gin[kk][j] = M ? GG[j * gld + (kHS * half + kk) * ld + i] : 0.0f;
        }
        #pragma unroll
        for (int c = 0; c < 3; ++c) l[c] = expf(l[c]);
        ok = tc_sync(ok);
        if (ok && t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            issue_layer1(tmem, s.x, s.wt);
            mma_commit(&s.mbar);
        }
        if (ok) ok = tc_wait(&s.mbar, phase, polls);
        uint32_t on = 0u;  // ReLU mask of this half's 32 pre-activations
        if (ok) {
            float hv[kHH];
            read_hidden(tmem + lb, s.wt, half, hv);
            #pragma unroll
            for (int c = 0; c < kHH; ++c) {
                const bool act = M && hv[c] > 0.0f;
                on |= act ? 1u << c : 0u;
                hv[c] = act ? hv[c] : 0.0f;
            }
            #pragma unroll
            for (int c0 = 0; c0 < kHH; c0 += 8) store_row8(s.h, row, kHH * half + c0, kHG, hv + c0);
        }
        ok = tc_sync(ok);
        if (ok && t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            issue_layer2(tmem + kColZ, s.h, kHG, s.wt);
            mma_commit(&s.mbar);
        }
        if (ok) ok = tc_wait(&s.mbar, phase, polls);
        if (ok) {
            // dL/dz of this half's kept Gaussians; their offset gradients and the log-scale ones
            float gL[3] = {0.0f, 0.0f, 0.0f};
            #pragma unroll
            for (int kk = 0; kk < kHS; ++kk) {
                const int k = kHS * half + kk;
                const float *g = gin[kk];
                float z[16], dz[16];
                read_slot(tmem + lb + kColZ, s.wt, k, z);
                #pragma unroll
                for (int j = 0; j < 16; ++j) dz[j] = 0.0f;
                float gO[3] = {0.0f, 0.0f, 0.0f};
                if (M && z[3] > 0.0f) {
                    #pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float O = off[3 * kk + c] + z[11 + c];
                        dz[11 + c] = g[c] * l[c];
                        gO[c] = g[c] * l[c];
                        gL[c] += g[c] * O * l[c] + g[3 + c];
                        dz[8 + c] = g[3 + c] * (1.0f - sigmoidf(z[8 + c]));
                        const float sc = sigmoidf(z[c]);
                        dz[c] = g[11 + c] * sc * (1.0f - sc) * kInvY00;
                    }
                    #pragma unroll
                    for (int c = 0; c < 4; ++c) dz[4 + c] = g[6 + c];
                    // d logit(tanh z) / dz = (1 + a) / a = 2 + 2 / expm1(2 z)
                    dz[3] = g[10] * (2.0f + 2.0f / expm1f(2.0f * z[3]));
                }
                store_row8(s.dz, row, kSlot * k, kOG, dz);
                store_row8(s.dz, row, kSlot * k + 8, kOG, dz + 8);
                if (valid) {
                    #pragma unroll
                    for (int c = 0; c < 3; ++c) gA[(kPlaneOffs + 3 * k + c) * ld + i] = gO[c];
                }
            }
            if (half) {
                #pragma unroll
                for (int c = 0; c < 3; ++c) s.gLx[c][row] = gL[c];
            } else {
                #pragma unroll
                for (int c = 0; c < 3; ++c) l[c] = gL[c];  // l is not needed any more
            }
        }
        ok = tc_sync(ok);
        if (ok && t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            // dh = dz W2 -> columns [0, 64), ten K = 16 steps
            #pragma unroll
            for (int kb = 0; kb < kOutP / 16; ++kb)
                mma_bf16(tmem, smem_desc(smem_addr(s.dz) + kb * 256, 128, kDzK),
                         smem_desc(smem_addr(s.w2t) + kb * 256, 128, kDzK), idesc_bf16(kM, kAH), kb > 0);
            // dW2 | db2 += [h | 1]^T dz over the tile's rows, 16 rows per step
            #pragma unroll
            for (int kb = 0; kb < kM / 16; ++kb)
                mma_bf16(tmem + kColW2, smem_desc_mn(smem_addr(s.h) + kb * 2 * kHK, kHK, 128),
                         smem_desc_mn(smem_addr(s.dz) + kb * 2 * kDzK, kDzK, 128), idesc_bf16_mn(kM, kOutP),
                         !first || kb > 0);
            mma_commit(&s.mbar);
        }
        if (ok && !half && valid) {
            #pragma unroll
            for (int c = 0; c < 3; ++c) gA[(kPlaneLogL + c) * ld + i] = l[c] + s.gLx[c][row];
        }
        if (ok) ok = tc_wait(&s.mbar, phase, polls);
        if (ok) {
            float d1[kHH];
            tmem_ld16(tmem + lb + (uint32_t)(kHH * half), d1);
            tmem_ld16(tmem + lb + (uint32_t)(kHH * half + 16), d1 + 16);
            #pragma unroll
            for (int c = 0; c < kHH; ++c) d1[c] = (on >> c) & 1u ? d1[c] : 0.0f;
            #pragma unroll
            for (int c0 = 0; c0 < kHH; c0 += 8) store_row8(s.dp, row, kHH * half + c0, kAH / 8, d1 + c0);
        }
        ok = tc_sync(ok);
        if (ok && t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            // df = dp W1 over the feature inputs -> columns [64, 96), four K = 16 steps
            #pragma unroll
            for (int kb = 0; kb < kAH / 16; ++kb)
                mma_bf16(tmem + kColDF, smem_desc(smem_addr(s.dp) + kb * 256, 128, kDpK),
                         smem_desc(smem_addr(s.w1t) + kb * 256, 128, kDpK), idesc_bf16(kM, kAF), kb > 0);
            // dW1 | db1 += dp^T [x | 1] over the tile's rows
            #pragma unroll
            for (int kb = 0; kb < kM / 16; ++kb)
                mma_bf16(tmem + kColW1, smem_desc_mn(smem_addr(s.dp) + kb * 2 * kDpK, kDpK, 128),
                         smem_desc_mn(smem_addr(s.x) + kb * 2 * kXK, kXK, 128), idesc_bf16_mn(kM, kXC),
                         !first || kb > 0);
            mma_commit(&s.mbar);
        }
        if (ok) ok = tc_wait(&s.mbar, phase, polls);
        first = false;
        if (ok) {
            float df[kHF];
            tmem_ld16(tmem + lb + (uint32_t)(kColDF + kHF * half), df);
            if (valid) {
                #pragma unroll
                for (int c = 0; c < kHF; ++c) gA[(kHF * half + c) * ld + i] = df[c];
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        ok = __syncthreads_and(ok);
    }
    if (ok && !first) {
        // the weight sums: TMEM lane c < 64 holds W2[.][c] (lane 64: b2) and W1[c][.] (column 36:
        // b1); half 0 reads slots 0-4 and W1 columns 0-31, half 1 slots 5-9 and columns 32-47
        #pragma unroll
        for (int kk = 0; kk < kHS; ++kk) {
            const int k = kHS * half + kk;
            float u[16];
            tmem_ld16(tmem + lb + (uint32_t)(kColW2 + kSlot * k), u);
            if (row < kAH) {
                #pragma unroll
                for (int j = 0; j < 14; ++j) atomicAdd(&gw[kAW2 + (14 * k + j) * kAH + row], u[j]);
            } else if (row == kAH) {
                #pragma unroll
                for (int j = 0; j < 14; ++j) atomicAdd(&gw[kAB2 + 14 * k + j], u[j]);
            }
        }
        float u[32];
        if (half == 0) {
            tmem_ld16(tmem + lb + (uint32_t)kColW1, u);
            tmem_ld16(tmem + lb + (uint32_t)(kColW1 + 16), u + 16);
            if (row < kAH) {
                #pragma unroll
                for (int c = 0; c < 32; ++c) atomicAdd(&gw[kAW1 + row * kAIn + c], u[c]);
            }
        } else {
            tmem_ld16(tmem + lb + (uint32_t)(kColW1 + 32), u);
            if (row < kAH) {
                #pragma unroll
                for (int c = 32; c < kAIn; ++c) atomicAdd(&gw[kAW1 + row * kAIn + c], u[c - 32]);
                atomicAdd(&gw[kAB1 + row], u[kAIn - 32]);
            }
        }
    }
    tc_end(&s.mbar, tmem, kBwdCols, ok, phase, status);
}

__global__ void k_adam_flat(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long n, float lr, float b1, float b2, float eps, float bc1,
                            float bc2, const long long *__restrict__ step_dev) {
    if (step_dev) {  // bias corrections from the device step counter (graph replay)
        __shared__ float s_bc[2];
        if (threadIdx.x == 0) {
            adam_bias(b1, b2, *step_dev, s_bc[0], s_bc[1]);
        }
        __syncthreads();
        bc1 = s_bc[0];
        bc2 = s_bc[1];
    }
    // float4 where the four arrays allow it (the anchor planes and the decoder weights do),
    // with the SFU's square root and division as in the Gaussians' Adam
    const bool vec = ((((uintptr_t)p | (uintptr_t)g | (uintptr_t)m | (uintptr_t)v) & 15u) == 0) && (n & 3) == 0;
    const float ibc1 = 1.0f / bc1, isbc2 = rsqrtf(bc2);
    auto upd = [&](float &pi, float gi, float &mi, float &vi) {
        mi = b1 * mi + (1.0f - b1) * gi;
        vi = b2 * vi + (1.0f - b2) * gi * gi;
        float sq;
        asm("sqrt.approx.f32 %0, %1;" : "=f"(sq) : "f"(vi));
        pi -= __fdividef(lr * (mi * ibc1), sq * isbc2 + eps);
    };
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (vec) {
        float4 *p4 = reinterpret_cast<float4 *>(p), *m4 = reinterpret_cast<float4 *>(m);
        float4 *v4 = reinterpret_cast<float4 *>(v);
        const float4 *g4 = reinterpret_cast<const float4 *>(g);
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n / 4; i += stride) {
            float4 pp = p4[i], mm = m4[i], vv = v4[i];
            const float4 gg = g4[i];
            upd(pp.x, gg.x, mm.x, vv.x); upd(pp.y, gg.y, mm.y, vv.y);
            upd(pp.z, gg.z, mm.z, vv.z); upd(pp.w, gg.w, mm.w, vv.w);
            p4[i] = pp; m4[i] = mm; v4[i] = vv;
        }
    } else {
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            float pi = p[i], mi = m[i], vi = v[i];
            upd(pi, g[i], mi, vi);
            p[i] = pi; m[i] = mi; v[i] = vi;
        }
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
                                 const float *w, const AnchorView &v, float *G, long long gld, int *status,
                                 long long max_polls, cudaStream_t s) {
    if (ld <= 0) return cudaSuccess;
    const size_t smem = sizeof(DecSmem) + 1024;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_anchor_decode, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    // two CTAs per SM (2 x 256 TMEM columns)
    const long long grid = std::min<long long>(ceil_div(ld, (long long)kM), 2ll * sm_count_anchor());
    k_anchor_decode<<<(unsigned)grid, kThreads, smem, s>>>(A, pos, level, n, ld, w, v, G, gld, status,
                                                     max_polls < 0 ? kSpin : max_polls);
    return cudaGetLastError();
}

cudaError_t launch_anchor_decode_bwd(const float *A, const float *pos, const int *level, long long n, long long ld,
                                     const float *w, const AnchorView &v, const float *GG, long long gld, float *gA,
                                     float *gw, int *status, long long max_polls, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(gA, 0, sizeof(float) * GS_ANCHOR_PLANES * (size_t)ld, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(gw, 0, sizeof(float) * kANW, s);
    if (e != cudaSuccess || n <= 0) return e;
    const size_t smem = sizeof(BwdSmem) + 1024;
    static bool attr = false;
    if (!attr) {
        e = cudaFuncSetAttribute(k_anchor_decode_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    // one CTA per SM (512 TMEM columns)
    const long long grid = std::min<long long>(ceil_div(n, (long long)kM), (long long)sm_count_anchor());
    k_anchor_decode_bwd<<<(unsigned)grid, kThreads, smem, s>>>(A, pos, level, n, ld, w, v, GG, gld, gA, gw, status,
                                                         max_polls < 0 ? kSpin : max_polls);
    return cudaGetLastError();
}

cudaError_t launch_adam_flat(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                             float eps, long long step, const long long *step_dev, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const double st = step_dev ? 1.0 : (double)step;  // placeholder when the device counter is used
    const float bc1 = (float)(1.0 - std::pow((double)b1, st));
    const float bc2 = (float)(1.0 - std::pow((double)b2, st));
    const long long blocks = std::min<long long>(ceil_div(n, 256ll), 4096ll);
    k_adam_flat<<<(unsigned)blocks, 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2, step_dev);
    return cudaGetLastError();
}

}  // namespace gs
