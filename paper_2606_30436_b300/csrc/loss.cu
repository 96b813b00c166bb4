// loss.cu -- photometric loss L = (1 - lambda) L1 + lambda (1 - SSIM) and its
// gradient (Supp. D.4; lambda = 0.2 in the paper).  SSIM: 11x11 Gaussian
// window (sigma 1.5), zero padding, C1 = 0.01^2, C2 = 0.03^2.
//
// Forward: one CTA per 32x32 output tile and channel stages the tile plus a
// 5-pixel halo of both images in shared memory and forms the five windowed
// moments with separable 11-tap passes.  With s = SSIM(mu_x, mu_y, s_xx, s_yy,
// s_xy) the gradient with respect to the rendered image x is
//   dSSIM/dx(q) = (G*A)(q) + 2 x(q) (G*B)(q) + y(q) (G*Cm)(q),
//   A = ds/dmu_x - 2 mu_x ds/ds_xx - mu_y ds/ds_xy,  B = ds/ds_xx,  Cm = ds/ds_xy,
// so the forward writes A, B, Cm and a second pass blurs them.  Both passes
// are register-blocked (below).  Sums for the scalar loss are reduced per CTA
// and then in a fixed order (deterministic).
#include <algorithm>
#include <cmath>
#include <mutex>

#include <cuda.h>  // driver types only: the two context queries are fetched at run time

#include "gs_internal.cuh"
#include "gs_kernels.h"

namespace gs {

constexpr int kLT = 32;          // output tile edge
constexpr int kLR = 5;           // window radius
constexpr int kLI = kLT + 2 * kLR;  // staged tile edge (42)

struct Win { float w[2 * kLR + 1]; };

__device__ __forceinline__ float sgn(float d) { return d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f); }

__device__ __forceinline__ double block_sum_d(double v, double *sm) {
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

// Sum of per-thread FP32 partials over the block, in FP32 and a fixed order
// (a CTA sums 1024 pixels' terms; the per-CTA totals are added in FP64 by the
// final reduction).  No FP64 operation per pixel or per block: FP64 issues at
// a small fraction of the FP32 rate here.
__device__ __forceinline__ double block_sum_f(float v, float *sm) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    float r = 0.0f;
    if (warp == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0.0f;
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return (double)r;
}

// Register-blocked separable passes over a staged tile.  Horizontal: a thread
// owns kHS consecutive outputs of one staged row and walks the kHS + 10 inputs
// once, adding each (and its products) into every output whose window holds
// it; the lanes of a warp take consecutive rows, so with odd row strides their
// shared-memory words fall in distinct banks.  Vertical: a lane owns one
// column and kVR consecutive output rows of it.  Every output still sums its
// 11 taps in window order.  Staging issues all of a thread's global loads
// before its first shared-memory store, so their latencies overlap.
constexpr int kHS = 8;                      // outputs per thread, horizontal pass
constexpr int kHItems = kLI * (kLT / kHS);  // 42 rows x 4 strips = 168 busy threads
constexpr int kVR = 4;                      // output rows per thread, vertical pass (8 warps x 4 = 32)
constexpr int kLH = kLT + 1;                // padded row of the horizontal results
constexpr int kStR = (kLI + 7) / 8;         // staged rows per warp (8 warps; 32 + 10 columns a row)

__global__ void __launch_bounds__(256) k_ssim_fwd(const float *__restrict__ x, const float *__restrict__ y, int H,
                                                   int W, Win win, float *__restrict__ maps, int want_grad,
                                                   double *__restrict__ partials) {
    griddep_wait();
    __shared__ float sx[kLI][kLI + 1], sy[kLI][kLI + 1];
    __shared__ float h[5][kLI][kLH];
    __shared__ float sm[8];
    const int ch = blockIdx.z;
    const long long plane = (long long)H * W;
    const float *xc = x + ch * plane, *yc = y + ch * plane;
    const int ox = blockIdx.x * kLT, oy = blockIdx.y * kLT;
    {
        float vx[kStR][2], vy[kStR][2];
        #pragma unroll
        for (int t = 0; t < kStR; ++t) {
            #pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int r = (threadIdx.x >> 5) + 8 * t, c = (threadIdx.x & 31) + 32 * e;
                const int gy = oy + r - kLR, gx = ox + c - kLR;
                const bool in = r < kLI && c < kLI && gy >= 0 && gy < H && gx >= 0 && gx < W;
                vx[t][e] = in ? xc[(long long)gy * W + gx] : 0.0f;
                vy[t][e] = in ? yc[(long long)gy * W + gx] : 0.0f;
            }
        }
        #pragma unroll
        for (int t = 0; t < kStR; ++t) {
            #pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int r = (threadIdx.x >> 5) + 8 * t, c = (threadIdx.x & 31) + 32 * e;
                if (r < kLI && c < kLI) { sx[r][c] = vx[t][e]; sy[r][c] = vy[t][e]; }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < kHItems) {
        const int r = threadIdx.x % kLI, c0 = (threadIdx.x / kLI) * kHS;
        float a[kHS], b[kHS], aa[kHS], bb[kHS], ab[kHS];
        #pragma unroll
        for (int o = 0; o < kHS; ++o) a[o] = b[o] = aa[o] = bb[o] = ab[o] = 0.0f;
        #pragma unroll
        for (int j = 0; j < kHS + 2 * kLR; ++j) {
            const float u = sx[r][c0 + j], v = sy[r][c0 + j];
            const float uu = u * u, vv = v * v, uv = u * v;
            #pragma unroll
            for (int o = 0; o < kHS; ++o) {
                const int k = j - o;
                if (k < 0 || k > 2 * kLR) continue;
                const float wk = win.w[k];
                a[o] += wk * u; b[o] += wk * v; aa[o] += wk * uu; bb[o] += wk * vv; ab[o] += wk * uv;
            }
        }
        #pragma unroll
        for (int o = 0; o < kHS; ++o) {
            h[0][r][c0 + o] = a[o]; h[1][r][c0 + o] = b[o]; h[2][r][c0 + o] = aa[o];
            h[3][r][c0 + o] = bb[o]; h[4][r][c0 + o] = ab[o];
        }
    }
    __syncthreads();
    const int c = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * kVR;
    float mom[5][kVR];
    #pragma unroll
    for (int m = 0; m < 5; ++m) {
        #pragma unroll
        for (int q = 0; q < kVR; ++q) mom[m][q] = 0.0f;
        #pragma unroll
        for (int i = 0; i < kVR + 2 * kLR; ++i) {
            const float v = h[m][r0 + i][c];
            #pragma unroll
            for (int q = 0; q < kVR; ++q) {
                const int k = i - q;
                if (k >= 0 && k <= 2 * kLR) mom[m][q] += win.w[k] * v;
            }
        }
    }
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    float l1 = 0.0f, ss = 0.0f;
    #pragma unroll
    for (int q = 0; q < kVR; ++q) {
        const int r = r0 + q, gy = oy + r, gx = ox + c;
        if (gy >= H || gx >= W) continue;
        const float mx = mom[0][q], my = mom[1][q];
        const float sxx = mom[2][q] - mx * mx, syy = mom[3][q] - my * my, sxy = mom[4][q] - mx * my;
        const float A1 = 2.0f * mx * my + C1, A2 = 2.0f * sxy + C2;
        const float B1 = mx * mx + my * my + C1, B2 = sxx + syy + C2;
        const float iB = 1.0f / (B1 * B2);
        const float s = A1 * A2 * iB;
        ss += s;
        l1 += fabsf(sx[r + kLR][c + kLR] - sy[r + kLR][c + kLR]);
        if (want_grad) {  // 1/B1 = B2 iB and 1/B2 = B1 iB: one division per pixel
            const float dmu = 2.0f * my * A2 * iB - 2.0f * mx * s * (B2 * iB);
            const float dsxx = -s * (B1 * iB);
            const float dsxy = 2.0f * A1 * iB;
            const long long o = (long long)gy * W + gx;
            maps[(3 * ch + 0) * plane + o] = dmu - 2.0f * mx * dsxx - my * dsxy;
            maps[(3 * ch + 1) * plane + o] = dsxx;
            maps[(3 * ch + 2) * plane + o] = dsxy;
        }
    }
    const double tl1 = block_sum_f(l1, sm);
    const double tss = block_sum_f(ss, sm);
    if (threadIdx.x == 0) {
        const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partials[2 * b] = tl1;
        partials[2 * b + 1] = tss;
    }
}

__global__ void __launch_bounds__(256) k_ssim_bwd(const float *__restrict__ x, const float *__restrict__ y, int H,
                                                   int W, Win win, const float *__restrict__ maps, float l1_scale,
                                                   float ssim_scale, float *__restrict__ dL,
                                                   const double *__restrict__ partials, int nb, double inv_n,
                                                   float lambda, float *__restrict__ loss_out) {
    griddep_wait();
    __shared__ float sm[3][kLI][kLI + 1];
    __shared__ float h[3][kLI][kLH];
    const int ch = blockIdx.z;
    const long long plane = (long long)H * W;
    const int ox = blockIdx.x * kLT, oy = blockIdx.y * kLT;
    const int c = threadIdx.x & 31, r0 = (threadIdx.x >> 5) * kVR;
    {
        float v[3][kStR][2];
        #pragma unroll
        for (int t = 0; t < kStR; ++t) {
            #pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int r = (threadIdx.x >> 5) + 8 * t, cc = c + 32 * e;
                const int gy = oy + r - kLR, gx = ox + cc - kLR;
                const bool in = r < kLI && cc < kLI && gy >= 0 && gy < H && gx >= 0 && gx < W;
                const long long o = (long long)gy * W + gx;
                #pragma unroll
                for (int m = 0; m < 3; ++m) v[m][t][e] = in ? maps[(3 * ch + m) * plane + o] : 0.0f;
            }
        }
        #pragma unroll
        for (int t = 0; t < kStR; ++t) {
            #pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int r = (threadIdx.x >> 5) + 8 * t, cc = c + 32 * e;
                if (r < kLI && cc < kLI) {
                    #pragma unroll
                    for (int m = 0; m < 3; ++m) sm[m][r][cc] = v[m][t][e];
                }
            }
        }
    }
    // this thread's image values for the epilogue, fetched while the tile is staged
    float xe[kVR], ye[kVR];
    #pragma unroll
    for (int q = 0; q < kVR; ++q) {
        const int gy = oy + r0 + q, gx = ox + c;
        const bool in = gy < H && gx < W;
        const long long o = ch * plane + (long long)gy * W + gx;
        xe[q] = in ? x[o] : 0.0f;
        ye[q] = in ? y[o] : 0.0f;
    }
    __syncthreads();
    if (threadIdx.x < kHItems) {
        const int r = threadIdx.x % kLI, c0 = (threadIdx.x / kLI) * kHS;
        float acc[3][kHS];
        #pragma unroll
        for (int m = 0; m < 3; ++m) {
            #pragma unroll
            for (int o = 0; o < kHS; ++o) acc[m][o] = 0.0f;
        }
        #pragma unroll
        for (int j = 0; j < kHS + 2 * kLR; ++j) {
            const float u0 = sm[0][r][c0 + j], u1 = sm[1][r][c0 + j], u2 = sm[2][r][c0 + j];
            #pragma unroll
            for (int o = 0; o < kHS; ++o) {
                const int k = j - o;
                if (k < 0 || k > 2 * kLR) continue;
                const float wk = win.w[k];
                acc[0][o] += wk * u0; acc[1][o] += wk * u1; acc[2][o] += wk * u2;
            }
        }
        #pragma unroll
        for (int m = 0; m < 3; ++m) {
            #pragma unroll
            for (int o = 0; o < kHS; ++o) h[m][r][c0 + o] = acc[m][o];
        }
    }
    __syncthreads();
    float g[3][kVR];
    #pragma unroll
    for (int m = 0; m < 3; ++m) {
        #pragma unroll
        for (int q = 0; q < kVR; ++q) g[m][q] = 0.0f;
        #pragma unroll
        for (int i = 0; i < kVR + 2 * kLR; ++i) {
            const float v = h[m][r0 + i][c];
            #pragma unroll
            for (int q = 0; q < kVR; ++q) {
                const int k = i - q;
                if (k >= 0 && k <= 2 * kLR) g[m][q] += win.w[k] * v;
            }
        }
    }
    #pragma unroll
    for (int q = 0; q < kVR; ++q) {
        const int gy = oy + r0 + q, gx = ox + c;
        if (gy >= H || gx >= W) continue;
        const long long o = ch * plane + (long long)gy * W + gx;
        const float xv = xe[q], yv = ye[q];
        dL[o] = l1_scale * sgn(xv - yv) - ssim_scale * (g[0][q] + 2.0f * xv * g[1][q] + yv * g[2][q]);
    }
    // the scalar loss from the forward's per-CTA sums, by one block (a launch fewer)
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) {
        __shared__ double sd[8];
        double a = 0.0, b = 0.0;
        for (int i = threadIdx.x; i < nb; i += 256) { a += partials[2 * i]; b += partials[2 * i + 1]; }
        const double l1 = block_sum_d(a, sd) * inv_n;
        const double ssim = block_sum_d(b, sd) * inv_n;
        if (threadIdx.x == 0) *loss_out = (float)((1.0 - lambda) * l1 + lambda * (1.0 - ssim));
    }
}

__global__ void __launch_bounds__(256) k_l1(const float *__restrict__ x, const float *__restrict__ y, long long n,
                                             float scale, float *__restrict__ dL, double *__restrict__ partials) {
    griddep_wait();
    __shared__ double sm[8];
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = x[i] - y[i];
        s += fabsf(d);
        if (dL) dL[i] = scale * sgn(d);
    }
    const double t = block_sum_d(s, sm);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = t;
        partials[2 * blockIdx.x + 1] = 0.0;
    }
}

__global__ void __launch_bounds__(256) k_loss_final(const double *__restrict__ partials, int nb, double inv_n,
                                                     float lambda, float *__restrict__ out) {
    griddep_wait();
    __shared__ double sm[8];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += 256) { a += partials[2 * i]; b += partials[2 * i + 1]; }
    const double l1 = block_sum_d(a, sm) * inv_n;
    const double ssim = block_sum_d(b, sm) * inv_n;
    if (threadIdx.x == 0) *out = (float)((1.0 - lambda) * l1 + (lambda > 0.0f ? lambda * (1.0 - ssim) : 0.0));
}

static int loss_blocks(int h, int w) { return (int)(ceil_div(w, kLT) * ceil_div(h, kLT) * 3); }
constexpr int kL1Blocks = 148 * 4;

size_t loss_workspace_bytes(int h, int w) {
    const size_t maps = align_up(sizeof(float) * 9 * (size_t)h * w, 256);
    const size_t nb = (size_t)std::max(loss_blocks(h, w), kL1Blocks);
    return maps + align_up(sizeof(double) * 2 * nb, 256);
}

cudaError_t launch_loss(const float *img, const float *target, int h, int w, float lambda, float *loss_out,
                        float *dL_dimg, void *ws, cudaStream_t s) {
    const long long n = 3ll * h * w;
    float *maps = (float *)ws;
    double *partials = (double *)((char *)ws + align_up(sizeof(float) * 9 * (size_t)h * w, 256));
    if (lambda <= 0.0f) {
        launch_pdl(k_l1, kL1Blocks, 256, 0, s, img, target, n, (float)(1.0 / (double)n), dL_dimg, partials);
        launch_pdl(k_loss_final, 1, 256, 0, s, partials, kL1Blocks, 1.0 / (double)n, 0.0f, loss_out);
        return cudaGetLastError();
    }
    Win win;
    {
        double wd[2 * kLR + 1], sum = 0.0;
        for (int k = -kLR; k <= kLR; ++k) { wd[k + kLR] = exp(-(double)(k * k) / (2.0 * 1.5 * 1.5)); sum += wd[k + kLR]; }
        for (int k = 0; k < 2 * kLR + 1; ++k) win.w[k] = (float)(wd[k] / sum);
    }
    dim3 grid((unsigned)ceil_div(w, kLT), (unsigned)ceil_div(h, kLT), 3);
    launch_pdl(k_ssim_fwd, grid, 256, 0, s, img, target, h, w, win, maps, dL_dimg != nullptr, partials);
    if (dL_dimg)
        launch_pdl(k_ssim_bwd, grid, 256, 0, s, img, target, h, w, win, maps, (float)((1.0 - lambda) / (double)n),
                   (float)(lambda / (double)n), dL_dimg, partials, loss_blocks(h, w), 1.0 / (double)n, lambda,
                   loss_out);
    else
        launch_pdl(k_loss_final, 1, 256, 0, s, partials, loss_blocks(h, w), 1.0 / (double)n, lambda, loss_out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free variant.  Some callers cannot allocate device memory at the
// point where they need the loss: code that runs while the caller's allocator
// is unavailable (inside a host callback, in a memory-capped process whose
// budget another component owns), or a plain C host that receives only the
// image and gradient pointers from its framework.  For them the scratch lives
// in this file-scope device array, which every GPU that loads the library
// holds until the process exits.  Its size covers one view of at most
// kStaticMaxPixels pixels (1280x720, width and height <= 2048): 9 FP32 maps of
// the SSIM gradient plus the per-CTA partial sums.  Every scratch word a call
// reads is written earlier in the same call, so nothing needs clearing.  Each
// device has its own copy of the array; calls that overlap on the same device
// (other streams, other threads) race on its contents.

constexpr long long kStaticMaxPixels = 1280ll * 720ll;
constexpr int kStaticMaxSide = 2048;
constexpr int kStaticMaxBlocks = 4096;
constexpr size_t kStaticMapBytes = 9ull * (size_t)kStaticMaxPixels * sizeof(float);
constexpr size_t kStaticBytes = kStaticMapBytes + 2ull * sizeof(double) * kStaticMaxBlocks;

static __device__ __align__(256) unsigned char g_loss_scratch[kStaticBytes];

namespace {
constexpr int kMaxDevices = 128;
std::mutex g_scratch_mu;
// per device: the array's address and the id of the context it was looked up in
struct ScratchCache {
    unsigned long long ctx_id;
    void *ptr;
};
ScratchCache g_scratch[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Unique id of the current context (never reused within a process), through
// the driver entry points the runtime hands out; false if there is no
// current context or the driver cannot say.
bool current_context_id(unsigned long long *id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<CtxGetCurrentFn>(a);
            get_id = reinterpret_cast<CtxGetIdFn>(b);
        }
        looked_up = true;
    }
    if (!get_current || !get_id) return false;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}
}  // namespace

bool loss_static_fits(int h, int w) {
    if (h <= 0 || w <= 0 || h > kStaticMaxSide || w > kStaticMaxSide) return false;
    if ((long long)h * w > kStaticMaxPixels) return false;
    return loss_workspace_bytes(h, w) <= kStaticBytes;
}

long long loss_static_max_pixels() { return kStaticMaxPixels; }

// The device address of the scratch array for the current device and
// context.  The first call in a context looks it up (cudaGetSymbolAddress,
// with that device current) and caches it under the context's id; later calls
// in the same context only read the cache.  A new context on the device (after
// a reset of the primary context, say) has a new id, so the address is looked
// up again there instead of reusing one of a destroyed context.
cudaError_t loss_static_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    unsigned long long ctx = 0;
    bool known = current_context_id(&ctx);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (known && g_scratch[dev].ptr && g_scratch[dev].ctx_id == ctx) {
        *out = g_scratch[dev].ptr;
        return cudaSuccess;
    }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_loss_scratch);  // makes the device's primary context current if none is
    if (e != cudaSuccess) return e;
    if (!known) known = current_context_id(&ctx);
    g_scratch[dev] = known ? ScratchCache{ctx, p} : ScratchCache{0, nullptr};  // no id: look up every call
    *out = p;
    return cudaSuccess;
}

}  // namespace gs
