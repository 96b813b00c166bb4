// project.cu -- per-Gaussian projection (forward) and its chain rule
// (backward) for every view of a chunk, one thread per Gaussian.  The
// parameters are read once per Gaussian and reused for all views in registers.
//
// Projection: EWA splatting of the cited 3DGS rasteriser (the paper relies on
// it for Supp. D.2): Sigma = R(q) S S^T R(q)^T, Sigma' = J W Sigma W^T J^T +
// dilation I, conic = Sigma'^-1, radius = ceil(3 sqrt(lambda_max)); colour from
// real spherical harmonics of degree D <= 3; opacity = sigmoid(logit).
#include "gs_internal.cuh"
#include "gs_kernels.h"

namespace gs {

// Real spherical harmonics with the Condon-Shortley phase, as Cartesian
// polynomials of the unit direction (x, y, z); index l^2 + l + m.
// Constants are sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the polynomial
// prefactors: C1 = sqrt(3/(4pi)), C2a = sqrt(15/(4pi)), C2b = sqrt(5/(16pi)),
// C2c = sqrt(15/(16pi)), C3a = sqrt(35/(32pi)), C3b = sqrt(105/(4pi)),
// C3c = sqrt(21/(32pi)), C3d = sqrt(7/(16pi)), C3e = sqrt(105/(16pi)).
namespace shc {
constexpr float C0 = 0.28209479177387814f;
constexpr float C1 = 0.4886025119029199f;
constexpr float C2a = 1.0925484305920792f;
constexpr float C2b = 0.31539156525252005f;
constexpr float C2c = 0.5462742152960396f;
constexpr float C3a = 0.5900435899266435f;
constexpr float C3b = 2.890611442640554f;
constexpr float C3c = 0.4570457994644658f;
constexpr float C3d = 0.3731763325901154f;
constexpr float C3e = 1.445305721320277f;
}  // namespace shc

template <int D>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float *Y) {
    using namespace shc;
    Y[0] = C0;
    if (D >= 1) { Y[1] = -C1 * y; Y[2] = C1 * z; Y[3] = -C1 * x; }
    if (D >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = C2a * x * y;
        Y[5] = -C2a * y * z;
        Y[6] = C2b * (3.0f * zz - 1.0f);
        Y[7] = -C2a * x * z;
        Y[8] = C2c * (xx - yy);
        if (D >= 3) {
            Y[9] = -C3a * y * (3.0f * xx - yy);
            Y[10] = C3b * x * y * z;
            Y[11] = -C3c * y * (5.0f * zz - 1.0f);
            Y[12] = C3d * z * (5.0f * zz - 3.0f);
            Y[13] = -C3c * x * (5.0f * zz - 1.0f);
            Y[14] = C3e * z * (xx - yy);
            Y[15] = -C3a * x * (xx - 3.0f * yy);
        }
    }
}

// Gradient of sum_k w_k Y_k with respect to (x, y, z), w_k given.
template <int D>
__device__ __forceinline__ void sh_basis_vjp(float x, float y, float z, const float *w, float &gx, float &gy,
                                             float &gz) {
    using namespace shc;
    gx = gy = gz = 0.0f;
    if (D >= 1) { gy -= C1 * w[1]; gz += C1 * w[2]; gx -= C1 * w[3]; }
    if (D >= 2) {
        gx += C2a * y * w[4]; gy += C2a * x * w[4];
        gy -= C2a * z * w[5]; gz -= C2a * y * w[5];
        gz += 6.0f * C2b * z * w[6];
        gx -= C2a * z * w[7]; gz -= C2a * x * w[7];
        gx += 2.0f * C2c * x * w[8]; gy -= 2.0f * C2c * y * w[8];
        if (D >= 3) {
            const float xx = x * x, yy = y * y, zz = z * z;
            gx -= 6.0f * C3a * x * y * w[9]; gy -= 3.0f * C3a * (xx - yy) * w[9];
            gx += C3b * y * z * w[10]; gy += C3b * x * z * w[10]; gz += C3b * x * y * w[10];
            gy -= C3c * (5.0f * zz - 1.0f) * w[11]; gz -= 10.0f * C3c * y * z * w[11];
            gz += C3d * (15.0f * zz - 3.0f) * w[12];
            gx -= C3c * (5.0f * zz - 1.0f) * w[13]; gz -= 10.0f * C3c * x * z * w[13];
            gx += 2.0f * C3e * x * z * w[14]; gy -= 2.0f * C3e * y * z * w[14]; gz += C3e * (xx - yy) * w[14];
            gx -= 3.0f * C3a * (xx - yy) * w[15]; gy += 6.0f * C3a * x * y * w[15];
        }
    }
}

struct Cov3 { float s00, s01, s02, s11, s12, s22; };

// EWA 2D covariance (before dilation) from the 3D covariance, for one view.
struct Ewa { float T[6]; float A, B, C; bool clx_lo, clx_hi, cly_lo, cly_hi; float tx, ty; };

__device__ __forceinline__ Ewa ewa(const ViewDesc &c, float x, float y, float z, const Cov3 &S) {
    Ewa e;
    const float rx = x / z, ry = y / z;
    e.clx_lo = rx < -c.limx; e.clx_hi = rx > c.limx;
    e.cly_lo = ry < -c.limy; e.cly_hi = ry > c.limy;
    e.tx = z * fminf(fmaxf(rx, -c.limx), c.limx);
    e.ty = z * fminf(fmaxf(ry, -c.limy), c.limy);
    const float iz = 1.0f / z;
    const float J00 = c.fx * iz, J02 = -c.fx * e.tx * iz * iz;
    const float J11 = c.fy * iz, J12 = -c.fy * e.ty * iz * iz;
    // T = J W (W = view rotation), 2 x 3
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
        e.T[k] = J00 * c.R[k] + J02 * c.R[6 + k];
        e.T[3 + k] = J11 * c.R[3 + k] + J12 * c.R[6 + k];
    }
    const float *T = e.T;
    const float ST0x = S.s00 * T[0] + S.s01 * T[1] + S.s02 * T[2];
    const float ST0y = S.s01 * T[0] + S.s11 * T[1] + S.s12 * T[2];
    const float ST0z = S.s02 * T[0] + S.s12 * T[1] + S.s22 * T[2];
    const float ST1x = S.s00 * T[3] + S.s01 * T[4] + S.s02 * T[5];
    const float ST1y = S.s01 * T[3] + S.s11 * T[4] + S.s12 * T[5];
    const float ST1z = S.s02 * T[3] + S.s12 * T[4] + S.s22 * T[5];
    e.A = T[0] * ST0x + T[1] * ST0y + T[2] * ST0z;
    e.B = T[0] * ST1x + T[1] * ST1y + T[2] * ST1z;
    e.C = T[3] * ST1x + T[4] * ST1y + T[5] * ST1z;
    return e;
}

template <int D>
__global__ void __launch_bounds__(256, 4) k_project(const float *__restrict__ P, long long n, long long ld, ViewTable vt,
                                                 RasterCfg cfg, float2 *__restrict__ xy, float4 *__restrict__ co,
                                                 float4 *__restrict__ rgbd, int *__restrict__ radius,
                                                 int *__restrict__ touched, int *__restrict__ status,
                                                 float4 *__restrict__ cj) {
    griddep_wait();
    constexpr int K = (D + 1) * (D + 1);
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ld) return;
    if (g >= n) {  // padding records: never visible
        for (int v = 0; v < vt.n_views; ++v) { radius[v * ld + g] = 0; touched[v * ld + g] = 0; }
        return;
    }
    const float mx = P[0 * ld + g], my = P[1 * ld + g], mz = P[2 * ld + g];

    // cheap near-plane pass first: skip the remaining loads if no view sees it; a
    // Gaussian whose opacity is below alpha_min can never blend and is culled too
    const bool bright = !(P[10 * ld + g] < cfg.logit_min);
    bool any = false;
    for (int v = 0; v < vt.n_views && bright; ++v) {
        const ViewDesc &c = vt.v[v];
        float zc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.R[6], mx), __fmul_rn(c.R[7], my)), __fmul_rn(c.R[8], mz)), c.t[2]);
        any |= zc > cfg.near_z;
    }
    if (!any) {
        for (int v = 0; v < vt.n_views; ++v) { radius[v * ld + g] = 0; touched[v * ld + g] = 0; }
        return;
    }

    Cov3 S;
    {
        float qw = P[6 * ld + g], qx = P[7 * ld + g], qy = P[8 * ld + g], qz = P[9 * ld + g];
        const float nq = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        qw /= nq; qx /= nq; qy /= nq; qz /= nq;
        float R[9];
        quat_rotation(qw, qx, qy, qz, R);
        const float s0 = expf(P[3 * ld + g]), s1 = expf(P[4 * ld + g]), s2 = expf(P[5 * ld + g]);
        float M[9];
        #pragma unroll
        for (int r = 0; r < 3; ++r) { M[3 * r] = R[3 * r] * s0; M[3 * r + 1] = R[3 * r + 1] * s1; M[3 * r + 2] = R[3 * r + 2] * s2; }
        S.s00 = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
        S.s01 = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
        S.s02 = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
        S.s11 = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
        S.s12 = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
        S.s22 = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    }
    const float opacity = 1.0f / (1.0f + expf(-P[10 * ld + g]));

    for (int v = 0; v < vt.n_views; ++v) {
        const ViewDesc &c = vt.v[v];
        const long long rec = v * ld + g;
        int rad = 0, tt = 0;
        const ExactPos p = exact_position(c, mx, my, mz);
        if (p.zc > cfg.near_z) {
            const Ewa e = ewa(c, p.xc, p.yc, p.zc, S);
            const float A = e.A + cfg.dilation, B = e.B, C = e.C + cfg.dilation;
            const float det = A * C - B * B;
            const float inv = 1.0f / det;
            const float ca = C * inv, cb = -B * inv, cc = A * inv;
            const float mid = 0.5f * (A + C);
            const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
            const float rr = ceilf(3.0f * sqrtf(lam));
            const bool finite = isfinite(p.u) && isfinite(p.v) && isfinite(ca) && isfinite(cb) && isfinite(cc) &&
                                isfinite(rr);
            if (!finite) {
                if (status) atomicOr(status, 1 << GS_ERR_NUMERIC);
            } else if (det > 0.0f) {
                rad = (int)fminf(rr, 16777216.0f);
                const Rect rc = tile_rect(p.u, p.v, rad, vt.tile_w, vt.tile_h, c.GW, c.GH);
                tt = (rc.x1 - rc.x0) * (rc.y1 - rc.y0);
                if (tt <= 0) { rad = 0; tt = 0; }
            }
            if (rad > 0) {
                xy[rec] = make_float2(p.u, p.v);
                co[rec] = make_float4(ca, cb, cc, opacity);
                // view-dependent colour
                float dx = mx - c.campos[0], dy = my - c.campos[1], dz = mz - c.campos[2];
                const float id = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
                dx *= id; dy *= id; dz *= id;
                float r = 0.5f, gch = 0.5f, b = 0.5f;
                if (D >= 1 && cj) {
                    // channel by channel (16 coefficients live at a time, for 64 registers per
                    // thread at four CTAs per SM), with the gradient of the unclamped colour with
                    // respect to the mean through the view direction, and the clamp flag, kept
                    // for the backward, which then reads no SH coefficient
                    #pragma unroll 1
                    for (int ch = 0; ch < 3; ++ch) {
                        float Y[K], w[K];
                        sh_basis<D>(dx, dy, dz, Y);
                        float raw = 0.5f;
                        #pragma unroll
                        for (int k = 0; k < K; ++k) {
                            w[k] = P[(11 + 3 * k + ch) * ld + g];
                            raw += Y[k] * w[k];
                        }
                        float gx, gy, gz;
                        sh_basis_vjp<D>(dx, dy, dz, w, gx, gy, gz);
                        const float dd = gx * dx + gy * dy + gz * dz;  // onto the sphere's tangent plane
                        cj[3 * rec + ch] = make_float4((gx - dx * dd) * id, (gy - dy * dd) * id, (gz - dz * dd) * id,
                                                       raw < 0.0f ? 0.0f : 1.0f);
                        r = ch == 0 ? raw : r;
                        gch = ch == 1 ? raw : gch;
                        b = ch == 2 ? raw : b;
                    }
                } else {
                    float Y[16];
                    sh_basis<D>(dx, dy, dz, Y);
                    #pragma unroll
                    for (int k = 0; k < K; ++k) {
                        r += Y[k] * P[(11 + 3 * k) * ld + g];
                        gch += Y[k] * P[(12 + 3 * k) * ld + g];
                        b += Y[k] * P[(13 + 3 * k) * ld + g];
                    }
                }
                rgbd[rec] = make_float4(fmaxf(r, 0.0f), fmaxf(gch, 0.0f), fmaxf(b, 0.0f), p.zc);
            }
        }
        radius[rec] = rad;
        touched[rec] = tt;
    }
}

// Backward of the projection.  acc holds, per record, the planes
// kAccU..kAccMaxW written by the compositing backward.  One thread per
// Gaussian: per view, first the colour (SH) part, whose gradients are written
// straight to their planes, then the geometric part, whose covariance
// gradient is summed over views; the view-independent rotation and scales are
// recomputed rather than kept live, to keep registers (and so occupancy) for
// this memory-bound pass.  Writes every parameter plane of the Gaussian once
// (zeros when no view saw it).
__device__ __forceinline__ void rot_scale(const float *__restrict__ P, long long ld, long long g, float *R, float *s,
                                          float &nq, float *qh) {
    float qw = P[6 * ld + g], qx = P[7 * ld + g], qy = P[8 * ld + g], qz = P[9 * ld + g];
    nq = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qh[0] = qw / nq; qh[1] = qx / nq; qh[2] = qy / nq; qh[3] = qz / nq;
    quat_rotation(qh[0], qh[1], qh[2], qh[3], R);
    s[0] = expf(P[3 * ld + g]); s[1] = expf(P[4 * ld + g]); s[2] = expf(P[5 * ld + g]);
}

__device__ __forceinline__ Cov3 cov3(const float *R, const float *s) {
    float M[9];
    #pragma unroll
    for (int r = 0; r < 3; ++r)
        #pragma unroll
        for (int c = 0; c < 3; ++c) M[3 * r + c] = R[3 * r + c] * s[c];
    Cov3 S;
    S.s00 = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    S.s01 = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    S.s02 = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    S.s11 = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    S.s12 = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    S.s22 = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    return S;
}

// Adam applied where the projection backward finishes a Gaussian's gradient
// (the fused mode): moments, rates and bias corrections of one step.
struct FusedAdam {
    float *m, *v;
    float lr[6];
    float b1, b2, eps, inv_bc1, inv_sqrt_bc2;
    const long long *step_dev;  // nullable: the step is read here at run time
    float iso_gscale;           // lambda_iso / n: the isotropic term's gradient scale (0: none)
    const float *G_in;          // nullable: gradient added to the computed one
};

__device__ __forceinline__ int adam_group(int plane) {
    // means, log-scales, quaternion, opacity, SH degree 0, SH degree >= 1
    return plane < 3 ? 0 : plane < 6 ? 1 : plane < 10 ? 2 : plane == 10 ? 3 : plane < 14 ? 4 : 5;
}

// Projection backward, one thread per Gaussian (planes of ld):
//  colour part, channel by channel: each SH plane's gradient sum_v gc_v Y(d_v)
//  is complete in registers after the view loop, and the direction term of the
//  mean is accumulated per (channel, view) through the SH vector-Jacobian product
//  (linear in its weights);
//  geometry part, view by view: opacity, conic -> 2D covariance -> Sigma
//  (summed over views), Jacobian and position; then Sigma -> scale, rotation.
// Each plane's gradient is emitted once: written to G (accumulated when
// `accumulate`), or, in the fused mode, turned into one Adam step of the
// parameter and its moments, with the isotropic term and G_in added first.
// Folds the lifecycle statistics of the views into stats (nullable).
constexpr int kFusedThreads = 128;  // fused mode: Gaussians per CTA (four CTAs per SM overlap the two phases)

template <int D, bool ADAM>
__global__ void __launch_bounds__(ADAM ? kFusedThreads : 256, ADAM ? 4 : 3) k_project_bwd(float *__restrict__ P, long long n, long long ld,
                                                     ViewTable vt, RasterCfg cfg, const int *__restrict__ radius,
                                                     const float *__restrict__ acc, long long nrec,
                                                     float *__restrict__ G, int accumulate,
                                                     const float *__restrict__ loss_per_view,
                                                     float *__restrict__ stats, long long stats_ld, FusedAdam fa,
                                                     const float4 *__restrict__ cj, uint8_t *__restrict__ rows) {
    griddep_wait();
    constexpr int K = (D + 1) * (D + 1);
    if (ADAM && fa.step_dev) {  // bias corrections from the device step counter (graph replay)
        __shared__ float s_bc[2];
        if (threadIdx.x == 0) {
            adam_bias_inv(fa.b1, fa.b2, *fa.step_dev, s_bc[0], s_bc[1]);
        }
        __syncthreads();
        fa.inv_bc1 = s_bc[0];
        fa.inv_sqrt_bc2 = s_bc[1];
    }
    constexpr int NP = 11 + 3 * K;  // parameter planes
    extern __shared__ float s_grad[];  // fused mode: [NP][kFusedThreads] gradients of the CTA's Gaussians
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (!ADAM) {
        if (g >= ld) return;
        if (rows) {
            // rows mode: a Gaussian no view sees has a zero gradient, which is marked instead
            // of written (the Adam step reads it as zero)
            bool any = false;
            if (g < n)
                for (int v = 0; v < vt.n_views; ++v) any |= radius[v * ld + g] > 0;
            rows[g] = any ? 1 : 0;
            if (!any) return;
        } else if (g >= n) {  // padding: zero gradient
            if (!accumulate)
                for (int k = 0; k < NP; ++k) G[k * ld + g] = 0.0f;
            return;
        }
    }
    // one plane's gradient: to G, or (fused) to the CTA's shared gradient block
    auto emit = [&](int plane, float grad) {
        if (ADAM) {
            s_grad[plane * kFusedThreads + threadIdx.x] = grad;
        } else {
            const long long i = (long long)plane * ld + g;
            G[i] = accumulate ? G[i] + grad : grad;
        }
    };
    if (ADAM && g >= n) {  // padding and the CTA's tail: zero gradient
        for (int k = 0; k < NP; ++k) emit(k, 0.0f);
    } else {

    const float mx = P[0 * ld + g], my = P[1 * ld + g], mz = P[2 * ld + g];
    float gmean[3] = {0, 0, 0};

    // ---- colour: SH gradients and the direction term of the mean ----
    if (D >= 1 && cj) {
        // from the forward's per-record colour gradients and clamp flags: no SH coefficient read
        #pragma unroll 1
        for (int ch = 0; ch < 3; ++ch) {
            float gsh[K];
            #pragma unroll
            for (int k = 0; k < K; ++k) gsh[k] = 0.0f;
            for (int v = 0; v < vt.n_views; ++v) {
                const long long rec = v * ld + g;
                if (radius[rec] <= 0) continue;
                const ViewDesc &c = vt.v[v];
                float ex = mx - c.campos[0], ey = my - c.campos[1], ez = mz - c.campos[2];
                const float idist = 1.0f / sqrtf(ex * ex + ey * ey + ez * ez);
                ex *= idist; ey *= idist; ez *= idist;
                float Y[K];
                sh_basis<D>(ex, ey, ez, Y);
                const float4 jc = cj[3 * rec + ch];
                const float gcv = jc.w * acc[rec * kAccStride + kAccR + ch];
                #pragma unroll
                for (int k = 0; k < K; ++k) gsh[k] += gcv * Y[k];
                gmean[0] += gcv * jc.x;
                gmean[1] += gcv * jc.y;
                gmean[2] += gcv * jc.z;
            }
            #pragma unroll
            for (int k = 0; k < K; ++k) emit(11 + 3 * k + ch, gsh[k]);
        }
    } else {
        #pragma unroll 1
        for (int ch = 0; ch < 3; ++ch) {
            float sh[K], gsh[K];
            #pragma unroll
            for (int k = 0; k < K; ++k) {
                sh[k] = P[(11 + 3 * k + ch) * ld + g];
                gsh[k] = 0.0f;
            }
            for (int v = 0; v < vt.n_views; ++v) {
                const long long rec = v * ld + g;
                if (radius[rec] <= 0) continue;
                const ViewDesc &c = vt.v[v];
                float ex = mx - c.campos[0], ey = my - c.campos[1], ez = mz - c.campos[2];
                const float idist = 1.0f / sqrtf(ex * ex + ey * ey + ez * ez);
                ex *= idist; ey *= idist; ez *= idist;
                float Y[K];
                sh_basis<D>(ex, ey, ez, Y);
                float raw = 0.5f;
                #pragma unroll
                for (int k = 0; k < K; ++k) raw += Y[k] * sh[k];
                const float gcv = raw < 0.0f ? 0.0f : acc[rec * kAccStride + kAccR + ch];
                #pragma unroll
                for (int k = 0; k < K; ++k) gsh[k] += gcv * Y[k];
                if (D > 0) {
                    float w[K];
                    #pragma unroll
                    for (int k = 0; k < K; ++k) w[k] = gcv * sh[k];
                    float gx, gy, gz;
                    sh_basis_vjp<D>(ex, ey, ez, w, gx, gy, gz);
                    const float dd = gx * ex + gy * ey + gz * ez;  // onto the sphere's tangent plane
                    gmean[0] += (gx - ex * dd) * idist;
                    gmean[1] += (gy - ey * dd) * idist;
                    gmean[2] += (gz - ez * dd) * idist;
                }
            }
            #pragma unroll
            for (int k = 0; k < K; ++k) emit(11 + 3 * k + ch, gsh[k]);
        }
    }

    // ---- geometry: opacity, conic -> 2D covariance -> Sigma, J, position ----
    float glogit = 0.0f;
    float dSig[6] = {0, 0, 0, 0, 0, 0};  // dL/dSigma entries 00 01 02 11 12 22 (each ordered pair)
    bool seen = false;
    float st_omega = 0, st_kappa = 0, st_gamma = 0, st_maxw = 0, st_gnorm = 0, st_views = 0;
    float R[9], s[3], nq, qh[4];
    rot_scale(P, ld, g, R, s, nq, qh);
    const Cov3 S = cov3(R, s);
    const float logit = P[10 * ld + g];
    const float o = 1.0f / (1.0f + expf(-logit));
    for (int v = 0; v < vt.n_views; ++v) {
        const long long rec = v * ld + g;
        if (radius[rec] <= 0) continue;
        seen = true;
        const ViewDesc &c = vt.v[v];
        // the record's sums: u v a b | c o r g | b z omega kappa | maxw
        const float4 *a4 = reinterpret_cast<const float4 *>(acc + rec * kAccStride);
        const float4 s0 = a4[0], s1 = a4[1], s2 = a4[2];
        const float du = s0.x, dv = s0.y;
        if (stats) {
            const float om = s2.z;
            st_omega += om;
            st_kappa += s2.w;
            st_gamma += (loss_per_view ? loss_per_view[v] : 0.0f) * om;
            st_maxw = fmaxf(st_maxw, acc[rec * kAccStride + kAccMaxW]);
            st_gnorm += sqrtf(du * du + dv * dv);
            st_views += om > 0.0f ? 1.0f : 0.0f;
        }
        glogit += s1.y * o * (1.0f - o);
        const float da = s0.z, db = s0.w, dc = s1.x;
        const float gdepth = s2.y;
        const ExactPos p = exact_position(c, mx, my, mz);
        const float x = p.xc, y = p.yc, z = p.zc;
        const Ewa e = ewa(c, x, y, z, S);
        const float A = e.A + cfg.dilation, B = e.B, C = e.C + cfg.dilation;
        const float idet = 1.0f / (A * C - B * B);
        const float qa = C * idet, qb = -B * idet, qcc = A * idet;
        // conic Q = Sigma'^-1: dL/dSigma' = -Q G Q, G = [[da, db/2], [db/2, dc]]
        const float hb = 0.5f * db;
        const float QG00 = qa * da + qb * hb, QG01 = qa * hb + qb * dc;
        const float QG10 = qb * da + qcc * hb, QG11 = qb * hb + qcc * dc;
        const float dA = -(QG00 * qa + QG01 * qb);
        const float dBh = -(QG00 * qb + QG01 * qcc);  // per entry of the symmetric off-diagonal
        const float dC = -(QG10 * qb + QG11 * qcc);
        // Sigma' = T Sigma T^T: dSigma = T^T Sd T, dT = 2 Sd T Sigma, Sd = [[dA, dBh], [dBh, dC]]
        const float *T = e.T;
        float U[6];
        #pragma unroll
        for (int k = 0; k < 3; ++k) {
            U[k] = dA * T[k] + dBh * T[3 + k];
            U[3 + k] = dBh * T[k] + dC * T[3 + k];
        }
        dSig[0] += T[0] * U[0] + T[3] * U[3];
        dSig[1] += T[0] * U[1] + T[3] * U[4];
        dSig[2] += T[0] * U[2] + T[3] * U[5];
        dSig[3] += T[1] * U[1] + T[4] * U[4];
        dSig[4] += T[1] * U[2] + T[4] * U[5];
        dSig[5] += T[2] * U[2] + T[5] * U[5];
        float dT[6];
        #pragma unroll
        for (int r = 0; r < 2; ++r) {
            const float u0 = U[3 * r], u1 = U[3 * r + 1], u2 = U[3 * r + 2];
            dT[3 * r + 0] = 2.0f * (u0 * S.s00 + u1 * S.s01 + u2 * S.s02);
            dT[3 * r + 1] = 2.0f * (u0 * S.s01 + u1 * S.s11 + u2 * S.s12);
            dT[3 * r + 2] = 2.0f * (u0 * S.s02 + u1 * S.s12 + u2 * S.s22);
        }
        // T = J W: dJ = dT W^T; J00 = fx/z, J02 = -fx tx/z^2, J11 = fy/z, J12 = -fy ty/z^2
        const float dJ00 = dT[0] * c.R[0] + dT[1] * c.R[1] + dT[2] * c.R[2];
        const float dJ02 = dT[0] * c.R[6] + dT[1] * c.R[7] + dT[2] * c.R[8];
        const float dJ11 = dT[3] * c.R[3] + dT[4] * c.R[4] + dT[5] * c.R[5];
        const float dJ12 = dT[3] * c.R[6] + dT[4] * c.R[7] + dT[5] * c.R[8];
        const float iz = 1.0f / z, iz2 = iz * iz, iz3 = iz2 * iz;
        const float dtx_dx = (e.clx_lo || e.clx_hi) ? 0.0f : 1.0f;
        const float dtx_dz = e.clx_lo ? -c.limx : (e.clx_hi ? c.limx : 0.0f);
        const float dty_dy = (e.cly_lo || e.cly_hi) ? 0.0f : 1.0f;
        const float dty_dz = e.cly_lo ? -c.limy : (e.cly_hi ? c.limy : 0.0f);
        const float gx = dJ02 * (-c.fx * iz2) * dtx_dx + du * c.fx * iz;
        const float gy = dJ12 * (-c.fy * iz2) * dty_dy + dv * c.fy * iz;
        const float gz = -dJ00 * c.fx * iz2 - dJ11 * c.fy * iz2 +
                         dJ02 * (-c.fx * dtx_dz * iz2 + 2.0f * c.fx * e.tx * iz3) +
                         dJ12 * (-c.fy * dty_dz * iz2 + 2.0f * c.fy * e.ty * iz3) -
                         du * c.fx * x * iz2 - dv * c.fy * y * iz2 + gdepth;
        gmean[0] += c.R[0] * gx + c.R[3] * gy + c.R[6] * gz;
        gmean[1] += c.R[1] * gx + c.R[4] * gy + c.R[7] * gz;
        gmean[2] += c.R[2] * gx + c.R[5] * gy + c.R[8] * gz;
    }

    float glogs[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0};
    if (seen) {
        float M[9];
        #pragma unroll
        for (int r = 0; r < 3; ++r)
            #pragma unroll
            for (int cix = 0; cix < 3; ++cix) M[3 * r + cix] = R[3 * r + cix] * s[cix];
        // Sigma = M M^T: dM = (dSig + dSig^T) M = 2 dSig M (dSig symmetric)
        const float F00 = 2.0f * dSig[0], F11 = 2.0f * dSig[3], F22 = 2.0f * dSig[5];
        const float F01 = 2.0f * dSig[1], F02 = 2.0f * dSig[2], F12 = 2.0f * dSig[4];
        float dM[9];
        #pragma unroll
        for (int m = 0; m < 3; ++m) {
            dM[0 + m] = F00 * M[0 + m] + F01 * M[3 + m] + F02 * M[6 + m];
            dM[3 + m] = F01 * M[0 + m] + F11 * M[3 + m] + F12 * M[6 + m];
            dM[6 + m] = F02 * M[0 + m] + F12 * M[3 + m] + F22 * M[6 + m];
        }
        float dR[9];
        #pragma unroll
        for (int m = 0; m < 3; ++m) {
            const float ds = dM[m] * R[m] + dM[3 + m] * R[3 + m] + dM[6 + m] * R[6 + m];
            glogs[m] = ds * s[m];
            dR[m] = dM[m] * s[m]; dR[3 + m] = dM[3 + m] * s[m]; dR[6 + m] = dM[6 + m] * s[m];
        }
        const float w_ = qh[0], x_ = qh[1], y_ = qh[2], z_ = qh[3];
        const float dqw = 2.f * (-z_ * dR[1] + y_ * dR[2] + z_ * dR[3] - x_ * dR[5] - y_ * dR[6] + x_ * dR[7]);
        const float dqx = 2.f * (y_ * dR[1] + z_ * dR[2] + y_ * dR[3] - 2.f * x_ * dR[4] - w_ * dR[5] + z_ * dR[6] +
                                 w_ * dR[7] - 2.f * x_ * dR[8]);
        const float dqy = 2.f * (-2.f * y_ * dR[0] + x_ * dR[1] + w_ * dR[2] + x_ * dR[3] + z_ * dR[5] - w_ * dR[6] +
                                 z_ * dR[7] - 2.f * y_ * dR[8]);
        const float dqz = 2.f * (-2.f * z_ * dR[0] - w_ * dR[1] + x_ * dR[2] + w_ * dR[3] - 2.f * z_ * dR[4] +
                                 y_ * dR[5] + x_ * dR[6] + y_ * dR[7]);
        const float qd = w_ * dqw + x_ * dqx + y_ * dqy + z_ * dqz;  // normalisation: project out q
        gq[0] = (dqw - w_ * qd) / nq;
        gq[1] = (dqx - x_ * qd) / nq;
        gq[2] = (dqy - y_ * qd) / nq;
        gq[3] = (dqz - z_ * qd) / nq;
    }
    if (ADAM && fa.iso_gscale != 0.0f) iso_grad(P[3 * ld + g], P[4 * ld + g], P[5 * ld + g], fa.iso_gscale, glogs);
    emit(0, gmean[0]); emit(1, gmean[1]); emit(2, gmean[2]);
    emit(3, glogs[0]); emit(4, glogs[1]); emit(5, glogs[2]);
    emit(6, gq[0]); emit(7, gq[1]); emit(8, gq[2]); emit(9, gq[3]);
    emit(10, glogit);

    if (stats) {
        stats[0 * stats_ld + g] += st_omega;
        stats[1 * stats_ld + g] += st_kappa;
        stats[2 * stats_ld + g] += st_gamma;
        stats[3 * stats_ld + g] = fmaxf(stats[3 * stats_ld + g], st_maxw);
        stats[4 * stats_ld + g] += st_gnorm;
        stats[5 * stats_ld + g] += st_views;
    }
    }  // g < n
    if (ADAM) {
        // the CTA's NP x kFusedThreads block of parameters and moments, streamed as
        // float4 (ld is a multiple of 32, so a float4 never crosses the end of a plane)
        __syncthreads();
        constexpr int Q = kFusedThreads / 4;  // float4 per plane
        constexpr int U = 4;                  // float4 updates whose loads are issued together
        const long long g0 = (long long)blockIdx.x * kFusedThreads;
        const int lim = ld - g0 < kFusedThreads ? (int)(ld - g0) : kFusedThreads;
        const float *__restrict__ Gin = fa.G_in;
        float *__restrict__ Mp = fa.m;
        float *__restrict__ Vp = fa.v;
        for (int base = threadIdx.x; base < NP * Q; base += U * kFusedThreads) {
            float4 m4[U], v4[U], p4[U], gi[U];
            long long ii[U];
            bool ok[U];
            int pl[U], qq[U];
            #pragma unroll
            for (int u = 0; u < U; ++u) {
                const int idx = base + u * kFusedThreads;
                pl[u] = idx / Q;
                qq[u] = (idx % Q) * 4;
                ok[u] = idx < NP * Q && qq[u] < lim;
                ii[u] = (long long)pl[u] * ld + g0 + qq[u];
                if (ok[u]) {
                    m4[u] = *reinterpret_cast<const float4 *>(Mp + ii[u]);
                    v4[u] = *reinterpret_cast<const float4 *>(Vp + ii[u]);
                    p4[u] = *reinterpret_cast<const float4 *>(P + ii[u]);
                    gi[u] = Gin ? *reinterpret_cast<const float4 *>(Gin + ii[u]) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            #pragma unroll
            for (int u = 0; u < U; ++u) {
                if (!ok[u]) continue;
                const float4 gs4 = *reinterpret_cast<const float4 *>(&s_grad[pl[u] * kFusedThreads + qq[u]]);
                const float gr[4] = {gs4.x + gi[u].x, gs4.y + gi[u].y, gs4.z + gi[u].z, gs4.w + gi[u].w};
                float *m = &m4[u].x, *v = &v4[u].x, *pp = &p4[u].x;
                const float a = fa.lr[adam_group(pl[u])];
                #pragma unroll
                for (int c = 0; c < 4; ++c) {
                    m[c] = fa.b1 * m[c] + (1.0f - fa.b1) * gr[c];
                    v[c] = fa.b2 * v[c] + (1.0f - fa.b2) * gr[c] * gr[c];
                    pp[c] -= a * (m[c] * fa.inv_bc1) / (sqrtf(v[c]) * fa.inv_sqrt_bc2 + fa.eps);
                }
                *reinterpret_cast<float4 *>(Mp + ii[u]) = m4[u];
                *reinterpret_cast<float4 *>(Vp + ii[u]) = v4[u];
                *reinterpret_cast<float4 *>(P + ii[u]) = p4[u];
            }
        }
    }
}

void launch_project(const float *P, long long n, long long ld, int D, const ViewTable &vt, const RasterCfg &cfg,
                    float2 *xy, float4 *co, float4 *rgbd, int *radius, int *touched, int *status, float4 *cj,
                    cudaStream_t s) {
    if (ld <= 0) return;
    const int blocks = (int)ceil_div(ld, 256);
    switch (D) {
        case 0: launch_pdl(k_project<0>, blocks, 256, 0, s, P, n, ld, vt, cfg, xy, co, rgbd, radius, touched, status, cj); break;
        case 1: launch_pdl(k_project<1>, blocks, 256, 0, s, P, n, ld, vt, cfg, xy, co, rgbd, radius, touched, status, cj); break;
        case 2: launch_pdl(k_project<2>, blocks, 256, 0, s, P, n, ld, vt, cfg, xy, co, rgbd, radius, touched, status, cj); break;
        default: launch_pdl(k_project<3>, blocks, 256, 0, s, P, n, ld, vt, cfg, xy, co, rgbd, radius, touched, status, cj); break;
    }
}

void launch_project_bwd(const float *P, long long n, long long ld, int D, const ViewTable &vt, const RasterCfg &cfg,
                        const int *radius, const float *acc, long long nrec, float *G, int accumulate,
                        const float *loss_per_view, float *stats, long long stats_ld, const float4 *cj,
                        uint8_t *rows, cudaStream_t s) {
    if (ld <= 0) return;
    const int blocks = (int)ceil_div(ld, 256);
    FusedAdam fa{};
#define GS_PB(DD) launch_pdl(k_project_bwd<DD, false>, blocks, 256, 0, s, const_cast<float *>(P), n, ld, vt, cfg, radius, acc, \
                                                                   nrec, G, accumulate, loss_per_view, stats, stats_ld, fa, \
                                                                   cj, rows)
    switch (D) {
        case 0: GS_PB(0); break;
        case 1: GS_PB(1); break;
        case 2: GS_PB(2); break;
        default: GS_PB(3); break;
    }
#undef GS_PB
}

void launch_project_bwd_adam(float *P, long long n, long long ld, int D, const ViewTable &vt, const RasterCfg &cfg,
                             const int *radius, const float *acc, long long nrec, const float *G_in, float *m,
                             float *v, const float lr[6], float beta1, float beta2, float eps, long long step,
                             const long long *step_dev, float iso_weight, const float *loss_per_view, float *stats,
                             long long stats_ld, cudaStream_t s) {
    if (ld <= 0) return;
    const int blocks = (int)ceil_div(ld, kFusedThreads);
    FusedAdam fa{};
    fa.m = m;
    fa.v = v;
    for (int k = 0; k < 6; ++k) fa.lr[k] = lr[k];
    fa.b1 = beta1;
    fa.b2 = beta2;
    fa.eps = eps;
    const double st = step_dev ? 1.0 : (double)step;  // placeholder when the device counter is used
    fa.inv_bc1 = (float)(1.0 / (1.0 - pow((double)beta1, st)));
    fa.inv_sqrt_bc2 = (float)(1.0 / sqrt(1.0 - pow((double)beta2, st)));
    fa.step_dev = step_dev;
    fa.iso_gscale = n > 0 ? (float)(iso_weight / (double)n) : 0.0f;
    fa.G_in = G_in;
#define GS_PBA(DD)                                                                                              \
    do {                                                                                                        \
        const int smem = (11 + 3 * (DD + 1) * (DD + 1)) * kFusedThreads * (int)sizeof(float);                   \
        static bool attr = false; /* once per process, before any capture uses it */                            \
        if (!attr) {                                                                                            \
            cudaFuncSetAttribute(k_project_bwd<DD, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);    \
            attr = true;                                                                                        \
        }                                                                                                       \
        launch_pdl(k_project_bwd<DD, true>, blocks, kFusedThreads, smem, s, P, n, ld, vt, cfg, radius, acc, nrec,       \
                                                                    nullptr, 0,                                 \
                                                          loss_per_view, stats, stats_ld, fa, nullptr, nullptr); \
    } while (0)
    switch (D) {
        case 0: GS_PBA(0); break;
        case 1: GS_PBA(1); break;
        case 2: GS_PBA(2); break;
        default: GS_PBA(3); break;
    }
#undef GS_PBA
}

}  // namespace gs
