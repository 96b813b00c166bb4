// tcgen05.cuh -- the 5th-generation tensor-core pieces shared by the kernels
// that run dense layers on it (the densify / prune predictor, the anchor
// decoder): shared-memory operand layout and descriptors, the BF16 MMA with
// FP32 accumulation in tensor memory, its commit to an mbarrier and the
// bounded wait, tensor-memory loads, allocation and release.
#pragma once
#include <cstdint>

#include <cuda_bf16.h>

namespace gs {

constexpr long long kSpin = 1 << 24;  // default bound of an mbarrier wait (polls)

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Element offset of (row, k) in a K-major no-swizzle operand with `kgroups`
// core matrices along K per 8-row group.
__device__ __forceinline__ int cm_off(int row, int k, int kgroups) {
    return (((row >> 3) * kgroups + (k >> 3)) << 6) + ((row & 7) << 3) + (k & 7);
}

// Shared-memory matrix descriptor (tcgen05): start >> 4, leading byte offset
// >> 4 at bit 16, stride byte offset >> 4 at bit 32, version 1 at bit 46,
// no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | ((uint64_t)1 << 46);
}

// The same for an MN-major no-swizzle operand (core matrix = 8 K-rows of 8
// contiguous M/N elements): the leading offset is the stride between core
// matrices along K, the stride offset the one between 8-element groups along
// M/N.
__device__ __forceinline__ uint64_t smem_desc_mn(uint32_t saddr, uint32_t k_stride, uint32_t mn_stride) {
    return smem_desc(saddr, k_stride, mn_stride);
}

// Instruction descriptor, kind::f16: FP32 accumulate (bit 4), BF16 A (bit 7)
// and B (bit 10), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t M, uint32_t N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// Both operands MN-major (transpose A at bit 15, transpose B at bit 16).
__host__ __device__ constexpr uint32_t idesc_bf16_mn(uint32_t M, uint32_t N) {
    return idesc_bf16(M, N) | (1u << 15) | (1u << 16);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, bool acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"((uint32_t)acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(smem_addr(mbar)));
}

// Wait for the mbarrier phase `parity`, giving up after `polls` polls (0:
// at once, without polling); false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, long long polls = kSpin) {
    uint32_t done = 0;
    for (long long it = 0; it < polls && !done; ++it)
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(smem_addr(mbar)), "r"(parity));
    return done != 0;
}

// 16 consecutive FP32 columns of this thread's TMEM lane (row) into v.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    #pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// 64 columns starting at `col` of this thread's row.
__device__ __forceinline__ void tmem_row64(uint32_t tmem, int col, float *v) {
    const uint32_t lane_base = (uint32_t)((threadIdx.x >> 5) * 32) << 16;
    #pragma unroll
    for (int c = 0; c < 64; c += 16) tmem_ld16(tmem + lane_base + (uint32_t)(col + c), v + c);
}

// Operand arrays start on 128-byte boundaries (descriptors need 16).
// Columns [c0, c0 + 8) of this thread's row (one core-matrix row, 16 bytes),
// rounded to BF16 (round to nearest even), as one 16-byte shared store.
__device__ __forceinline__ void store_row8(__nv_bfloat16 *base, int row, int c0, int kgroups, const float *v) {
    uint4 u;
    __nv_bfloat162 b;
    b = __floats2bfloat162_rn(v[0], v[1]); u.x = *reinterpret_cast<uint32_t *>(&b);
    b = __floats2bfloat162_rn(v[2], v[3]); u.y = *reinterpret_cast<uint32_t *>(&b);
    b = __floats2bfloat162_rn(v[4], v[5]); u.z = *reinterpret_cast<uint32_t *>(&b);
    b = __floats2bfloat162_rn(v[6], v[7]); u.w = *reinterpret_cast<uint32_t *>(&b);
    *reinterpret_cast<uint4 *>(base + cm_off(row, c0, kgroups)) = u;
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t cols) {
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_addr(slot)),
                     "r"(cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
}

__device__ __forceinline__ void tmem_free(uint32_t tmem, uint32_t cols) {
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem),
                                               "r"(cols));
}

}  // namespace gs
