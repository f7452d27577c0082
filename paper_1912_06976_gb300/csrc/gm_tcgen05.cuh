// gm_tcgen05.cuh -- inline-PTX wrappers for the 5th-generation tensor cores of sm_103a:
// tensor-memory allocation, shared-memory matrix descriptors, tcgen05.mma (kind::f16,
// BF16 x BF16 -> FP32), commits to an mbarrier with bounded waits, and tcgen05.ld.
//
// Operand layout used throughout (no swizzle, K-major): a tile of R rows x 64 K-elements (BF16)
// is stored as core matrices of 8 rows x 16 bytes; core matrix (row / 8, k / 8) starts at byte
//   (row / 8) * 1024 + (k / 8) * 128
// and row (row % 8) of it at + 16 * (row % 8).  In descriptor terms the leading-dimension byte
// offset (next core matrix along K) is 128 and the stride-dimension byte offset (next group of
// 8 rows) is 1024; one MMA consumes K = 16, i.e. two core matrices, and the k-th MMA of a tile
// starts 256 * k bytes in.
#pragma once
#include <cstdint>

namespace gm {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) of a K-major no-swizzle tile with 64 K-elements per row
__device__ __forceinline__ uint32_t tile_offset(int row, int kcore) {
    return (uint32_t)((row >> 3) * 1024 + kcore * 128 + (row & 7) * 16);
}

// shared-memory matrix descriptor: start address, LBO 128, SBO 1024, descriptor version 1,
// base offset 0, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t instr_desc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// one warp: allocate `cols` TMEM columns (a power of two >= 32) and write the base to *dst
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_free(uint32_t base, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols));
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;"); }
// make this thread's generic-proxy shared-memory writes visible to the tensor cores
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;"); }

// D[tmem] (+)= A[smem] * B[smem]^T, M x N x 16; accumulate = false overwrites D
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"((uint32_t)accumulate));
}

// the mbarrier at `bar` receives one arrival when every earlier tcgen05 op of this thread is done
__device__ __forceinline__ void commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(bar)));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// wait for the phase with the given parity to complete; false after `limit` polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long limit) {
    uint32_t done = 0;
    for (long it = 0; it < limit && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity));
    }
    return done != 0;
}

// 32 lanes x 8 consecutive 32-bit columns from TMEM (lane = the warp's quarter + lane id)
__device__ __forceinline__ void tmem_ld8(uint32_t addr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
}  // namespace gm
