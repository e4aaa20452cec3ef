// Fifth-generation tensor-core (tcgen05) building blocks for sm_103a, as inline PTX: tensor
// memory allocation, the shared-memory matrix descriptor of a no-swizzle K-major operand, the
// instruction descriptor of a BF16 x BF16 -> FP32 MMA, the MMA, its completion through an
// mbarrier, and loads from tensor memory.
//
// Operand layout (no swizzle, K-major): the matrix is tiled by core matrices of 8 rows x 16
// bytes (8 BF16 values of one row along K); a core matrix is 128 contiguous bytes, row r at
// 16 r.  The core matrices of one 8-row group follow each other along K, and the row groups
// follow each other: element (r, k) of a matrix with Kd columns sits at byte
// (r / 8) * 16 Kd + (k / 8) * 128 + 16 (r % 8) + 2 (k % 8), so the core matrices adjacent along K
// are 128 bytes apart (the descriptor's leading byte offset) and those adjacent along the rows
// 16 Kd bytes apart (its stride byte offset).
#pragma once

#include <cstdint>

namespace {

__device__ __forceinline__ uint32_t tc_smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (r, k) of an operand with Kd columns in the layout above.
__host__ __device__ __forceinline__ uint32_t tc_kmajor_offset(int Kd, int r, int k) {
    return (uint32_t)((r >> 3) * 16 * Kd + (k >> 3) * 128 + 16 * (r & 7) + 2 * (k & 7));
}

// Shared-memory matrix descriptor: start address, leading byte offset (between core matrices
// adjacent along K), stride byte offset (between core matrices adjacent along M or N), all in
// 16-byte units; bits 46-48 hold the descriptor version 1; base offset 0; no swizzle.
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16, dense: D in FP32 (bits 4-5 = 1), A and B in BF16
// (bits 7-9 and 10-12 = 1), both K-major (bits 15 and 16 clear), N / 8 in bits 17-22, M / 16 in
// bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Tensor-memory allocation of ncols columns (a power of 2 >= 32) by one whole warp; the base
// address is written to *slot.  The permit is released at once: a CTA allocates once.
__device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Ordering of tensor-core operations across a thread synchronisation.
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Shared-memory writes of this thread made visible to the tensor core's reads (async proxy).
__device__ __forceinline__ void tc_fence_proxy() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D = A B^T, or D += A B^T when acc != 0: A [M x K] and B [N x K] in shared memory (descriptors),
// D [M x N] FP32 in tensor memory (lane = row, column = n).  Issued by one thread.
__device__ __forceinline__ void tc_mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// One arrival on the mbarrier once every MMA this thread issued before has completed.
__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     tc_smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ void tc_mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem_addr(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// True once the mbarrier's phase of the given parity has completed.
__device__ __forceinline__ bool tc_mbar_try_wait(uint64_t* mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(tc_smem_addr(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 16 consecutive 32-bit columns, starting at taddr's column, of the 32 tensor-memory lanes of
// this warp's quarter (thread t: lane t of the quarter); tc_wait_ld before the values are used.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace
