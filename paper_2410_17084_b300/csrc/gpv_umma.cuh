// gpv_umma.cuh -- fifth-generation tensor core (tcgen05) building blocks for sm_103a,
// written as inline PTX: tensor-memory allocation, shared-memory matrix descriptors,
// the instruction descriptor of kind::tf32, the MMA, its commit to an mbarrier, and
// loads of the accumulator from tensor memory.
//
// Operand layout used here: K-major, no swizzle ("interleaved").  A matrix of R rows and
// KC (a multiple of 4) 32-bit elements per row is stored as core matrices of 8 rows x 16
// bytes; element (r, k) sits at
//     (r / 8) * SBO + (k / 4) * LBO + (r % 8) * 16 + (k % 4) * 4      bytes,
// with LBO = 128 (core matrices adjacent along K are contiguous) and SBO = (KC / 4) * 128
// (all K core matrices of one 8-row group, then the next group).  One MMA consumes K = 8
// (two core matrices along K); the next K step starts 2 * LBO bytes further.
#pragma once
#include <stdint.h>

namespace gpv {
namespace umma {

constexpr int kLBO = 128;

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (r, k) in a K-major, unswizzled operand with kc elements per row.
__device__ __forceinline__ int kmajor_offset(int r, int k, int kc)
{
    return (r >> 3) * (kc >> 2) * kLBO + (k >> 2) * kLBO + (r & 7) * 16 + (k & 3) * 4;
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (8-row group)
// byte offsets, each encoded >> 4; bits 46-47 = 1 (descriptor version of this tensor
// core generation); base offset 0; layout type 0 = no swizzle (bits 61-63).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, int lbo, int sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
    return d;
}

// Instruction descriptor of kind::tf32 with an FP32 accumulator, both operands K-major,
// dense, no negation: D format F32 (bits 4-5 = 1), A and B format TF32 (bits 7-9 and
// 10-12 = 2), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor of kind::f16 with BF16 operands and an FP32 accumulator, both
// K-major: D format F32 (bits 4-5 = 1), A and B format BF16 (bits 7-9 and 10-12 = 1).
// With 2-byte elements a core matrix row of 16 bytes holds 8 elements and one MMA
// consumes K = 16, again two core matrices along K.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// ---- tensor memory ------------------------------------------------------------------
// One warp allocates ncols columns (a power of two, >= 32) and writes the address into
// shared memory; the same warp frees them.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_addr(dst_smem)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_after_sync()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Make this thread's ordinary shared-memory stores visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// D (tensor memory) = A * B^T (+ D when accumulate), issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate ? 1u : 0u)
        : "memory");
}

// D (tensor memory) = A * B^T (+ D when accumulate), BF16 operands, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate ? 1u : 0u)
        : "memory");
}

// The mbarrier receives one arrival once every MMA issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t* mbar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
        :: "r"(smem_addr(mbar)) : "memory");
}

// 16 consecutive 32-bit columns of this thread's tensor-memory lane (warp w of the CTA
// reads lanes 32 (w % 4) .. 32 (w % 4) + 31; taddr carries the lane in its upper half).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
          "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
          "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- mbarrier ---------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(mbar)), "r"(count)
                 : "memory");
}

// Wait for the phase of the given parity to complete, giving up after max_iter polls.
// Returns false on time-out.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t max_iter)
{
    const uint32_t a = smem_addr(mbar);
    for (uint32_t it = 0; it < max_iter; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

// TF32 split of an FP32 value: big keeps the 10 explicit mantissa bits the tensor core
// reads, small = x - big (exact), so big * big + big * small + small * big carries about
// 21 bits of each product (the "3xTF32" scheme).
__device__ __forceinline__ void tf32_split(float x, float& big, float& small)
{
    big = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
    small = x - big;
}

}  // namespace umma
}  // namespace gpv
