// labs_tc.cuh -- 5th-generation tensor cores on sm_103a as inline PTX: tensor memory
// (TMEM) allocation, tcgen05.mma with BF16 operands in shared memory and an FP32
// accumulator in TMEM, tcgen05.ld of the accumulator, and two-dimensional tiled TMA loads
// (cp.async.bulk.tensor) that stage the operands.  Used by the network's GEMMs.
//
// Operand layouts in shared memory, without swizzling; a core matrix is 8 rows of 16
// bytes stored contiguously (128 bytes).
//  - K-major (the forward products): a core-matrix row is 8 BF16 values of K for one M
//    (or N) index.  Core matrices adjacent in K lie `lbo` bytes apart and those adjacent
//    in M (N) `sbo` bytes apart.  The network keeps every operand row 16 bytes after the
//    previous one (sbo = 128): a block of 8 K values for all rows is one contiguous
//    column of 16-byte rows, and a shift of the operand by whole rows is a shift of the
//    descriptor's start address by 16 bytes a row.
//  - MN-major (the weight gradients, whose K is the activation rows): a core-matrix row
//    is 8 BF16 values of M (N) for one K index.  The leading byte offset `lbo` steps
//    along K (the next 8 rows) and the stride byte offset `sbo` along M (N); the same
//    staged columns serve, with lbo = 128 and sbo = one column.
#pragma once

#include <cuda.h>

#include <cstdint>

#include "labs_async.cuh"

namespace labsgpu {

// Shared-memory matrix descriptor (tcgen05): start address, leading (K) and stride (M/N)
// byte offsets, each in 16-byte units; descriptor version 1 (bits 46-47); base offset
// 0; no swizzling (layout type 0 in bits 61-63).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4
// in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// TMEM columns for the CTA (a power of two >= 32); one whole warp calls it.  The base
// address lands in the shared word at `slot`.
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] x B[smem]; issued by one thread.
__device__ __forceinline__ void tc_mma_bf16(uint32_t taddr, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            bool accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// The barrier at `bar` receives one arrival when every MMA this thread issued before
// has completed.
__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 16 consecutive 32-bit columns of this thread's TMEM lane (32x32b shape: thread t of
// warp w reads lane 32 (w % 4) + t); complete after tc_wait_ld.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_wait_ld()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Tile (x, y) of a two-dimensional tensor map into shared memory at dst, counted on
// barrier bar; coordinates outside the tensor read zeros.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

}  // namespace labsgpu
