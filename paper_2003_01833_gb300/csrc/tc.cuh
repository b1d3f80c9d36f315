// Inline-PTX helpers for the 5th-generation tensor cores of sm_103a: tensor
// memory (TMEM) allocation, tcgen05.mma with shared-memory operand
// descriptors, completion through an mbarrier, and tcgen05.ld of the
// accumulator.  Only the forms the kernels of this library use.
//
// Operand layout: K-major tiles with the 128-byte swizzle.  A tile of R rows
// (R a multiple of 8) holds 128 bytes of K per row (32 tf32 or 64 bf16
// values); row r lives at r * 128 bytes and its 16-byte chunk c at chunk
// position c ^ (r % 8).  Tiles start on 1024-byte boundaries, so groups of
// 8 rows are 1024 bytes apart (the descriptor's stride offset), and one MMA
// step of K (32 bytes) advances the descriptor's start address by 32 bytes.
#pragma once

#include <stdint.h>

namespace tagi {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element k (4-byte elements, 0 <= k < 32) of row r in a
// 128B-swizzled K-major tile
__device__ __forceinline__ uint32_t swz4(int r, int k) { return r * 128 + ((((k >> 2) ^ (r & 7))) << 4) + ((k & 3) << 2); }

// round to the nearest tf32 value (ties away from zero); low 13 bits zero
__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// shared-memory matrix descriptor of a 128B-swizzled K-major tile at `addr`
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);  // start address / 16
    d |= (uint64_t)1 << 16;                          // leading offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride offset: 8-row groups 1024 B apart
    d |= (uint64_t)1 << 46;                          // descriptor version of sm_10x
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// instruction descriptor: D float32, A and B tf32 (kind::tf32), both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// instruction descriptor: D float32, A and B bf16 (kind::f16), both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// wait for the completion of the phase with parity `parity`; gives up after
// `limit` SM clocks and returns false
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit)
{
    const uint32_t a = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// the mbarrier completes one phase once every tcgen05 operation this thread
// issued before has completed
__device__ __forceinline__ void commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// one warp: allocate `ncols` TMEM columns (a power of two >= 32); the base
// address is written to *slot
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, kind::tf32; accumulate = 0 overwrites D
__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 with bf16 operands
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}

// 8 consecutive 32-bit TMEM columns of this thread's lane (warp w of a
// 4-warp group reads lanes 32 (w % 4) ... 32 (w % 4) + 31); waits for them
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v)
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
}  // namespace tagi
