// tc_ptx.cuh -- inline-PTX wrappers for the 5th-generation tensor cores (tcgen05),
// the Tensor Memory, mbarriers and bulk / tensor copies, as the surrogate MLP's
// kernels use them (sm_103a).  Written from the PTX ISA: one thread issues
// tcgen05.mma from shared-memory descriptors into a TMEM accumulator and commits
// to an mbarrier; warps read the accumulator back with tcgen05.ld.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace tcx {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of 16-byte chunk c of row r in a K-major tile with the 128-byte
// swizzle (rows of 128 B, 8-row atoms of 1024 B, base 1024-aligned)
__device__ __forceinline__ uint32_t sw128(uint32_t r, uint32_t c)
{
    return (r >> 3) * 1024u + (r & 7u) * 128u + (((c ^ r) & 7u) << 4);
}

// shared-memory matrix descriptor of a K-major SW128 tile: start address, leading
// byte offset 16 B (unused by this layout), stride byte offset 1024 B between
// 8-row atoms, descriptor version 1, 128-byte swizzle
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) |
           ((uint64_t)1u << 46) | ((uint64_t)2u << 61);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major
__device__ __forceinline__ uint32_t idesc_bf16(uint32_t M, uint32_t N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

// the issuing thread's tcgen05 operations so far arrive on mbar when complete
__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count));
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    return done != 0;
}

// non-blocking test of the phase of the given parity
__device__ __forceinline__ bool mbar_test(uint32_t mbar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    return done != 0;
}

// wait for the phase of the given parity, at most `polls` tries (potentially
// blocking ones); false = gave up.  polls <= 1: one non-blocking test.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t polls)
{
    if (polls <= 1u) return mbar_test(mbar, parity);
    for (uint32_t it = 0; it < polls; ++it)
        if (mbar_try(mbar, parity)) return true;
    return false;
}

// the same, also giving up as soon as *abort is set by another thread
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t mbar, uint32_t parity, uint32_t polls,
                                                   const volatile int *abort)
{
    if (polls <= 1u) return mbar_test(mbar, parity);
    for (uint32_t it = 0; it < polls; ++it) {
        if (mbar_try(mbar, parity)) return true;
        if (*abort) return false;
    }
    return false;
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// warp-wide: allocate / free `cols` TMEM columns (power of two >= 32); the address
// lands in shared memory at dst
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t cols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(dst_smem), "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(cols));
}

// warp-wide: 32 consecutive FP32 columns of the accumulator, one TMEM lane per thread
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// bulk copy global -> shared of `bytes` (16-byte multiple, both ends 16-byte
// aligned), completing as a transaction count on mbar
__device__ __forceinline__ void bulk_load(uint32_t dst_smem, const void *src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst_smem),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void expect_tx(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}

// tiled 2-D tensor copy global -> shared through a tensor map (x = innermost
// coordinate, in elements; here always a multiple of 64 BF16 = 128 bytes)
__device__ __forceinline__ void tma_load_2d(uint32_t dst_smem, const void *tmap, int32_t x, int32_t y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            dst_smem),
        "l"(tmap), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

}  // namespace tcx
