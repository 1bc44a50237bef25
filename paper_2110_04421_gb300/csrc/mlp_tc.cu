// mlp_tc.cu -- fused forward pass of the surrogate MLP on the 5th-generation
// tensor cores (tcgen05, sm_103a).
//
// One CTA (256 threads) carries 128 samples through every layer:
//   * the layer input a_{l-1} [128 x K] (BF16) lives in shared memory in the
//     K-major 128-byte-swizzled layout the tensor core reads (8-row atoms of
//     1024 B, 16-byte chunk c of row r stored at chunk c ^ (r % 8));
//   * the layer's weights W_l^T [N x K] (BF16, K-major) arrive 64 K-columns at a
//     time in a 32 KB shared buffer, each chunk one cp.async.bulk copy of an
//     image prepared in the swizzled layout (mbarrier transaction count);
//   * one thread issues tcgen05.mma (M = 128, N <= 256, K = 16, BF16 inputs,
//     FP32 accumulate) into a TMEM accumulator of 128 lanes x 256 columns and
//     commits each chunk to an mbarrier; two CTAs share an SM so one's epilogue
//     overlaps the other's MMAs;
//   * the epilogue reads the accumulator with tcgen05.ld (warp w: TMEM lanes
//     32 (w % 4) .. +31, half w / 4 of the columns), adds the bias, applies the
//     GELU (tanh form) and writes the BF16 activations back to shared memory as the next
//     layer's input; after the last layer each warp turns its 32 rows x 32
//     columns around in shared memory so that every global store of the FP32
//     output writes one row's 128 consecutive bytes (a thread per row storing
//     its own columns would touch 32 rows, 32 cache lines, per instruction).
// Every mbarrier wait is bounded: on time-out the kernel records an error,
// frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "gelu.cuh"
#include "mlp_tc.h"

namespace mlptc {

constexpr uint32_t kRows = 128;              // samples per CTA = UMMA M
constexpr uint32_t kThreads = 256;
constexpr uint32_t kAChunkBytes = kRows * 128;  // 128 rows x 64 BF16
constexpr uint32_t kBBufBytes = 256 * 128;      // up to 256 rows x 64 BF16
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kMaxWaitPolls = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of 16-byte chunk c of row r in a K-major SW128 tile (base 1024-aligned)
__device__ __forceinline__ uint32_t sw128(uint32_t r, uint32_t c) { return (r >> 3) * 1024u + (r & 7u) * 128u + (((c ^ r) & 7u) << 4); }

// shared-memory matrix descriptor: start address, LBO 16 B (unused for this
// layout), SBO 1024 B between 8-row atoms, descriptor version 1, 128-byte swizzle
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) |
           ((uint64_t)1u << 46) | ((uint64_t)2u << 61);
}

// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major
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

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar) : "memory");
}

// polls <= 1: one non-blocking test (mbarrier.test_wait)
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t polls)
{
    if (polls <= 1u) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        return done != 0;
    }
    for (uint32_t it = 0; it < polls; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

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

// 16 columns of the warp's 32 TMEM lanes, issued without waiting: the registers
// are read only after tmem_wait16 on the same array (which names them as
// operands, so that no read of them is scheduled before the wait)
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *(const uint32_t *)&h;
}

__device__ __forceinline__ void bulk_load(uint32_t dst_smem, const void *src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst_smem),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// Two CTAs per SM (97 KB of shared memory, 256 TMEM columns each): while one
// runs its GELU epilogue on the CUDA cores the other's MMAs use the tensor core.
// Weight chunks arrive by one bulk copy each, already in the swizzled layout;
// the next layer's first chunk is copied while the epilogue runs.
__global__ void __launch_bounds__(kThreads, 2) mlp_forward_tc_kernel(const FusedArgs g)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t mbar_w, mbar_mma;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023u) & ~(uintptr_t)1023u);
    unsigned char *sA = smem;                               // kMaxKChunks x 16 KB
    unsigned char *sB = smem + kMaxKChunks * kAChunkBytes;  // one 32 KB weight chunk
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
    const uint32_t row0 = blockIdx.x * kRows;
    const uint32_t mw = smem_u32(&mbar_w), mm = smem_u32(&mbar_mma), sB_addr = smem_u32(sB);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mw));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mm));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_abort = 0;
        bulk_load(sB_addr, g.wimg, (uint32_t)g.N[0] * 128u, mw);  // first chunk of layer 0
    }
    // the input tile: x rows (FP32, n_in columns) -> BF16, zero-padded to 64 columns
    for (uint32_t q = tid; q < kRows * 8u; q += kThreads) {
        const uint32_t r = q >> 3, c = q & 7u, row = row0 + r;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const uint32_t k = c * 8u + e;
            v[e] = (row < (uint32_t)g.M && k < (uint32_t)g.n_in) ? g.x[(size_t)row * g.n_in + k] : 0.0f;
        }
        uint4 pk = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                              pack_bf16x2(v[6], v[7]));
        *(uint4 *)(sA + sw128(r, c)) = pk;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    bool ok = true;
    uint32_t gchunk = 0;  // weight chunks consumed so far
    size_t woff = 0;      // byte offset of the next chunk image

    for (int l = 0; l < g.L && ok; ++l) {
        const uint32_t K = (uint32_t)g.K[l], N = (uint32_t)g.N[l], nch = K / 64u;
        if (tid == 0) {
            const uint32_t idesc = idesc_bf16(kRows, N);
            const uint32_t a_base0 = smem_u32(sA);
            for (uint32_t c = 0; c < nch; ++c, ++gchunk) {
                if (!mbar_wait(mw, gchunk & 1u, g.polls)) { s_abort = 1; break; }  // chunk in shared memory
                tc_fence_after();
#pragma unroll
                for (uint32_t kk = 0; kk < 4; ++kk)
                    mma_bf16(tmem, sw128_desc(a_base0 + c * kAChunkBytes + kk * 32u), sw128_desc(sB_addr + kk * 32u),
                             idesc, (c > 0 || kk > 0) ? 1u : 0u);
                mma_commit(mm);
                if (!mbar_wait(mm, gchunk & 1u, g.polls)) { s_abort = 2; break; }  // buffer free again
                woff += (size_t)N * 128u;
                // next chunk: this layer's, or the first of the next layer (overlaps the epilogue)
                if (c + 1 < nch) bulk_load(sB_addr, (const unsigned char *)g.wimg + woff, N * 128u, mw);
                else if (l + 1 < g.L)
                    bulk_load(sB_addr, (const unsigned char *)g.wimg + woff, (uint32_t)g.N[l + 1] * 128u, mw);
            }
        }
        __syncthreads();
        if (s_abort) { ok = false; break; }
        tc_fence_after();
        const uint32_t quad = warp & 3u, half = warp >> 2, row = quad * 32u + lane;
        const uint32_t ncol = N / 2u, c0 = half * ncol;
        const bool last = (l == g.L - 1);
        if (!last) {
            // hidden layer: bias, GELU, BF16 into the next layer's input tile; the
            // next 16 columns' TMEM load is in flight while these 16 are worked
            // (ncol is a multiple of 32)
            const float *bias = g.bias[l];
            auto hidden16 = [&](const uint32_t (&r)[16], uint32_t n0) {
                float v[16];
#pragma unroll
                for (int e = 0; e < 16; e += 4) {  // the bias four columns at a time (16-byte loads)
                    const float4 bb = __ldg((const float4 *)(bias + n0 + e));
                    v[e] = gelu_act(__uint_as_float(r[e]) + bb.x);
                    v[e + 1] = gelu_act(__uint_as_float(r[e + 1]) + bb.y);
                    v[e + 2] = gelu_act(__uint_as_float(r[e + 2]) + bb.z);
                    v[e + 3] = gelu_act(__uint_as_float(r[e + 3]) + bb.w);
                }
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const uint32_t n = n0 + q * 8u;
                    uint4 pk = make_uint4(pack_bf16x2(v[q * 8 + 0], v[q * 8 + 1]), pack_bf16x2(v[q * 8 + 2], v[q * 8 + 3]),
                                          pack_bf16x2(v[q * 8 + 4], v[q * 8 + 5]), pack_bf16x2(v[q * 8 + 6], v[q * 8 + 7]));
                    *(uint4 *)(sA + (n >> 6) * kAChunkBytes + sw128(row, (n & 63u) >> 3)) = pk;
                }
            };
            const uint32_t tb = tmem + ((quad * 32u) << 16) + c0;
            uint32_t ra[16], rb[16];
            tmem_ld16_issue(tb, ra);
            tmem_wait16(ra);
            for (uint32_t cb = 0; cb < ncol; cb += 32u) {
                tmem_ld16_issue(tb + cb + 16u, rb);
                hidden16(ra, c0 + cb);
                tmem_wait16(rb);
                const bool more = cb + 32u < ncol;
                if (more) tmem_ld16_issue(tb + cb + 32u, ra);
                hidden16(rb, c0 + cb + 16u);
                if (more) tmem_wait16(ra);
            }
        }
        for (uint32_t cb = 0; last && cb < ncol; cb += 32u) {
            float v[32];
            tmem_ld32(tmem + ((quad * 32u) << 16) + c0 + cb, v);
            const uint32_t n0 = c0 + cb;
            {
                // output layer: the warp's 32 rows x 32 columns go through shared memory
                // (the layer input is no longer read: the MMAs have completed) so that
                // each global store writes one row's 32 consecutive columns
                float *stg = (float *)sA + warp * 1024u;  // [32 rows][32], float4 q of row r at q ^ (r % 8)
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint32_t n = n0 + 4u * q;
                    float4 o;
                    o.x = v[4 * q] + (n < (uint32_t)g.n_out ? __ldg(g.bias[l] + n) : 0.0f);
                    o.y = v[4 * q + 1] + (n + 1u < (uint32_t)g.n_out ? __ldg(g.bias[l] + n + 1u) : 0.0f);
                    o.z = v[4 * q + 2] + (n + 2u < (uint32_t)g.n_out ? __ldg(g.bias[l] + n + 2u) : 0.0f);
                    o.w = v[4 * q + 3] + (n + 3u < (uint32_t)g.n_out ? __ldg(g.bias[l] + n + 3u) : 0.0f);
                    *(float4 *)(stg + lane * 32u + (((uint32_t)q ^ (lane & 7u)) << 2)) = o;
                }
                __syncwarp();
                const uint32_t col = n0 + lane;
#pragma unroll 4
                for (uint32_t r = 0; r < 32u; ++r) {
                    const uint32_t grow = row0 + quad * 32u + r;
                    const float val = stg[r * 32u + ((((lane >> 2) ^ r) & 7u) << 2) + (lane & 3u)];
                    if (grow < (uint32_t)g.M && col < (uint32_t)g.n_out) g.y[(size_t)grow * g.n_out + col] = val;
                }
                __syncwarp();
            }
        }
        tc_fence_before();
        fence_async_smem();
        __syncthreads();
        tc_fence_after();
    }
    if (!ok && tid == 0) {
        atomicExch(g.err, 1);
        // what the gave-up wait was waiting for is still in flight: the chunk's copy,
        // or its MMAs; let it land (long fixed bound) before TMEM and the buffers go
        if (s_abort == 1) (void)mbar_wait(mw, gchunk & 1u, kMaxWaitPolls);
        else (void)mbar_wait(mm, gchunk & 1u, kMaxWaitPolls);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
    }
}

// weight images: for every layer l and 64-column chunk c, W_l^T[0:N_l, 64c:64c+64] in
// the K-major 128-byte-swizzled layout (one contiguous N_l x 128 B block each)
__global__ void weight_image_kernel(const float *W, int fin, int fout, int k_pad, int n_pad, __nv_bfloat16 *img)
{
    const long total = (long)n_pad * k_pad;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
        const int n = (int)(q / k_pad), k = (int)(q % k_pad);
        const int c = k >> 6, cc = (k & 63) >> 3, e = k & 7;
        const size_t off = (size_t)c * n_pad * 128u + sw128((uint32_t)n, (uint32_t)cc) + (size_t)e * 2u;
        *(__nv_bfloat16 *)((unsigned char *)img + off) = __float2bfloat16(n < fout && k < fin ? W[(long)k * fout + n] : 0.0f);
    }
}

}  // namespace mlptc

cudaError_t mlptc_prepare_weights(const float *W, int fin, int fout, int k_pad, int n_pad, __nv_bfloat16 *img,
                                  cudaStream_t s)
{
    mlptc::weight_image_kernel<<<256, 256, 0, s>>>(W, fin, fout, k_pad, n_pad, img);
    return cudaGetLastError();
}

cudaError_t mlptc_forward(const FusedArgs &g, cudaStream_t s)
{
    static bool attr_set = false;
    const size_t smem = kMaxKChunks * mlptc::kAChunkBytes + mlptc::kBBufBytes + 1024;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(mlptc::mlp_forward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const unsigned blocks = (unsigned)((g.M + mlptc::kRows - 1) / mlptc::kRows);
    if (blocks == 0) return cudaSuccess;
    mlptc::mlp_forward_tc_kernel<<<blocks, mlptc::kThreads, smem, s>>>(g);
    return cudaGetLastError();
}
