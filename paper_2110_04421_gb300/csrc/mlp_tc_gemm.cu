// mlp_tc_gemm.cu -- the surrogate MLP's training GEMMs on the 5th-generation
// tensor cores (tcgen05, sm_103a): the forward pass that keeps what the backward
// pass needs, the input gradients (dgrad) and the weight gradients (wgrad).
//
// C[M x N] = A[M x K] . B[N x K]^T, BF16 operands with K contiguous in memory,
// FP32 accumulation.  One CTA (320 threads) computes a 128 x BN tile of C over
// its K range (a split of K for the weight gradients):
//   * warp 0, one thread: TMA (cp.async.bulk.tensor, 128-byte swizzle) brings
//     64-column K chunks of A (128 rows) and B (BN rows) into a ring of two
//     shared-memory stages (four for the weight gradients); each stage completes
//     on its "full" mbarrier;
//   * warp 1, one thread: four tcgen05.mma (M = 128, N = BN, K = 16) per chunk
//     into the TMEM accumulator (128 lanes x BN columns), then tcgen05.commit to
//     the stage's "empty" mbarrier (the buffer may be refilled) and, after the
//     last chunk, to the accumulator's mbarrier;
//   * warps 2-9: the epilogue, two warps per 32 TMEM lanes (rows), each reading
//     every other block of 32 columns with tcgen05.ld and writing what the MLP
//     needs (bias, GELU (tanh form) or its derivative, FP32 / BF16 / transposed
//     BF16 stores).
// Two CTAs of the two-stage kernel share an SM (97 KB of shared memory and 256
// TMEM columns each), so one CTA's epilogue overlaps the other's copies and
// MMAs.  Operand tiles are read only from this GPU's global memory (no cluster
// multicast).
// Every mbarrier wait is bounded: a wait that gives up records an error, the
// kernel waits (with a long fixed bound) for the copies and MMAs it started,
// frees its TMEM and returns.
#include <cuda.h>  // CUtensorMap and its enums; the encoder comes from the runtime's driver entry point
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "gelu.cuh"
#include "mlp_tc.h"
#include "tc_ptx.cuh"

namespace mlpgemm {

using namespace tcx;

constexpr uint32_t kBM = 128;
constexpr uint32_t kThreads = 320;
constexpr uint32_t kATile = kBM * 128;     // 128 rows x 64 BF16
constexpr uint32_t kBTileMax = 256 * 128;  // up to 256 rows x 64 BF16
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kDrainPolls = 1u << 26;  // bound of the waits for work already started
// dynamic shared memory of a kernel with S stages (S = 2: two CTAs per SM; the
// weight gradients, 128 CTAs or fewer, take 4 stages and one CTA per SM)
constexpr size_t smem_bytes(uint32_t S) { return S * (kATile + kBTileMax) + 1024; }


__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *(const uint32_t *)&h;
}

struct KArgs {
    TcGemm g;
    uint32_t bn;  // N tile (multiple of 16, <= 256)
};

// A warp's 32 rows x 32 FP32 columns between registers (a thread per row) and
// global memory, through a [32][36] shared tile: each global access instruction
// then covers 4 rows x 128 contiguous bytes instead of 32 rows x 16 bytes (the
// padding keeps both shared-memory access patterns free of bank conflicts).
// base = the block's first row at its first column; rows at or past nrows are
// neither read nor written.
constexpr uint32_t kStgPitch = 36;

__device__ __forceinline__ void rows_store_f32(float *stg, const float (&v)[32], float *base, size_t ld, uint32_t nrows,
                                               uint32_t lane)
{
#pragma unroll
    for (uint32_t q = 0; q < 8u; ++q)
        *(float4 *)(stg + lane * kStgPitch + 4u * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    __syncwarp();
#pragma unroll
    for (uint32_t i = 0; i < 8u; ++i) {
        const uint32_t r = 4u * i + (lane >> 3), c = 4u * (lane & 7u);
        const float4 x = *(const float4 *)(stg + r * kStgPitch + c);
        if (r < nrows) *(float4 *)(base + (size_t)r * ld + c) = x;
    }
    __syncwarp();
}

__device__ __forceinline__ void rows_load_f32(float *stg, float (&v)[32], const float *base, size_t ld, uint32_t nrows,
                                              uint32_t lane)
{
#pragma unroll
    for (uint32_t i = 0; i < 8u; ++i) {
        const uint32_t r = 4u * i + (lane >> 3), c = 4u * (lane & 7u);
        const float4 x = r < nrows ? __ldg((const float4 *)(base + (size_t)r * ld + c)) : make_float4(0.f, 0.f, 0.f, 0.f);
        *(float4 *)(stg + r * kStgPitch + c) = x;
    }
    __syncwarp();
#pragma unroll
    for (uint32_t q = 0; q < 8u; ++q) {
        const float4 x = *(const float4 *)(stg + lane * kStgPitch + 4u * q);
        v[4 * q] = x.x;
        v[4 * q + 1] = x.y;
        v[4 * q + 2] = x.z;
        v[4 * q + 3] = x.w;
    }
    __syncwarp();
}

template <uint32_t kStages>
__global__ void __launch_bounds__(kThreads, 2) tc_gemm_kernel(const __grid_constant__ CUtensorMap ta,
                                                              const __grid_constant__ CUtensorMap tb, const KArgs ka)
{
    const TcGemm &g = ka.g;
    const uint32_t BN = ka.bn;
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t full[kStages], empty[kStages], accb;
    __shared__ uint32_t s_tmem, s_issued, s_consumed;
    __shared__ int s_abort;
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023u) & ~(uintptr_t)1023u);
    const uint32_t stage_bytes = kATile + BN * 128u;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
    const uint32_t m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const uint32_t k0 = blockIdx.z * (uint32_t)g.kps;
    const uint32_t k1 = min((uint32_t)g.K, k0 + (uint32_t)g.kps);
    const uint32_t nch = k1 > k0 ? (k1 - k0 + 63u) / 64u : 0u;

    if (warp == 1) tmem_alloc(smem_u32(&s_tmem), kTmemCols);
    if (tid == 0) {
        for (uint32_t s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(&accb), 1);
        fence_mbar_init();
        s_abort = 0;
        s_issued = 0;
        s_consumed = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    volatile int *abort = &s_abort;

    if (warp == 0) {
        if (lane == 0) {  // producer
            for (uint32_t c = 0; c < nch; ++c) {
                const uint32_t s = c % kStages;
                if (c >= kStages && !mbar_wait_or_abort(smem_u32(&empty[s]), ((c / kStages) - 1u) & 1u, g.polls, abort)) {
                    *abort = 1;
                    break;
                }
                if (*abort) break;
                unsigned char *sa = smem + s * stage_bytes;
                const uint32_t fb = smem_u32(&full[s]);
                expect_tx(fb, stage_bytes);
                tma_load_2d(smem_u32(sa), &ta, (int32_t)(k0 + c * 64u), (int32_t)m0, fb);
                tma_load_2d(smem_u32(sa + kATile), &tb, (int32_t)(k0 + c * 64u), (int32_t)n0, fb);
                *(volatile uint32_t *)&s_issued = c + 1u;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            const uint32_t idesc = idesc_bf16(kBM, BN);
            bool done = true;
            for (uint32_t c = 0; c < nch; ++c) {
                const uint32_t s = c % kStages;
                if (!mbar_wait_or_abort(smem_u32(&full[s]), (c / kStages) & 1u, g.polls, abort)) {
                    *abort = 1;
                    done = false;
                    break;
                }
                *(volatile uint32_t *)&s_consumed = c + 1u;
                tc_fence_after();
                const uint32_t a_base = smem_u32(smem + s * stage_bytes), b_base = a_base + kATile;
#pragma unroll
                for (uint32_t kk = 0; kk < 4; ++kk)
                    mma_bf16(tmem, sw128_desc(a_base + kk * 32u), sw128_desc(b_base + kk * 32u), idesc,
                             (c > 0 || kk > 0) ? 1u : 0u);
                mma_commit(smem_u32(&empty[s]));
            }
            if (done) mma_commit(smem_u32(&accb));
        }
    } else {  // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, every other 32 columns
        const uint32_t ew = warp - 2u, half = ew >> 2;
        const uint32_t q = warp & 3u, row = q * 32u + lane, gm = m0 + row;
        const bool ok = nch > 0 ? mbar_wait_or_abort(smem_u32(&accb), 0u, g.polls, abort) : true;
        if (!ok) *abort = 1;
        tc_fence_after();
        double sq = 0.0;  // MSE: this row's squared errors
        // bias-gradient partials: each epilogue warp's column sums over its 32 rows,
        // through a transposed tile in the (no longer read) operand buffers
        const bool colsums = g.bpart && (g.epi == TC_EPI_DGRAD || g.epi == TC_EPI_MSE);
        float *tile = (float *)smem + ew * (32u * 33u);           // [32 columns][33]
        float *wsum = (float *)smem + 8u * 32u * 33u + q * 256u;  // the quarter's sums of BN <= 256 columns
        float *stg = (float *)smem + 8u * 32u * 33u + 4u * 256u + ew * (32u * kStgPitch);  // this warp's row tile
        const uint32_t r0 = m0 + q * 32u;  // the warp's first row
        const uint32_t nrows = r0 < (uint32_t)g.M ? min(32u, (uint32_t)g.M - r0) : 0u;
        if (ok) {
            const bool rv = gm < (uint32_t)g.M;
            for (uint32_t cb = half * 32u; cb < BN; cb += 64u) {
                float v[32];
                if (nch > 0) {
                    tmem_ld32(tmem + ((q * 32u) << 16) + cb, v);
                } else {
#pragma unroll
                    for (int e = 0; e < 32; ++e) v[e] = 0.0f;
                }
                const uint32_t n = n0 + cb;
                if (n >= (uint32_t)g.N) break;  // warp-uniform
                // 32 whole columns: 16-byte vector loads and stores along the row
                // (row strides and n are multiples of 4 elements); else one by one
                const bool full32 = n + 32u <= (uint32_t)g.N;
                if (g.epi == TC_EPI_WGRAD) {
                    float *part = g.outf + (size_t)blockIdx.z * g.M * g.ldf;
                    if (full32) {
                        rows_store_f32(stg, v, part + (size_t)r0 * g.ldf + n, g.ldf, nrows, lane);
                    } else if (rv) {
                        float *o = part + (size_t)gm * g.ldf + n;
                        for (int e = 0; e < 32; ++e)
                            if (n + e < (uint32_t)g.N) o[e] = v[e];
                    }
                    continue;
                }
                // bias (OUTPUT, HIDDEN, MSE)
                if (g.epi != TC_EPI_DGRAD) {
                    if (full32) {
#pragma unroll
                        for (int c4 = 0; c4 < 8; ++c4) {
                            const float4 bb = __ldg((const float4 *)(g.bias + n) + c4);
                            v[4 * c4] += bb.x;
                            v[4 * c4 + 1] += bb.y;
                            v[4 * c4 + 2] += bb.z;
                            v[4 * c4 + 3] += bb.w;
                        }
                    } else {
                        for (int e = 0; e < 32; ++e) v[e] += (n + e < (uint32_t)g.N) ? __ldg(g.bias + n + e) : 0.0f;
                    }
                }
                if (g.epi == TC_EPI_OUTPUT) {
                    if (full32) {
                        rows_store_f32(stg, v, g.outf + (size_t)r0 * g.ldf + n, g.ldf, nrows, lane);
                    } else if (rv) {
                        float *o = g.outf + (size_t)gm * g.ldf + n;
                        for (int e = 0; e < 32; ++e)
                            if (n + e < (uint32_t)g.N) o[e] = v[e];
                    }
                    continue;
                }
                // the FP32 value this epilogue keeps: z (HIDDEN), dz (DGRAD, MSE)
                float other[32];
                if (g.epi != TC_EPI_HIDDEN && full32) {  // DGRAD: the pre-activation; MSE: the target
                    if (g.epi == TC_EPI_DGRAD) rows_load_f32(stg, other, g.zin + (size_t)r0 * g.ldz + n, g.ldz, nrows, lane);
                    else rows_load_f32(stg, other, g.y + (size_t)r0 * g.N + n, (size_t)g.N, nrows, lane);
                } else if (rv && g.epi != TC_EPI_HIDDEN) {
                    const float *src = g.epi == TC_EPI_DGRAD ? g.zin + (size_t)gm * g.ldz + n : g.y + (size_t)gm * g.N + n;
                    for (int e = 0; e < 32; ++e) other[e] = (n + e < (uint32_t)g.N) ? __ldg(src + e) : 0.0f;
                } else {
#pragma unroll
                    for (int e = 0; e < 32; ++e) other[e] = 0.0f;
                }
                if (g.epi == TC_EPI_DGRAD) {
#pragma unroll
                    for (int e = 0; e < 32; ++e) v[e] = v[e] * gelu_act_grad(other[e]);
                } else if (g.epi == TC_EPI_MSE) {
                    float sq32 = 0.0f;  // this block's 32 squares in FP32, then one FP64 add
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        const float d = v[e] - other[e];
                        if (rv && n + e < (uint32_t)g.N) sq32 += d * d;
                        v[e] = 2.0f * d * g.scale;
                    }
                    sq += (double)sq32;
                }
                if (g.outf) {
                    if (full32) {
                        rows_store_f32(stg, v, g.outf + (size_t)r0 * g.ldf + n, g.ldf, nrows, lane);
                    } else if (rv) {
                        float *o = g.outf + (size_t)gm * g.ldf + n;
                        for (int e = 0; e < 32; ++e)
                            if (n + e < (uint32_t)g.N) o[e] = v[e];
                    }
                }
                if (colsums) {  // lane e's column: its 32 rows in order
#pragma unroll
                    for (int e = 0; e < 32; ++e) tile[e * 33 + lane] = rv ? v[e] : 0.0f;
                    __syncwarp();
                    float cs = 0.0f;
#pragma unroll 8
                    for (int r = 0; r < 32; ++r) cs += tile[lane * 33 + r];
                    wsum[cb + lane] = cs;
                    __syncwarp();
                }
                if (g.epi == TC_EPI_HIDDEN) {
#pragma unroll
                    for (int e = 0; e < 32; ++e) v[e] = gelu_act(v[e]);
                }
                // the BF16 copies: row-major (whole 64-byte row segments through the
                // row tile), then transposed (for each column the warp's 32 rows are 64
                // contiguous bytes)
                if (full32) {  // row-major through the row tile: 4 lanes per row's 64 bytes
                    uint32_t *st32 = (uint32_t *)stg;  // [32 rows][20 words]
#pragma unroll
                    for (int c8 = 0; c8 < 4; ++c8)
                        *(uint4 *)(st32 + lane * 20u + 4u * c8) =
                            make_uint4(pack_bf16x2(v[c8 * 8 + 0], v[c8 * 8 + 1]), pack_bf16x2(v[c8 * 8 + 2], v[c8 * 8 + 3]),
                                       pack_bf16x2(v[c8 * 8 + 4], v[c8 * 8 + 5]), pack_bf16x2(v[c8 * 8 + 6], v[c8 * 8 + 7]));
                    __syncwarp();
#pragma unroll
                    for (uint32_t i = 0; i < 4u; ++i) {
                        const uint32_t r = 8u * i + (lane >> 2), c = lane & 3u;
                        const uint4 x = *(const uint4 *)(st32 + r * 20u + 4u * c);
                        if (r < nrows) *(uint4 *)(g.outb + (size_t)(r0 + r) * g.ldo + n + 8u * c) = x;
                    }
                    __syncwarp();
                } else if (rv) {
                    for (int e = 0; e < 32; ++e)
                        if (n + e < (uint32_t)g.N) g.outb[(size_t)gm * g.ldo + n + e] = __float2bfloat16(v[e]);
                }
                if (rv) {
#pragma unroll
                    for (int e = 0; e < 32; ++e)
                        if (n + e < (uint32_t)g.N) g.outt[(size_t)(n + e) * g.ldt + gm] = __float2bfloat16(v[e]);
                }
            }
        }
        if (g.epi == TC_EPI_MSE) {  // the CTA's squared errors, rows in a fixed order
            __shared__ double s_sq[2][kBM];
            s_sq[half][row] = sq;
            asm volatile("bar.sync 1, 256;\n" ::: "memory");  // the eight epilogue warps
            if (row == 0 && half == 0) {
                double t = 0.0;
                for (uint32_t r = 0; r < kBM; ++r) t += s_sq[0][r] + s_sq[1][r];
                g.loss_part[blockIdx.x] = t;
            }
        }
        if (colsums) {  // the CTA's column sums: the four warps' sums in warp order
            asm volatile("bar.sync 1, 256;\n" ::: "memory");
            const float *ws = (const float *)smem + 8u * 32u * 33u;
            for (uint32_t c = half * kBM + row; c < BN && n0 + c < (uint32_t)g.N; c += 2u * kBM) {
                const float t = ok ? (ws[c] + ws[256u + c]) + (ws[512u + c] + ws[768u + c]) : 0.0f;
                g.bpart[(size_t)blockIdx.x * g.N + n0 + c] = t;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort) {
        atomicExch(g.err, 1);
        // copies issued but never consumed, then the MMAs already issued, land
        // before the buffers and the accumulator are given up
        for (uint32_t c = s_consumed; c < s_issued; ++c)
            (void)mbar_wait(smem_u32(&full[c % kStages]), (c / kStages) & 1u, kDrainPolls);
        if (s_consumed > 0) {
            const uint32_t c = s_consumed - 1u;
            (void)mbar_wait(smem_u32(&empty[c % kStages]), (c / kStages) & 1u, kDrainPolls);
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// ------------------------------------------------------------------ host side
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encoder()
{
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)p;
    });
    return fn;
}

// a 2-D BF16 tensor [rows x cols] with row stride ld elements, read in boxes of
// 64 columns x box_rows rows with the 128-byte swizzle; zeros outside
static bool make_map(CUtensorMap *m, const void *base, uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_rows)
{
    EncodeTiled enc = encoder();
    if (!enc || ((uintptr_t)base & 15u) || (ld * 2u) % 16u || rows == 0 || cols == 0) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {ld * 2u};
    const cuuint32_t box[2] = {64u, box_rows};
    const cuuint32_t estr[2] = {1u, 1u};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace mlpgemm

cudaError_t mlptc_gemm(const TcGemm &g, cudaStream_t s)
{
    using namespace mlpgemm;
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(tc_gemm_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(2));
        if (attr_err == cudaSuccess)
            attr_err = cudaFuncSetAttribute(tc_gemm_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(4));
    });
    if (attr_err != cudaSuccess) return attr_err;
    if (g.M <= 0 || g.N <= 0 || g.K <= 0 || g.kps <= 0 || g.kps % 64 || !g.err) return cudaErrorInvalidValue;
    if ((g.epi == TC_EPI_HIDDEN || g.epi == TC_EPI_DGRAD || g.epi == TC_EPI_MSE) &&
        (g.ldo % 8 || !g.outb || !g.outt || (!g.outf && !g.bpart) || (g.epi == TC_EPI_HIDDEN && !g.outf)))
        return cudaErrorInvalidValue;
    if (g.bpart && g.N > 256) return cudaErrorInvalidValue;  // one column tile per CTA row block
    if (g.ldf % 4 || (g.epi == TC_EPI_DGRAD && g.ldz % 4) || (g.epi == TC_EPI_MSE && (!g.y || !g.loss_part || g.N % 4)))
        return cudaErrorInvalidValue;
    if (g.epi == TC_EPI_MSE && g.N > 256) return cudaErrorInvalidValue;  // one column tile per CTA row block
    KArgs ka{};
    ka.g = g;
    const uint32_t n16 = ((uint32_t)g.N + 15u) / 16u * 16u;
    ka.bn = n16 < 256u ? n16 : 256u;
    CUtensorMap ta, tb;
    if (!make_map(&ta, g.A, (uint64_t)g.M, (uint64_t)g.K, (uint64_t)g.lda, kBM) ||
        !make_map(&tb, g.B, (uint64_t)g.N, (uint64_t)g.K, (uint64_t)g.ldb, ka.bn))
        return cudaErrorInvalidValue;
    const uint32_t splits = (uint32_t)((g.K + g.kps - 1) / g.kps);
    const dim3 grid((g.M + kBM - 1) / kBM, (g.N + ka.bn - 1) / ka.bn, splits);
    if (grid.y > 65535u || grid.z > 65535u) return cudaErrorInvalidValue;
    if (g.epi == TC_EPI_WGRAD)  // long K, few CTAs: deeper copy pipeline
        tc_gemm_kernel<4><<<grid, kThreads, smem_bytes(4), s>>>(ta, tb, ka);
    else
        tc_gemm_kernel<2><<<grid, kThreads, smem_bytes(2), s>>>(ta, tb, ka);
    return cudaGetLastError();
}
