// mlp.cu -- surrogate MLP (simulation parameters -> daily log incidence) trained
// and evaluated on the GPU: BF16 operands, FP32 accumulation on the tensor cores.
//
// Layers: n_in -> H -> ... -> H (depth hidden layers, GELU in its tanh form,
// gelu.cuh) -> n_out (linear).
// Forward of layer l:  z_l = a_{l-1} W_l + b_l  (FP32 accumulate of BF16 products),
// a_l = bf16(gelu(z_l)) for hidden layers, the output z_L in FP32.
// Backward (MSE loss (1/(B n_out)) sum (y_hat - y)^2):
//   dz_L = 2 (y_hat - y) / (B n_out);  dW_l = a_{l-1}^T bf16(dz_l);  db_l = sum_rows dz_l;
//   dz_{l-1} = (bf16(dz_l) W_l^T) * gelu'(z_{l-1}).
// Adam keeps FP32 master weights and refreshes the BF16 copies after each step.
// The input layer's K is padded to a multiple of 16 with zero columns / rows.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <algorithm>
#include <vector>

#include "deabm.h"
#include "gelu.cuh"
#include "mlp_tc.h"

namespace mlpk {

// ------------------------------------------------------------------ tensor-core GEMM
// C[M x N] = A[M x K] * B[K x N] with A(i, r) = A[i*sAi + r*sAr], B(r, j) = B[r*sBr + j*sBj]
// (BF16), FP32 accumulate, fused epilogue.  Tile 128 x 64 x 32, 4 warps of 64 x 32,
// mma.sync m16n8k16 with ldmatrix fragments.
constexpr int BM = 128, BN = 64, BK = 32, PAD = 8;

enum Epi : int {
    EPI_HIDDEN = 0,   // z = acc + bias -> zf (FP32), a = bf16(gelu(z))
    EPI_OUTPUT = 1,   // y = acc + bias (FP32)
    EPI_DGRAD = 2,    // dz = acc * gelu'(zf) -> out (FP32) and bf16 copy
    EPI_WGRAD = 3,    // plain FP32 store
};

struct GemmArgs {
    const __nv_bfloat16 *A, *B;
    long sAi, sAr, sBr, sBj;
    int M, N, K;
    const float *bias;    // EPI_HIDDEN / EPI_OUTPUT
    const float *zin;     // EPI_DGRAD: pre-activation of the layer below [M x N]
    float *outf;          // FP32 output [M x ldo]
    __nv_bfloat16 *outb;  // BF16 output [M x ldo] (hidden, dgrad)
    int ldo;
    int epi;
};


__device__ __forceinline__ void ldmatrix_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float *d, const uint32_t *a, uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(128) gemm_bf16_kernel(const GemmArgs g)
{
    __shared__ __align__(16) __nv_bfloat16 sA[BM][BK + PAD];  // [i][r]
    __shared__ __align__(16) __nv_bfloat16 sB[BN][BK + PAD];  // [j][r]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;  // 2 x 2 warps, each 64 x 32
    const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
    // split-K (weight gradients): this CTA reduces K range [kb, ke) into its own partial
    const int kchunk = (g.K + (int)gridDim.z - 1) / (int)gridDim.z;
    const int kb = (int)blockIdx.z * kchunk, ke = min(g.K, kb + kchunk);
    float acc[4][4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0f;
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);
    for (int r0 = kb; r0 < ke; r0 += BK) {
        // A tile: walk the contiguous dimension with consecutive threads
        if (g.sAr == 1) {
            for (int q = tid; q < BM * BK; q += 128) {
                const int i = q / BK, r = q % BK, gi = i0 + i, gr = r0 + r;
                sA[i][r] = (gi < g.M && gr < ke) ? g.A[(long)gi * g.sAi + gr] : zero;
            }
        } else {
            for (int q = tid; q < BM * BK; q += 128) {
                const int r = q / BM, i = q % BM, gi = i0 + i, gr = r0 + r;
                sA[i][r] = (gi < g.M && gr < ke) ? g.A[(long)gi * g.sAi + (long)gr * g.sAr] : zero;
            }
        }
        if (g.sBj == 1) {
            for (int q = tid; q < BN * BK; q += 128) {
                const int r = q / BN, j = q % BN, gj = j0 + j, gr = r0 + r;
                sB[j][r] = (gj < g.N && gr < ke) ? g.B[(long)gr * g.sBr + gj] : zero;
            }
        } else {
            for (int q = tid; q < BN * BK; q += 128) {
                const int j = q / BK, r = q % BK, gj = j0 + j, gr = r0 + r;
                sB[j][r] = (gj < g.N && gr < ke) ? g.B[(long)gr * g.sBr + (long)gj * g.sBj] : zero;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[4][4];
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                const int row = wm * 64 + mt * 16 + (lane & 15), col = kk + (lane >> 4) * 8;
                ldmatrix_x4(af[mt][0], af[mt][1], af[mt][2], af[mt][3], &sA[row][col]);
            }
#pragma unroll
            for (int np = 0; np < 2; ++np) {  // pairs of 8-wide n tiles
                uint32_t b0, b1, b2, b3;
                // matrices: (n 0-7, k 0-7), (n 0-7, k 8-15), (n 8-15, k 0-7), (n 8-15, k 8-15)
                const int nrow = wn * 32 + np * 16 + (lane & 7) + ((lane >> 4) << 3);
                const int kcol = kk + ((lane >> 3) & 1) * 8;
                ldmatrix_x4(b0, b1, b2, b3, &sB[nrow][kcol]);
#pragma unroll
                for (int mt = 0; mt < 4; ++mt) {
                    mma_bf16(acc[mt][np * 2 + 0], af[mt], b0, b1);
                    mma_bf16(acc[mt][np * 2 + 1], af[mt], b2, b3);
                }
            }
        }
        __syncthreads();
    }
    // epilogue: thread owns rows (g, g+8) and columns (2t, 2t+1) of each 16 x 8 tile
    const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int i = i0 + wm * 64 + mt * 16 + gid + h * 8;
                    const int j = j0 + wn * 32 + nt * 8 + tig * 2 + e;
                    if (i >= g.M || j >= g.N) continue;
                    const float v = acc[mt][nt][h * 2 + e];
                    const long o = (long)i * g.ldo + j;
                    if (g.epi == EPI_HIDDEN) {
                        const float z = v + g.bias[j];
                        if (g.outf) g.outf[o] = z;
                        g.outb[o] = __float2bfloat16(gelu_act(z));
                    } else if (g.epi == EPI_OUTPUT) {
                        g.outf[o] = v + g.bias[j];
                    } else if (g.epi == EPI_DGRAD) {
                        const float d = v * gelu_act_grad(g.zin[o]);
                        g.outf[o] = d;
                        g.outb[o] = __float2bfloat16(d);
                    } else {
                        g.outf[o + (long)blockIdx.z * g.M * g.ldo] = v;
                    }
                }
}

// ------------------------------------------------------------------ small kernels
// out[q] = sum over splits of part[s][q] in split order (deterministic)
__global__ void splitk_reduce_kernel(const float *part, int splits, long n, float *out)
{
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
        float v = 0.0f;
        for (int z = 0; z < splits; ++z) v += part[(long)z * n + q];
        out[q] = v;
    }
}

__global__ void to_bf16_pad_kernel(const float *x, int rows, int cols, int ld, __nv_bfloat16 *out)
{
    const long n = (long)rows * ld;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
        const int r = (int)(q / ld), c = (int)(q % ld);
        out[q] = __float2bfloat16(c < cols ? x[(long)r * cols + c] : 0.0f);
    }
}

// dz_L = 2 (y_hat - y) / (B n_out), its bf16 copy, and the loss (block partials)
__global__ void mse_grad_kernel(const float *yhat, const float *y, long n, float scale, float *dz, __nv_bfloat16 *dzb,
                                double *loss_part)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
        const float d = yhat[q] - y[q];
        acc += (double)d * d;
        const float gq = 2.0f * d * scale;
        dz[q] = gq;
        dzb[q] = __float2bfloat16(gq);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// the loss from its partials: one block of 256 threads, each summing a strided
// share, then a fixed tree (deterministic)
__global__ void loss_reduce_kernel(const double *part, int nparts, float scale, float *loss)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int q = threadIdx.x; q < nparts; q += blockDim.x) s += part[q];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(red[0] * scale);
}

// db[j] = sum_i dz[i][j]: row chunks summed in parallel (partials [chunk][col]),
// then the chunks in order (deterministic)
constexpr int kColChunks = 64;
__global__ void colsum_partial_kernel(const float *dz, int rows, int cols, float *part)
{
    const int j = blockIdx.x * 32 + (threadIdx.x & 31), sub = threadIdx.x >> 5;  // 8 row lanes
    const int chunk = (rows + kColChunks - 1) / kColChunks, r0 = blockIdx.y * chunk, r1 = min(rows, r0 + chunk);
    __shared__ float red[8][32];
    float s = 0.0f;
    if (j < cols)
        for (int i = r0 + sub; i < r1; i += 8) s += dz[(long)i * cols + j];
    red[sub][threadIdx.x & 31] = s;
    __syncthreads();
    if (sub == 0 && j < cols) {
        float t = 0.0f;
        for (int q = 0; q < 8; ++q) t += red[q][threadIdx.x];
        part[(long)blockIdx.y * cols + j] = t;
    }
}

__global__ void colsum_final_kernel(const float *part, int cols, float *db)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float s = 0.0f;
    for (int c = 0; c < kColChunks; ++c) s += part[(long)c * cols + j];
    db[j] = s;
}

__global__ void adam_update_kernel(float *w, float *m, float *v, const float *g, long n, float lr, float b1, float b2,
                                   float eps, float c1, float c2, __nv_bfloat16 *wb, int rows, int cols, int ldb)
{
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
        const float gq = g[q];
        const float mq = b1 * m[q] + (1.0f - b1) * gq, vq = b2 * v[q] + (1.0f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        const float wq = w[q] - lr * (mq / c1) / (sqrtf(vq / c2) + eps);
        w[q] = wq;
        if (wb) {
            const int r = (int)(q / cols), c = (int)(q % cols);
            if (r < rows) wb[(long)r * ldb + c] = __float2bfloat16(wq);
        }
    }
}

__global__ void weights_to_bf16_kernel(const float *w, int rows, int cols, int rows_pad, __nv_bfloat16 *wb)
{
    const long n = (long)rows_pad * cols;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
        const int r = (int)(q / cols);
        wb[q] = __float2bfloat16(r < rows ? w[q] : 0.0f);
    }
}

// tensor-core training path: x -> a_0 (BF16 [rows x ld], zero-padded) and its
// transpose a_0^T [ld x ldt]
__global__ void to_bf16_pad_t_kernel(const float *x, int rows, int cols, int ld, __nv_bfloat16 *out,
                                     __nv_bfloat16 *outt, int ldt)
{
    const long n = (long)rows * ld;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
        const int r = (int)(q / ld), c = (int)(q % ld);
        const __nv_bfloat16 v = __float2bfloat16(c < cols ? x[(long)r * cols + c] : 0.0f);
        out[q] = v;
        outt[(long)c * ldt + r] = v;
    }
}

// BF16 weight copies of the tensor-core training path: W [fi x ldf] (the input
// gradients' operand, K = fan-out) and W^T [fo x ldt] (the forward operand,
// K = fan-in), zero in the padding
__global__ void weights_tc_kernel(const float *w, int fi, int fo, __nv_bfloat16 *wf, int ldf, __nv_bfloat16 *wt, int ldt)
{
    const long n = (long)fi * ldf;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
        const int r = (int)(q / ldf), c = (int)(q % ldf);
        wf[q] = __float2bfloat16(c < fo ? w[(long)r * fo + c] : 0.0f);
    }
    const long nt = (long)fo * ldt;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < nt; q += (long)gridDim.x * blockDim.x) {
        const int r = (int)(q / ldt), c = (int)(q % ldt);
        wt[q] = __float2bfloat16(c < fi ? w[(long)c * fo + r] : 0.0f);
    }
}

// After the tensor-core training GEMMs, one launch finishes every layer: the
// weight gradient from its split partials (summed in split order) and the bias
// gradient from the per-CTA column partials (a block per column, a fixed tree),
// the same sums as the per-layer reductions; with `adam`, the Adam step (Kingma
// and Ba, Algorithm 1) on each element right after its gradient, and the BF16
// copies both GEMM paths read written in place.
struct FinishLayer {
    const float *wpart;  // [splits][fi * fo]; splits == 0: gW already holds the gradient
    const float *bpart;  // [nparts][fo]
    float *gW, *gb, *W, *mW, *vW, *b, *mb, *vb;
    __nv_bfloat16 *Wb, *Wf, *WT;
    int splits, nparts, fi, fo, ldf, ldt;  // Wf [fi][ldf], WT [fo][ldt], Wb [kpad][fo]
};
struct FinishSet {
    int L, adam, wblocks;
    float lr, b1, b2, eps, c1, c2;
    long wstart[kMaxTcLayers + 1];  // prefix sums of fi * fo
    int bstart[kMaxTcLayers + 1];   // prefix sums of fo (one block per bias column)
    FinishLayer ly[kMaxTcLayers];
};
constexpr int kFinishThreads = 128;

__device__ __forceinline__ float adam_elem(float *w, float *m, float *v, float gq, const FinishSet &F)
{
    const float mq = F.b1 * *m + (1.0f - F.b1) * gq, vq = F.b2 * *v + (1.0f - F.b2) * gq * gq;
    *m = mq;
    *v = vq;
    const float wq = *w - F.lr * (mq / F.c1) / (sqrtf(vq / F.c2) + F.eps);
    *w = wq;
    return wq;
}

__global__ void __launch_bounds__(kFinishThreads) grad_finish_kernel(const FinishSet F)
{
    if ((int)blockIdx.x < F.wblocks) {
        const long total = F.wstart[F.L];
        for (long q = (long)blockIdx.x * kFinishThreads + threadIdx.x; q < total;
             q += (long)F.wblocks * kFinishThreads) {
            int l = 0;
            while (q >= F.wstart[l + 1]) ++l;
            const FinishLayer &Y = F.ly[l];
            const long n = F.wstart[l + 1] - F.wstart[l], i = q - F.wstart[l];
            float gq;
            if (Y.splits > 0) {
                gq = 0.0f;
                for (int z = 0; z < Y.splits; ++z) gq += Y.wpart[(long)z * n + i];
                Y.gW[i] = gq;
            } else {
                gq = Y.gW[i];
            }
            if (F.adam) {
                const float wq = adam_elem(Y.W + i, Y.mW + i, Y.vW + i, gq, F);
                const int r = (int)(i / Y.fo), c = (int)(i % Y.fo);
                const __nv_bfloat16 h = __float2bfloat16(wq);
                Y.Wb[(long)r * Y.fo + c] = h;
                Y.Wf[(long)r * Y.ldf + c] = h;
                Y.WT[(long)c * Y.ldt + r] = h;
            }
        }
        return;
    }
    const int col = (int)blockIdx.x - F.wblocks;
    int l = 0;
    while (col >= F.bstart[l + 1]) ++l;
    const FinishLayer &Y = F.ly[l];
    const int j = col - F.bstart[l];
    __shared__ float red[kFinishThreads];
    float s = 0.0f;
    for (int c = threadIdx.x; c < Y.nparts; c += kFinishThreads) s += Y.bpart[(long)c * Y.fo + j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kFinishThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        Y.gb[j] = red[0];
        if (F.adam) (void)adam_elem(Y.b + j, Y.mb + j, Y.vb + j, red[0], F);
    }
}

}  // namespace mlpk

using namespace mlpk;

// ------------------------------------------------------------------------------------ host side
struct deabm_mlp {
    cudaStream_t stream = nullptr;
    int n_in = 0, k_in = 0, H = 0, depth = 0, n_out = 0, L = 0, max_batch = 0;
    std::vector<void *> allocs;
    std::vector<int> fin, fout, kpad;  // per layer: fan-in, fan-out, padded fan-in
    std::vector<float *> W, b, gW, gb, mW, vW, mb, vb;   // FP32 master, grads, Adam moments
    std::vector<__nv_bfloat16 *> Wb;                      // BF16 copies [kpad x fout]
    std::vector<__nv_bfloat16 *> act;                     // a_l, l = 0..L-1 (a_0 = input) [B x ld]
    std::vector<float *> z;                               // pre-activations of hidden layers [B x H]
    float *yhat = nullptr, *dz = nullptr, *dz2 = nullptr, *loss = nullptr, *wpart = nullptr;
    int max_splits = 1;
    __nv_bfloat16 *dzb = nullptr, *dzb2 = nullptr;
    double *loss_part = nullptr;
    int step = 0;
    // fused tcgen05 forward (inference): eligible shapes, K-major BF16 weight copies
    bool tc_ok = false, tc_on = true, wt_dirty = true;
    std::vector<__nv_bfloat16 *> Wt;
    std::vector<int> tcK, tcN;
    int *tc_err = nullptr;
    // tensor-core training path: transposed activations a_l^T [kpad_l x bpad],
    // BF16 output gradients row-major [B x ld8] and transposed [width x bpad],
    // BF16 weights W_l [fi x ld8(fo)] and W_l^T [fo x ld8(fi)]
    bool tr_ok = false, tr_dirty = true;
    int bpad = 0, ldg = 0;
    std::vector<__nv_bfloat16 *> actT, Wf, WT;
    __nv_bfloat16 *gb16[2] = {nullptr, nullptr}, *gT[2] = {nullptr, nullptr};
    uint32_t polls = 1u << 26;
    // per layer, kept until the step's one finishing launch: weight-gradient split
    // partials [max_splits][fi x fo] and bias-gradient column partials [parts][fo]
    std::vector<float *> wpartL, bpartL;
    std::vector<int> splitsL;
};

static int ld8(int v) { return (v + 7) / 8 * 8; }

static thread_local std::string g_mlp_err;

static int mlp_fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_mlp_err = buf;
    return code;
}

#define MCU(call)                                                                                                   \
    do {                                                                                                            \
        cudaError_t e_ = (call);                                                                                    \
        if (e_ != cudaSuccess)                                                                                      \
            return mlp_fail(e_ == cudaErrorMemoryAllocation ? DEABM_ENOMEM : DEABM_ECUDA, "%s: %s (%s:%d)", #call, \
                            cudaGetErrorString(e_), __FILE__, __LINE__);                                            \
    } while (0)

template <class T>
static int m_alloc(deabm_mlp *m, T **out, size_t count)
{
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, (count ? count : 1) * sizeof(T));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return mlp_fail(DEABM_ENOMEM, "cudaMalloc failed (%zu bytes)", count * sizeof(T));
    }
    m->allocs.push_back(p);
    *out = (T *)p;
    return DEABM_OK;
}

static int gemm(cudaStream_t s, const GemmArgs &g, int splits = 1)
{
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, splits);
    if (grid.y > 65535) return mlp_fail(DEABM_EINVAL, "GEMM with M = %d is too tall", g.M);
    gemm_bf16_kernel<<<grid, 128, 0, s>>>(g);
    MCU(cudaGetLastError());
    return DEABM_OK;
}

extern "C" void deabm_mlp_destroy(deabm_mlp *m)
{
    if (!m) return;
    if (!m->allocs.empty()) (void)cudaStreamSynchronize(m->stream);
    for (void *p : m->allocs) (void)cudaFree(p);
    delete m;
}

extern "C" int deabm_mlp_create(uint32_t n_in, uint32_t hidden, uint32_t depth, uint32_t n_out, uint32_t max_batch,
                                void *stream, deabm_mlp **out)
{
    if (!out) return mlp_fail(DEABM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_in == 0 || n_in > 4096 || hidden == 0 || hidden > 4096 || depth == 0 || depth > 16 || n_out == 0 ||
        n_out > 4096 || max_batch == 0 || max_batch > (1u << 22))
        return mlp_fail(DEABM_EINVAL, "sizes out of range");
    if (hidden % 8 || n_out % 2) return mlp_fail(DEABM_EINVAL, "hidden must be a multiple of 8 and n_out even");
    deabm_mlp *m = new (std::nothrow) deabm_mlp();
    if (!m) return mlp_fail(DEABM_ENOMEM, "host allocation failed");
    int rc = [&]() -> int {
        m->stream = (cudaStream_t)stream;
        m->n_in = (int)n_in;
        m->k_in = (int)((n_in + 15) / 16 * 16);
        m->H = (int)hidden;
        m->depth = (int)depth;
        m->n_out = (int)n_out;
        m->L = (int)depth + 1;
        m->max_batch = (int)max_batch;
        int r;
        for (int l = 0; l < m->L; ++l) {
            const int fi = l == 0 ? m->n_in : m->H, fo = l == m->L - 1 ? m->n_out : m->H;
            const int kp = l == 0 ? m->k_in : m->H;
            m->fin.push_back(fi);
            m->fout.push_back(fo);
            m->kpad.push_back(kp);
            float *W, *b, *gW, *gb, *mW, *vW, *mb, *vb;
            __nv_bfloat16 *Wb;
            if ((r = m_alloc(m, &W, (size_t)fi * fo))) return r;
            if ((r = m_alloc(m, &b, fo))) return r;
            if ((r = m_alloc(m, &gW, (size_t)fi * fo))) return r;
            if ((r = m_alloc(m, &gb, fo))) return r;
            if ((r = m_alloc(m, &mW, (size_t)fi * fo))) return r;
            if ((r = m_alloc(m, &vW, (size_t)fi * fo))) return r;
            if ((r = m_alloc(m, &mb, fo))) return r;
            if ((r = m_alloc(m, &vb, fo))) return r;
            if ((r = m_alloc(m, &Wb, (size_t)kp * fo))) return r;
            MCU(cudaMemsetAsync(W, 0, 4ull * fi * fo, m->stream));
            MCU(cudaMemsetAsync(b, 0, 4ull * fo, m->stream));
            MCU(cudaMemsetAsync(Wb, 0, 2ull * kp * fo, m->stream));
            m->W.push_back(W); m->b.push_back(b); m->gW.push_back(gW); m->gb.push_back(gb);
            m->mW.push_back(mW); m->vW.push_back(vW); m->mb.push_back(mb); m->vb.push_back(vb); m->Wb.push_back(Wb);
        }
        const size_t B = max_batch;
        for (int l = 0; l < m->L; ++l) {  // a_0 .. a_{L-1}: inputs of each layer
            __nv_bfloat16 *a;
            if ((r = m_alloc(m, &a, B * m->kpad[l]))) return r;
            m->act.push_back(a);
        }
        for (int l = 0; l < m->L - 1; ++l) {
            float *zz;
            if ((r = m_alloc(m, &zz, B * m->H))) return r;
            m->z.push_back(zz);
        }
        const int wmax = m->H > m->n_out ? m->H : m->n_out;
        if ((r = m_alloc(m, &m->yhat, B * m->n_out))) return r;
        if ((r = m_alloc(m, &m->dz, B * wmax))) return r;
        if ((r = m_alloc(m, &m->dz2, B * wmax))) return r;
        if ((r = m_alloc(m, &m->dzb, B * wmax))) return r;
        if ((r = m_alloc(m, &m->dzb2, B * wmax))) return r;
        if ((r = m_alloc(m, &m->loss, 1))) return r;
        // split-K partials of the largest weight gradient: enough splits to fill the GPU
        m->max_splits = (int)std::min<uint32_t>(64u, std::max<uint32_t>(1u, max_batch / 256u));
        size_t wmax_params = 0;
        for (int l = 0; l < m->L; ++l) wmax_params = std::max(wmax_params, (size_t)m->fin[l] * m->fout[l]);
        // also holds the bias-gradient partials [kColChunks][fan_out]
        const size_t wp = std::max(wmax_params * m->max_splits, (size_t)kColChunks * (size_t)std::max(m->H, m->n_out));
        if ((r = m_alloc(m, &m->wpart, wp))) return r;
        if ((r = m_alloc(m, &m->loss_part, std::max<size_t>(1024, (B + 127) / 128)))) return r;
        m->tc_ok = m->n_in <= 64 && m->H % 64 == 0 && m->H <= 256 && m->n_out <= 256 && m->L <= kMaxTcLayers;
        if (m->tc_ok) {
            size_t total = 0;
            for (int l = 0; l < m->L; ++l) {
                const int kp = l == 0 ? 64 : m->H;
                const int np = l < m->L - 1 ? m->H : (m->n_out + 63) / 64 * 64;
                m->tcK.push_back(kp);
                m->tcN.push_back(np);
                total += (size_t)kp * np;
            }
            __nv_bfloat16 *img;
            if ((r = m_alloc(m, &img, total))) return r;
            for (int l = 0, off = 0; l < m->L; ++l) {
                m->Wt.push_back(img + off);  // this layer's chunk images
                off += m->tcK[l] * m->tcN[l];
            }
            if ((r = m_alloc(m, &m->tc_err, 1))) return r;
            MCU(cudaMemsetAsync(m->tc_err, 0, sizeof(int), m->stream));
            // the training path on the same tensor cores
            m->tr_ok = true;
            m->bpad = ld8((int)max_batch);
            m->ldg = ld8(std::max(m->H, m->n_out));
            for (int l = 0; l < m->L; ++l) {
                __nv_bfloat16 *at, *wf, *wt;
                if ((r = m_alloc(m, &at, (size_t)m->kpad[l] * m->bpad))) return r;
                if ((r = m_alloc(m, &wf, (size_t)m->fin[l] * ld8(m->fout[l])))) return r;
                if ((r = m_alloc(m, &wt, (size_t)m->fout[l] * ld8(m->kpad[l])))) return r;
                m->actT.push_back(at);
                m->Wf.push_back(wf);
                m->WT.push_back(wt);
            }
            for (int q = 0; q < 2; ++q) {
                if ((r = m_alloc(m, &m->gb16[q], B * m->ldg))) return r;
                if ((r = m_alloc(m, &m->gT[q], (size_t)m->ldg * m->bpad))) return r;
            }
            for (int l = 0; l < m->L; ++l) {
                float *wp, *bp;
                if ((r = m_alloc(m, &wp, (size_t)m->max_splits * m->fin[l] * m->fout[l]))) return r;
                if ((r = m_alloc(m, &bp, ((B + 127) / 128) * (size_t)m->fout[l]))) return r;
                m->wpartL.push_back(wp);
                m->bpartL.push_back(bp);
            }
            m->splitsL.assign(m->L, 0);
        }
        MCU(cudaStreamSynchronize(m->stream));
        return DEABM_OK;
    }();
    if (rc != DEABM_OK) {
        deabm_mlp_destroy(m);
        return rc;
    }
    *out = m;
    return DEABM_OK;
}

size_t mlp_param_count(const deabm_mlp *m)
{
    size_t n = 0;
    for (int l = 0; l < m->L; ++l) n += (size_t)m->fin[l] * m->fout[l] + m->fout[l];
    return n;
}

extern "C" int deabm_mlp_param_count(const deabm_mlp *m, uint64_t *count)
{
    if (!m || !count) return mlp_fail(DEABM_EINVAL, "NULL argument");
    *count = mlp_param_count(m);
    return DEABM_OK;
}

extern "C" int deabm_mlp_set_params(deabm_mlp *m, const float *params)
{
    if (!m || !params) return mlp_fail(DEABM_EINVAL, "NULL argument");
    size_t off = 0;
    for (int l = 0; l < m->L; ++l) {
        const size_t nw = (size_t)m->fin[l] * m->fout[l];
        MCU(cudaMemcpyAsync(m->W[l], params + off, 4 * nw, cudaMemcpyHostToDevice, m->stream));
        off += nw;
        MCU(cudaMemcpyAsync(m->b[l], params + off, 4ull * m->fout[l], cudaMemcpyHostToDevice, m->stream));
        off += m->fout[l];
        weights_to_bf16_kernel<<<256, 256, 0, m->stream>>>(m->W[l], m->fin[l], m->fout[l], m->kpad[l], m->Wb[l]);
        MCU(cudaMemsetAsync(m->mW[l], 0, 4 * nw, m->stream));
        MCU(cudaMemsetAsync(m->vW[l], 0, 4 * nw, m->stream));
        MCU(cudaMemsetAsync(m->mb[l], 0, 4ull * m->fout[l], m->stream));
        MCU(cudaMemsetAsync(m->vb[l], 0, 4ull * m->fout[l], m->stream));
    }
    m->step = 0;
    m->wt_dirty = true;
    m->tr_dirty = true;
    MCU(cudaGetLastError());
    MCU(cudaStreamSynchronize(m->stream));
    return DEABM_OK;
}

extern "C" int deabm_mlp_get_params(deabm_mlp *m, float *params, float *grads)
{
    if (!m || (!params && !grads)) return mlp_fail(DEABM_EINVAL, "NULL argument");
    size_t off = 0;
    for (int l = 0; l < m->L; ++l) {
        const size_t nw = (size_t)m->fin[l] * m->fout[l];
        if (params) MCU(cudaMemcpyAsync(params + off, m->W[l], 4 * nw, cudaMemcpyDeviceToHost, m->stream));
        if (grads) MCU(cudaMemcpyAsync(grads + off, m->gW[l], 4 * nw, cudaMemcpyDeviceToHost, m->stream));
        off += nw;
        if (params) MCU(cudaMemcpyAsync(params + off, m->b[l], 4ull * m->fout[l], cudaMemcpyDeviceToHost, m->stream));
        if (grads) MCU(cudaMemcpyAsync(grads + off, m->gb[l], 4ull * m->fout[l], cudaMemcpyDeviceToHost, m->stream));
        off += m->fout[l];
    }
    MCU(cudaStreamSynchronize(m->stream));
    return DEABM_OK;
}

// forward over `batch` rows of x (device FP32 [batch x n_in]) into yhat (device FP32);
// `keep` stores the pre-activations for a backward pass
static int mlp_forward_dev(deabm_mlp *m, const float *x, int batch, float *yhat, bool keep)
{
    cudaStream_t s = m->stream;
    to_bf16_pad_kernel<<<512, 256, 0, s>>>(x, batch, m->n_in, m->k_in, m->act[0]);
    MCU(cudaGetLastError());
    int r;
    for (int l = 0; l < m->L; ++l) {
        GemmArgs g{};
        g.A = m->act[l];
        g.sAi = m->kpad[l];
        g.sAr = 1;
        g.B = m->Wb[l];
        g.sBr = m->fout[l];
        g.sBj = 1;
        g.M = batch;
        g.N = m->fout[l];
        g.K = m->kpad[l];
        g.bias = m->b[l];
        if (l < m->L - 1) {
            g.epi = EPI_HIDDEN;
            g.outf = keep ? m->z[l] : nullptr;
            g.outb = m->act[l + 1];
            g.ldo = m->H;
        } else {
            g.epi = EPI_OUTPUT;
            g.outf = yhat;
            g.ldo = m->n_out;
        }
        if ((r = gemm(s, g))) return r;
    }
    return DEABM_OK;
}

static int mlp_backward_dev(deabm_mlp *m, const float *y, int batch, float *loss_host)
{
    cudaStream_t s = m->stream;
    const long n = (long)batch * m->n_out;
    const int nparts = 256;
    mse_grad_kernel<<<nparts, 256, 0, s>>>(m->yhat, y, n, 1.0f / (float)n, m->dz, m->dzb, m->loss_part);
    loss_reduce_kernel<<<1, 256, 0, s>>>(m->loss_part, nparts, 1.0f / (float)n, m->loss);
    MCU(cudaGetLastError());
    float *dz = m->dz, *dzo = m->dz2;
    __nv_bfloat16 *dzb = m->dzb, *dzbo = m->dzb2;
    int r;
    for (int l = m->L - 1; l >= 0; --l) {
        const int fo = m->fout[l], fi = m->fin[l];
        // dW_l = a_{l-1}^T dz_l : [fi x fo], reduction over the batch
        GemmArgs gw{};
        gw.A = m->act[l];
        gw.sAi = 1;
        gw.sAr = m->kpad[l];
        gw.B = dzb;
        gw.sBr = fo;
        gw.sBj = 1;
        gw.M = fi;
        gw.N = fo;
        gw.K = batch;
        gw.ldo = fo;
        gw.epi = EPI_WGRAD;
        const int splits = std::max(1, std::min(m->max_splits, batch / 512));
        gw.outf = splits > 1 ? m->wpart : m->gW[l];
        if ((r = gemm(s, gw, splits))) return r;
        if (splits > 1) {
            splitk_reduce_kernel<<<256, 256, 0, s>>>(m->wpart, splits, (long)fi * fo, m->gW[l]);
            MCU(cudaGetLastError());
        }
        colsum_partial_kernel<<<dim3((fo + 31) / 32, kColChunks), 256, 0, s>>>(dz, batch, fo, m->wpart);
        colsum_final_kernel<<<(fo + 127) / 128, 128, 0, s>>>(m->wpart, fo, m->gb[l]);
        MCU(cudaGetLastError());
        if (l > 0) {
            // dz_{l-1} = (dz_l W_l^T) * gelu'(z_{l-1})
            GemmArgs gd{};
            gd.A = dzb;
            gd.sAi = fo;
            gd.sAr = 1;
            gd.B = m->Wb[l];
            gd.sBr = 1;
            gd.sBj = fo;
            gd.M = batch;
            gd.N = m->H;
            gd.K = fo;
            gd.zin = m->z[l - 1];
            gd.outf = dzo;
            gd.outb = dzbo;
            gd.ldo = m->H;
            gd.epi = EPI_DGRAD;
            if ((r = gemm(s, gd))) return r;
            float *tf = dz;
            dz = dzo;
            dzo = tf;
            __nv_bfloat16 *tb = dzb;
            dzb = dzbo;
            dzbo = tb;
        }
    }
    if (loss_host) {
        MCU(cudaMemcpyAsync(loss_host, m->loss, 4, cudaMemcpyDeviceToHost, s));
        MCU(cudaStreamSynchronize(s));
    }
    return DEABM_OK;
}

extern "C" int deabm_mlp_forward(deabm_mlp *m, const float *x, uint32_t batch, float *y)
{
    if (!m || !x || !y) return mlp_fail(DEABM_EINVAL, "NULL argument");
    if (batch == 0) return DEABM_OK;
    if ((int)batch > m->max_batch) return mlp_fail(DEABM_EINVAL, "batch %u > max_batch %d", batch, m->max_batch);
    if (!(m->tc_ok && m->tc_on)) return mlp_forward_dev(m, x, (int)batch, y, false);
    if (m->wt_dirty) {
        for (int l = 0; l < m->L; ++l)
            MCU(mlptc_prepare_weights(m->W[l], m->fin[l], m->fout[l], m->tcK[l], m->tcN[l], m->Wt[l], m->stream));
        m->wt_dirty = false;
    }
    FusedArgs g{};
    g.x = x;
    g.y = y;
    g.M = (int)batch;
    g.n_in = m->n_in;
    g.n_out = m->n_out;
    g.L = m->L;
    g.wimg = m->Wt[0];
    for (int l = 0; l < m->L; ++l) {
        g.bias[l] = m->b[l];
        g.K[l] = m->tcK[l];
        g.N[l] = m->tcN[l];
    }
    g.err = m->tc_err;
    g.polls = m->polls;
    MCU(mlptc_forward(g, m->stream));
    return DEABM_OK;
}

extern "C" int deabm_mlp_use_tcgen05(deabm_mlp *m, int enable, int *available)
{
    if (!m) return mlp_fail(DEABM_EINVAL, "NULL argument");
    m->tc_on = enable != 0;
    if (available) *available = m->tc_ok ? 1 : 0;
    return DEABM_OK;
}

// forward (keeping z_l, a_l and a_l^T) and backward of one batch on the tcgen05
// GEMMs (mlp_tc_gemm.cu); same quantities and rounding points as the mma.sync path
static int mlp_grad_tc(deabm_mlp *m, const float *x, const float *y, int batch, float *loss_host, bool adam = false,
                       float lr = 0.0f)
{
    cudaStream_t s = m->stream;
    if (m->tr_dirty) {
        for (int l = 0; l < m->L; ++l)
            weights_tc_kernel<<<256, 256, 0, s>>>(m->W[l], m->fin[l], m->fout[l], m->Wf[l], ld8(m->fout[l]), m->WT[l],
                                                   ld8(m->kpad[l]));
        MCU(cudaGetLastError());
        m->tr_dirty = false;
    }
    to_bf16_pad_t_kernel<<<512, 256, 0, s>>>(x, batch, m->n_in, m->k_in, m->act[0], m->actT[0], m->bpad);
    MCU(cudaGetLastError());
    for (int l = 0; l < m->L; ++l) {
        TcGemm g{};
        g.A = m->act[l];
        g.lda = m->kpad[l];
        g.B = m->WT[l];
        g.ldb = ld8(m->kpad[l]);
        g.M = batch;
        g.N = m->fout[l];
        g.K = m->kpad[l];
        g.kps = (g.K + 63) / 64 * 64;
        g.bias = m->b[l];
        g.polls = m->polls;
        g.err = m->tc_err;
        if (l < m->L - 1) {
            g.epi = TC_EPI_HIDDEN;
            g.outf = m->z[l];
            g.ldf = m->H;
            g.outb = m->act[l + 1];
            g.ldo = m->kpad[l + 1];
            g.outt = m->actT[l + 1];
            g.ldt = m->bpad;
        } else {
            // the output layer's epilogue is the loss gradient itself: dz_L, its BF16
            // copies and the loss partials (y_hat is not stored)
            g.epi = TC_EPI_MSE;
            g.y = y;
            g.scale = 1.0f / (float)((long)batch * m->n_out);
            g.outf = nullptr;  // dz_L stays in BF16; its column sums (the bias gradient) come as partials
            g.ldf = m->n_out;
            g.bpart = m->bpartL[m->L - 1];
            g.outb = m->gb16[0];
            g.ldo = m->ldg;
            g.outt = m->gT[0];
            g.ldt = m->bpad;
            g.loss_part = m->loss_part;
        }
        MCU(mlptc_gemm(g, s));
    }
    const long n = (long)batch * m->n_out;
    const int nparts = (batch + 127) / 128;
    int cur = 0;
    loss_reduce_kernel<<<1, 256, 0, s>>>(m->loss_part, nparts, 1.0f / (float)n, m->loss);
    MCU(cudaGetLastError());
    for (int l = m->L - 1; l >= 0; --l) {
        const int fo = m->fout[l], fi = m->fin[l];
        // dW_l = a_l^T dz_l, split over the batch, partials summed in split order
        TcGemm gw{};
        gw.A = m->actT[l];
        gw.lda = m->bpad;
        gw.B = m->gT[cur];
        gw.ldb = m->bpad;
        gw.M = fi;
        gw.N = fo;
        gw.K = batch;
        const int tiles = ((fi + 127) / 128) * ((fo + 255) / 256);
        int splits = std::max(1, std::min(m->max_splits, 2 * 152 / tiles));
        splits = std::min(splits, (batch + 63) / 64);
        gw.kps = ((batch + splits - 1) / splits + 63) / 64 * 64;
        splits = (batch + gw.kps - 1) / gw.kps;
        gw.epi = TC_EPI_WGRAD;
        gw.outf = splits > 1 ? m->wpartL[l] : m->gW[l];
        gw.ldf = fo;
        gw.polls = m->polls;
        gw.err = m->tc_err;
        MCU(mlptc_gemm(gw, s));
        m->splitsL[l] = splits > 1 ? splits : 0;  // summed, with db_l, in the finishing launch
        if (l > 0) {
            // dz_{l-1} = (dz_l W_l^T) * gelu'(z_{l-1})
            TcGemm gd{};
            gd.A = m->gb16[cur];
            gd.lda = m->ldg;
            gd.B = m->Wf[l];
            gd.ldb = ld8(fo);
            gd.M = batch;
            gd.N = m->H;
            gd.K = fo;
            gd.kps = (fo + 63) / 64 * 64;
            gd.epi = TC_EPI_DGRAD;
            gd.zin = m->z[l - 1];
            gd.ldz = m->H;
            gd.outf = nullptr;
            gd.ldf = m->H;
            gd.bpart = m->bpartL[l - 1];
            gd.outb = m->gb16[cur ^ 1];
            gd.ldo = m->ldg;
            gd.outt = m->gT[cur ^ 1];
            gd.ldt = m->bpad;
            gd.polls = m->polls;
            gd.err = m->tc_err;
            MCU(mlptc_gemm(gd, s));
            cur ^= 1;
        }
    }
    FinishSet F{};
    F.L = m->L;
    F.adam = adam ? 1 : 0;
    F.wblocks = 2 * 152;
    if (adam) {
        m->step += 1;
        F.lr = lr;
        F.b1 = 0.9f;
        F.b2 = 0.999f;
        F.eps = 1e-8f;
        F.c1 = 1.0f - powf(F.b1, (float)m->step);
        F.c2 = 1.0f - powf(F.b2, (float)m->step);
    }
    F.wstart[0] = 0;
    F.bstart[0] = 0;
    for (int l = 0; l < m->L; ++l) {
        FinishLayer &Y = F.ly[l];
        Y.wpart = m->wpartL[l];
        Y.splits = m->splitsL[l];
        Y.bpart = m->bpartL[l];
        Y.nparts = nparts;
        Y.gW = m->gW[l];
        Y.gb = m->gb[l];
        Y.W = m->W[l];
        Y.mW = m->mW[l];
        Y.vW = m->vW[l];
        Y.b = m->b[l];
        Y.mb = m->mb[l];
        Y.vb = m->vb[l];
        Y.Wb = m->Wb[l];
        Y.Wf = m->Wf[l];
        Y.WT = m->WT[l];
        Y.fi = m->fin[l];
        Y.fo = m->fout[l];
        Y.ldf = ld8(m->fout[l]);
        Y.ldt = ld8(m->kpad[l]);
        F.wstart[l + 1] = F.wstart[l] + (long)m->fin[l] * m->fout[l];
        F.bstart[l + 1] = F.bstart[l] + m->fout[l];
    }
    grad_finish_kernel<<<F.wblocks + F.bstart[m->L], kFinishThreads, 0, s>>>(F);
    MCU(cudaGetLastError());
    if (adam) {  // the BF16 copies are current; the fused forward's weight images are not
        m->wt_dirty = true;
        m->tr_dirty = false;
    }
    if (loss_host) {
        MCU(cudaMemcpyAsync(loss_host, m->loss, 4, cudaMemcpyDeviceToHost, s));
        MCU(cudaStreamSynchronize(s));
    }
    return DEABM_OK;
}

extern "C" int deabm_mlp_grad(deabm_mlp *m, const float *x, const float *y, uint32_t batch, float *loss)
{
    if (!m || !x || !y) return mlp_fail(DEABM_EINVAL, "NULL argument");
    if (batch == 0 || (int)batch > m->max_batch) return mlp_fail(DEABM_EINVAL, "batch must be in 1..max_batch");
    if (m->tr_ok && m->tc_on) return mlp_grad_tc(m, x, y, (int)batch, loss);
    int r;
    if ((r = mlp_forward_dev(m, x, (int)batch, m->yhat, true))) return r;
    return mlp_backward_dev(m, y, (int)batch, loss);
}

// one Adam step (Kingma and Ba, Algorithm 1) on the FP32 master weights from the
// gradients in gW / gb; refreshes the BF16 copies
static int mlp_adam(deabm_mlp *m, float lr)
{
    m->step += 1;
    m->wt_dirty = true;
    m->tr_dirty = true;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)m->step), c2 = 1.0f - powf(b2, (float)m->step);
    for (int l = 0; l < m->L; ++l) {
        const long nw = (long)m->fin[l] * m->fout[l];
        adam_update_kernel<<<256, 256, 0, m->stream>>>(m->W[l], m->mW[l], m->vW[l], m->gW[l], nw, lr, b1, b2, 1e-8f, c1,
                                                       c2, m->Wb[l], m->fin[l], m->fout[l], m->fout[l]);
        adam_update_kernel<<<4, 256, 0, m->stream>>>(m->b[l], m->mb[l], m->vb[l], m->gb[l], m->fout[l], lr, b1, b2,
                                                     1e-8f, c1, c2, nullptr, 0, 0, 0);
    }
    MCU(cudaGetLastError());
    return DEABM_OK;
}

extern "C" int deabm_mlp_train_step(deabm_mlp *m, const float *x, const float *y, uint32_t batch, float lr, float *loss)
{
    int r;
    if (m && x && y && batch > 0 && (int)batch <= m->max_batch && m->tr_ok && m->tc_on) {
        // tensor-core path: the gradients' reductions and the Adam step in one launch
        if ((r = mlp_grad_tc(m, x, y, (int)batch, nullptr, true, lr))) return r;
    } else {
        if ((r = deabm_mlp_grad(m, x, y, batch, nullptr))) return r;
        if ((r = mlp_adam(m, lr))) return r;
    }
    if (loss) {
        MCU(cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToHost, m->stream));
        MCU(cudaStreamSynchronize(m->stream));
    }
    return DEABM_OK;
}

extern "C" int deabm_mlp_apply_grads(deabm_mlp *m, const float *grads, uint32_t on_device, float lr)
{
    if (!m || !grads) return mlp_fail(DEABM_EINVAL, "NULL argument");
    if (!(lr > 0.0f) || !std::isfinite(lr)) return mlp_fail(DEABM_EINVAL, "lr must be finite and > 0");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    size_t off = 0;
    for (int l = 0; l < m->L; ++l) {
        const size_t nw = (size_t)m->fin[l] * m->fout[l];
        MCU(cudaMemcpyAsync(m->gW[l], grads + off, 4 * nw, kind, m->stream));
        off += nw;
        MCU(cudaMemcpyAsync(m->gb[l], grads + off, 4ull * m->fout[l], kind, m->stream));
        off += m->fout[l];
    }
    int r;
    if ((r = mlp_adam(m, lr))) return r;
    if (!on_device) MCU(cudaStreamSynchronize(m->stream));  // the host buffer may be reused on return
    return DEABM_OK;
}

extern "C" int deabm_mlp_set_wait_limit(deabm_mlp *m, uint32_t polls)
{
    if (!m) return mlp_fail(DEABM_EINVAL, "NULL argument");
    m->polls = polls ? polls : (1u << 26);
    return DEABM_OK;
}

extern "C" int deabm_mlp_sync(deabm_mlp *m)
{
    if (!m) return mlp_fail(DEABM_EINVAL, "NULL argument");
    MCU(cudaStreamSynchronize(m->stream));
    if (m->tc_err) {
        int err = 0;
        MCU(cudaMemcpy(&err, m->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (err) {
            MCU(cudaMemset(m->tc_err, 0, sizeof(int)));
            return mlp_fail(DEABM_ETIMEOUT, "a bounded wait of the tensor-core forward gave up");
        }
    }
    return DEABM_OK;
}

extern "C" const char *deabm_mlp_last_error(void) { return g_mlp_err.c_str(); }
