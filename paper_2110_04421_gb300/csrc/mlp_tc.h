// mlp_tc.h -- host interface of the fused tcgen05 forward pass of the surrogate MLP (internal).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

constexpr int kMaxKChunks = 4;  // hidden width <= 256 (64-column chunks)
constexpr int kMaxTcLayers = 8;

struct FusedArgs {
    const float *x;  // [M x n_in] FP32
    float *y;        // [M x n_out] FP32
    int M, n_in, n_out, L;
    const void *wimg;     // all layers' weight chunk images, in order (layer, chunk)
    const float *bias[kMaxTcLayers];
    int K[kMaxTcLayers];  // 64 for the input layer, the hidden width after
    int N[kMaxTcLayers];  // the hidden width, and n_out rounded up to 64 for the last layer
    int *err;             // set to 1 when a bounded wait gave up
    uint32_t polls;       // tries of each bounded wait before the kernel gives up
};

// swizzled weight chunk images of one layer (n_pad * k_pad BF16 at img)
cudaError_t mlptc_prepare_weights(const float *W, int fin, int fout, int k_pad, int n_pad, __nv_bfloat16 *img,
                                  cudaStream_t s);
cudaError_t mlptc_forward(const FusedArgs &g, cudaStream_t s);

// ---- training GEMMs on the tcgen05 tensor cores (mlp_tc_gemm.cu)
// C[M x N] = A[M x K] . B[N x K]^T with A and B BF16, K contiguous in memory (row
// strides lda / ldb elements, multiples of 8), FP32 accumulate in TMEM, and one of
// the MLP's epilogues.  Operands are read by TMA in 128-row (A) and up to 256-row
// (B) tiles of 64 K-columns; entries past M, N or K read as zero.
enum TcEpi : int {
    TC_EPI_HIDDEN = 0,  // z = acc + bias -> outf [M x ldf]; a = bf16(gelu(z)) -> outb [M x ldo] and outt [N x ldt]
    TC_EPI_OUTPUT = 1,  // y = acc + bias -> outf [M x ldf]
    TC_EPI_DGRAD = 2,   // d = acc * gelu'(zin) -> outf (FP32), outb (BF16) and outt (BF16, transposed)
    TC_EPI_WGRAD = 3,   // acc -> outf + split * M * ldf (split-K partials over blockIdx.z)
    TC_EPI_MSE = 4,     // y_hat = acc + bias; d = 2 (y_hat - y) scale -> outf (FP32), outb, outt;
                        // sum of (y_hat - y)^2 over the CTA's rows -> loss_part[blockIdx.x] (FP64)
};

struct TcGemm {
    const void *A, *B;
    int M, N, K;
    int lda, ldb;            // row strides of A [M x K] and B [N x K], elements
    int kps;                 // K columns per split (multiple of 64); splits = ceil(K / kps)
    int epi;
    const float *bias;       // [N]
    const float *zin;        // DGRAD: pre-activation [M x ldz]
    int ldz;
    float *outf;
    int ldf;
    __nv_bfloat16 *outb;
    int ldo;
    __nv_bfloat16 *outt;     // transposed copy [N x ldt]
    int ldt;
    uint32_t polls;          // tries of each bounded wait before the kernel gives up
    int *err;                // set to 1 when a bounded wait gave up
    const float *y;          // MSE: targets [M x N] (row stride N)
    float scale;             // MSE: 1 / (M N)
    double *loss_part;       // MSE: one partial per CTA row block (grid.x entries)
    float *bpart;            // DGRAD, MSE: if set, the column sums of the CTA's rows of d
                             // [grid.x x N] (the bias gradient's partials); outf may then be null
};

// one launch (asynchronous); cudaErrorInvalidValue for shapes it does not take
cudaError_t mlptc_gemm(const TcGemm &g, cudaStream_t s);
