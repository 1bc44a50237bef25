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
};

// swizzled weight chunk images of one layer (n_pad * k_pad BF16 at img)
cudaError_t mlptc_prepare_weights(const float *W, int fin, int fout, int k_pad, int n_pad, __nv_bfloat16 *img,
                                  cudaStream_t s);
cudaError_t mlptc_forward(const FusedArgs &g, cudaStream_t s);
