// gelu.cuh -- the surrogate MLP's activation, GELU in its tanh form (Hendrycks
// and Gimpel, 2016):
//     gelu(z) = z/2 (1 + tanh(u)),  u = sqrt(2/pi) (z + 0.044715 z^3),
//     gelu'(z) = (1 + tanh(u))/2 + z/2 (1 - tanh(u)^2) sqrt(2/pi) (1 + 3 * 0.044715 z^2),
// with one hardware tanh per element (tanh.approx.f32, relative error near
// 2^-11, below the BF16 rounding the hidden activations get).  Shared by the
// fused forward, the tcgen05 training GEMMs and the mma.sync path.
#pragma once

constexpr float kGeluC1 = 0.7978845608028654f;   // sqrt(2/pi)
constexpr float kGeluC3 = 0.035677408136300125f;  // 0.044715 sqrt(2/pi)

__device__ __forceinline__ float tanh_hw(float u)
{
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
    return t;
}

__device__ __forceinline__ float gelu_act(float z)
{
    const float hz = 0.5f * z;
    return fmaf(hz, tanh_hw(z * fmaf(kGeluC3, z * z, kGeluC1)), hz);
}

__device__ __forceinline__ float gelu_act_grad(float z)
{
    const float z2 = z * z;
    const float t = tanh_hw(z * fmaf(kGeluC3, z2, kGeluC1));
    const float du = fmaf(3.0f * kGeluC3, z2, kGeluC1);
    return fmaf(0.5f * z * (1.0f - t * t), du, 0.5f * (1.0f + t));
}
