// curand_philox_ref.cu -- test helper: Philox4x32-10 outputs from cuRAND's device
// API (curand_kernel.h, used as a library) for a list of (key, counter) pairs, so
// the oracle's Philox can be checked against an implementation it shares nothing
// with.  Mapping: curand_init(seed, subsequence, offset) starts the 128-bit
// counter at (offset / 4) in words x, y and subsequence in words z, w, with the
// 64-bit seed as the key; for offset a multiple of 4, curand4 then returns
// Philox4x32-10 of that counter.  So counter (c0, c1, c2, c3) is reached with
// offset = 4 * (c0 | c1 << 32) (c1 < 2^30 here) and subsequence = c2 | c3 << 32.
//
// usage: curand_philox_ref <in.bin> <out.bin>
//   in.bin : uint32 n, then n records of uint32 {key_lo, key_hi, c0, c1, c2, c3}
//   out.bin: n records of uint32 {x, y, z, w}
#include <cuda_runtime.h>
#include <curand_kernel.h>

#include <cstdint>
#include <cstdio>
#include <vector>

__global__ void philox_ref(const uint32_t *in, uint32_t n, uint4 *out)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t *r = in + (size_t)i * 6;
    const unsigned long long seed = (unsigned long long)r[0] | ((unsigned long long)r[1] << 32);
    const unsigned long long offset = 4ull * ((unsigned long long)r[2] | ((unsigned long long)r[3] << 32));
    const unsigned long long subseq = (unsigned long long)r[4] | ((unsigned long long)r[5] << 32);
    curandStatePhilox4_32_10_t st;
    curand_init(seed, subseq, offset, &st);
    out[i] = curand4(&st);
}

int main(int argc, char **argv)
{
    if (argc != 3) return 2;
    FILE *f = std::fopen(argv[1], "rb");
    if (!f) return 3;
    uint32_t n = 0;
    if (std::fread(&n, 4, 1, f) != 1 || n == 0 || n > (1u << 24)) return 4;
    std::vector<uint32_t> in((size_t)n * 6);
    if (std::fread(in.data(), 4, in.size(), f) != in.size()) return 5;
    std::fclose(f);
    uint32_t *d_in = nullptr;
    uint4 *d_out = nullptr;
    if (cudaMalloc(&d_in, in.size() * 4) != cudaSuccess || cudaMalloc(&d_out, (size_t)n * 16) != cudaSuccess) return 6;
    cudaMemcpy(d_in, in.data(), in.size() * 4, cudaMemcpyHostToDevice);
    philox_ref<<<(n + 255) / 256, 256>>>(d_in, n, d_out);
    std::vector<uint4> out(n);
    if (cudaMemcpy(out.data(), d_out, (size_t)n * 16, cudaMemcpyDeviceToHost) != cudaSuccess) return 7;
    cudaFree(d_in);
    cudaFree(d_out);
    FILE *g = std::fopen(argv[2], "wb");
    if (!g) return 8;
    std::fwrite(out.data(), 16, n, g);
    std::fclose(g);
    return 0;
}
