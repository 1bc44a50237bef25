// relabel.cu -- the library's internal agent numbering, built on the GPU.
//
// Agents are renumbered so that the members of a group (a workplace) sit next
// to each other and a warp's in-edge gathers touch few cache lines.  The order
// is: agents grouped by the smallest id that reaches them along the in-edges
// of the network with the most edges (a min-label propagation, a fixed number
// of rounds), groups in order of that label, ids ascending inside a group.
// Any permutation gives the same results (draws and outputs use the caller's
// ids); this one only decides where data sits.  Also here: the CSR rebuilt in
// the new numbering and the copy of internal-order arrays back to caller order.
#include <cuda_runtime.h>
#include <cstdint>

#include "kernels.h"

namespace deabm {

__global__ void label_init_kernel(uint32_t *label, uint32_t n)
{
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) label[v] = v;
}

// one Jacobi round: out[v] = min(in[v], in[u] for every in-edge u -> v)
__global__ void label_round_kernel(const uint32_t *__restrict__ rp, const uint32_t *__restrict__ col,
                                   const uint32_t *__restrict__ in, uint32_t *__restrict__ out, uint32_t n)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    uint32_t m = in[v];
    const uint32_t e1 = rp[v + 1];
    for (uint32_t e = rp[v]; e < e1; ++e) m = min(m, __ldg(in + col[e]));
    out[v] = m;
}

cudaError_t launch_locality_labels(const uint32_t *rp, const uint32_t *col, uint32_t n, uint32_t rounds,
                                   uint32_t *label, uint32_t *tmp, cudaStream_t stream)
{
    const uint32_t blocks = (n + 255u) / 256u;
    label_init_kernel<<<blocks, 256, 0, stream>>>(label, n);
    for (uint32_t r = 0; r < rounds; ++r) {  // rounds is even: the result ends in `label`
        label_round_kernel<<<blocks, 256, 0, stream>>>(rp, col, (r & 1u) ? tmp : label, (r & 1u) ? label : tmp, n);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- CSR in the new numbering
// deg[q + 1] = in-degree of the agent now at row q (deg[0] = 0)
__global__ void csr_degree_kernel(const uint32_t *__restrict__ rp, const uint32_t *__restrict__ new2orig, uint32_t n,
                                  uint32_t *__restrict__ deg)
{
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q == 0) deg[0] = 0;
    if (q >= n) return;
    const uint32_t o = new2orig[q];
    deg[q + 1] = rp[o + 1] - rp[o];
}

// inclusive scan of a[0..m) in place, in blocks of 1024 (block totals to `sums`)
constexpr uint32_t kScanBlock = 1024;

__device__ __forceinline__ uint32_t block_inclusive_scan(uint32_t x, uint32_t *warp_tot)
{
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
#pragma unroll
    for (uint32_t d = 1; d < 32u; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31u) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = lane < kScanBlock / 32u ? warp_tot[lane] : 0u;
#pragma unroll
        for (uint32_t d = 1; d < 32u; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, d);
            if (lane >= d) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    return x + (wid ? warp_tot[wid - 1] : 0u);
}

__global__ void __launch_bounds__(kScanBlock) scan_blocks_kernel(uint32_t *a, size_t m, uint32_t *sums)
{
    __shared__ uint32_t warp_tot[32];
    const size_t i = (size_t)blockIdx.x * kScanBlock + threadIdx.x;
    const uint32_t x = block_inclusive_scan(i < m ? a[i] : 0u, warp_tot);
    if (i < m) a[i] = x;
    if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = x;
}

__global__ void add_block_offsets_kernel(uint32_t *a, size_t m, const uint32_t *sums)
{
    const size_t i = (size_t)blockIdx.x * kScanBlock + threadIdx.x;
    if (blockIdx.x > 0 && i < m) a[i] += sums[blockIdx.x - 1];
}

// scratch: 2 * ceil(m / 1024) + 2 words (recursive block sums)
static cudaError_t scan_inplace(uint32_t *a, size_t m, uint32_t *scratch, cudaStream_t stream)
{
    const size_t nb = (m + kScanBlock - 1) / kScanBlock;
    scan_blocks_kernel<<<(unsigned)nb, kScanBlock, 0, stream>>>(a, m, scratch);
    if (nb > 1) {
        cudaError_t e = scan_inplace(scratch, nb, scratch + nb, stream);
        if (e != cudaSuccess) return e;
        add_block_offsets_kernel<<<(unsigned)nb, kScanBlock, 0, stream>>>(a, m, scratch);
    }
    return cudaGetLastError();
}

size_t scan_scratch_words(size_t m)
{
    size_t words = 0;
    while (m > 1) {
        m = (m + kScanBlock - 1) / kScanBlock;
        words += m;
    }
    return words + 2;
}

// one warp per new row: its edges in the caller's order, sources renumbered
__global__ void csr_copy_kernel(const uint32_t *__restrict__ rp, const uint32_t *__restrict__ col,
                                const uint32_t *__restrict__ new2orig, const uint32_t *__restrict__ orig2new,
                                const uint32_t *__restrict__ rp_new, uint32_t n, uint32_t *__restrict__ col_new)
{
    const uint32_t q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31u;
    if (q >= n) return;
    const uint32_t o = new2orig[q], b0 = rp[o], len = rp[o + 1] - b0, d0 = rp_new[q];
    for (uint32_t i = lane; i < len; i += 32u) col_new[d0 + i] = orig2new[col[b0 + i]];
}

cudaError_t launch_csr_renumber(const uint32_t *rp, const uint32_t *col, const uint32_t *new2orig,
                                const uint32_t *orig2new, uint32_t n, uint32_t *rp_new, uint32_t *col_new,
                                uint32_t *scratch, cudaStream_t stream)
{
    csr_degree_kernel<<<(n + 256u) / 256u, 256, 0, stream>>>(rp, new2orig, n, rp_new);
    cudaError_t e = scan_inplace(rp_new, (size_t)n + 1, scratch, stream);
    if (e != cudaSuccess) return e;
    const uint64_t threads = (uint64_t)n * 32u;
    csr_copy_kernel<<<(unsigned)((threads + 255u) / 256u), 256, 0, stream>>>(rp, col, new2orig, orig2new, rp_new, n,
                                                                             col_new);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- from caller order
// out[q * n_rep + b] = in[orig[q]] (in[q] when orig is null), or
// in[orig[q] * n_rep + b] when the input has its replicates: a caller-order array
// put in internal order (and repeated over the replicates when it has none)
template <class T>
__global__ void from_caller_kernel(T *__restrict__ out, const T *__restrict__ in, const uint32_t *__restrict__ orig,
                                   uint32_t n, uint32_t n_rep, bool in_reps)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (uint64_t)n * n_rep) return;
    const uint32_t q = (uint32_t)(i / n_rep), b = (uint32_t)(i % n_rep);
    const uint64_t o = orig ? orig[q] : q;
    out[i] = in_reps ? in[o * n_rep + b] : in[o];
}

cudaError_t launch_from_caller(void *out, const void *in, const uint32_t *orig, uint32_t n, uint32_t n_rep,
                               uint32_t elem, bool in_reps, cudaStream_t stream)
{
    const uint64_t total = (uint64_t)n * n_rep;
    const unsigned blocks = (unsigned)((total + 255u) / 256u);
    if (elem == 1)
        from_caller_kernel<uint8_t><<<blocks, 256, 0, stream>>>((uint8_t *)out, (const uint8_t *)in, orig, n, n_rep,
                                                                 in_reps);
    else
        from_caller_kernel<uint16_t><<<blocks, 256, 0, stream>>>((uint16_t *)out, (const uint16_t *)in, orig, n,
                                                                  n_rep, in_reps);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- back to caller order
// out[(orig[q] * n_rep + b) * elem ...] = in[(q * n_rep + b) * elem ...]
template <class T>
__global__ void to_caller_kernel(T *__restrict__ out, const T *__restrict__ in, const uint32_t *__restrict__ orig,
                                 uint32_t n, uint32_t n_rep)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (uint64_t)n * n_rep) return;
    const uint32_t q = (uint32_t)(i / n_rep), b = (uint32_t)(i % n_rep);
    out[(uint64_t)orig[q] * n_rep + b] = in[i];
}

cudaError_t launch_to_caller(void *out, const void *in, const uint32_t *orig, uint32_t n, uint32_t n_rep,
                             uint32_t elem, cudaStream_t stream)
{
    const uint64_t total = (uint64_t)n * n_rep;
    const unsigned blocks = (unsigned)((total + 255u) / 256u);
    if (elem == 1)
        to_caller_kernel<uint8_t><<<blocks, 256, 0, stream>>>((uint8_t *)out, (const uint8_t *)in, orig, n, n_rep);
    else if (elem == 2)
        to_caller_kernel<uint16_t><<<blocks, 256, 0, stream>>>((uint16_t *)out, (const uint16_t *)in, orig, n, n_rep);
    else
        to_caller_kernel<uint32_t><<<blocks, 256, 0, stream>>>((uint32_t *)out, (const uint32_t *)in, orig, n, n_rep);
    return cudaGetLastError();
}

}  // namespace deabm
