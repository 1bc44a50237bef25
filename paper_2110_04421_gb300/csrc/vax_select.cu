// vax_select.cu -- daily dose selection of the vaccination priority strategies
// (Sec. 5, Table 1): a shared supply of Q doses goes to the eligible agents with
// the smallest (priority key, agent id).
//
// Keys are small integers (class < 160), so the day's selection is a counting
// problem: (1) every agent computes its class from the state at the start of the
// day and scatters it to its caller id, with a class histogram; (2) one block
// finds the class c* where the cumulative count reaches Q; (3) classes before c*
// are dosed entirely, and inside c* the first Q - (earlier classes) agents by
// caller id, ranked with per-block counts and a scan.
#include <cuda_runtime.h>

#include <cstdint>

#include "deabm_device.cuh"
#include "kernels.h"

namespace deabm {

constexpr uint32_t kVaxClasses = 160;
constexpr uint32_t kSelBlock = 1024;

__device__ __forceinline__ uint32_t vax_key(uint32_t strategy, uint32_t elderly_bin, int age, uint32_t type)
{
    const uint32_t older = (uint32_t)(8 - age);
    if (strategy == 1) return (type == 2u ? 0u : 1u) * 16u + older;
    if (strategy == 2) return (type == 1u ? 0u : 1u) * 16u + older;
    if ((uint32_t)age >= elderly_bin) return older * 2u + (type - 1u);
    return (type == 1u ? 1u : 2u) * 64u + older * 2u;
}

__global__ void vax_class_kernel(const KParams P, uint32_t day, uint32_t dose2_delay, uint32_t elderly_bin,
                                 StateRef S, uint8_t *cls_caller, uint32_t *counts)
{
    __shared__ uint32_t h[kVaxClasses];
    for (uint32_t q = threadIdx.x; q < kVaxClasses; q += blockDim.x) h[q] = 0;
    __syncthreads();
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < P.n) {
        const int st = S.stage[j];
        const uint32_t fl = S.flags[j];
        uint32_t type = 0;
        if (!(st == DEABM_HOSP || st == DEABM_ICU || st == DEABM_DEAD)) {
            if (!(fl & DEABM_FL_DOSE1)) type = 1;
            else if (!(fl & DEABM_FL_DOSE2) && (int64_t)day - (int64_t)S.vd1[j] >= (int64_t)dose2_delay) type = 2;
        }
        uint8_t c = 255;
        if (type) {
            c = (uint8_t)vax_key(P.vax_strategy, elderly_bin, P.age[j], type);
            atomicAdd(&h[c], 1u);
        }
        cls_caller[P.orig_id ? P.orig_id[j] : j] = c;
    }
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < kVaxClasses; q += blockDim.x)
        if (h[q]) atomicAdd(&counts[q], h[q]);
}

// one thread: threshold class and how many of it are dosed (sel[0] = c*, sel[1] = r)
__global__ void vax_threshold_kernel(const uint32_t *counts, uint32_t supply, uint32_t *sel)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint32_t cum = 0, c = 0;
    for (; c < kVaxClasses; ++c) {
        if (cum + counts[c] >= supply) break;
        cum += counts[c];
    }
    sel[0] = c;                               // kVaxClasses: every eligible agent is dosed
    sel[1] = c < kVaxClasses ? supply - cum : 0u;
}

__global__ void __launch_bounds__(kSelBlock) vax_block_count_kernel(const uint8_t *cls, uint32_t n, const uint32_t *sel,
                                                                    uint32_t *bcnt)
{
    __shared__ uint32_t s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    const uint32_t o = blockIdx.x * kSelBlock + threadIdx.x;
    const bool m = o < n && cls[o] == sel[0];
    const unsigned b = __ballot_sync(0xFFFFFFFFu, m);
    if ((threadIdx.x & 31u) == 0 && b) atomicAdd(&s, (uint32_t)__popc(b));
    __syncthreads();
    if (threadIdx.x == 0) bcnt[blockIdx.x] = s;
}

// one warp: exclusive scan of the per-block counts (in place)
__global__ void vax_scan_kernel(uint32_t *bcnt, uint32_t blocks)
{
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t running = 0;
    for (uint32_t q0 = 0; q0 < blocks; q0 += 32u) {
        const uint32_t q = q0 + lane;
        const uint32_t c = q < blocks ? bcnt[q] : 0u;
        uint32_t incl = c;
        for (uint32_t off = 1; off < 32u; off <<= 1) {
            const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, off);
            if (lane >= off) incl += v;
        }
        if (q < blocks) bcnt[q] = running + incl - c;
        running += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
}

__global__ void __launch_bounds__(kSelBlock) vax_decide_kernel(const uint8_t *cls, uint32_t n, const uint32_t *sel,
                                                               const uint32_t *boff, uint8_t *dose)
{
    __shared__ uint32_t wcnt[kSelBlock / 32];
    const uint32_t o = blockIdx.x * kSelBlock + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const uint32_t cstar = sel[0], r = sel[1];
    const uint32_t c = o < n ? cls[o] : 255u;
    const bool m = o < n && c == cstar;
    const unsigned b = __ballot_sync(0xFFFFFFFFu, m);
    if (lane == 0) wcnt[w] = __popc(b);
    __syncthreads();
    if (o >= n) return;
    uint32_t rank = boff[blockIdx.x] + __popc(b & ((1u << lane) - 1u));
    for (uint32_t v = 0; v < w; ++v) rank += wcnt[v];
    dose[o] = (c != 255u && (c < cstar || (m && rank < r))) ? 1 : 0;
}

size_t vax_select_scratch_words(uint32_t n) { return kVaxClasses + 2 + (n + kSelBlock - 1) / kSelBlock; }

cudaError_t launch_vax_select(const KParams &P, uint32_t day, uint32_t dose2_delay, uint32_t elderly_bin,
                              uint32_t supply, const StateRef &S, uint8_t *cls_caller, uint8_t *dose_caller,
                              uint32_t *scratch, cudaStream_t stream)
{
    const uint32_t n = P.n;
    uint32_t *counts = scratch, *sel = scratch + kVaxClasses, *bcnt = scratch + kVaxClasses + 2;
    const uint32_t blocks = (n + kSelBlock - 1) / kSelBlock;
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * kVaxClasses, stream);
    if (e != cudaSuccess) return e;
    vax_class_kernel<<<(n + 255u) / 256u, 256, 0, stream>>>(P, day, dose2_delay, elderly_bin, S, cls_caller, counts);
    vax_threshold_kernel<<<1, 32, 0, stream>>>(counts, supply, sel);
    vax_block_count_kernel<<<blocks, kSelBlock, 0, stream>>>(cls_caller, n, sel, bcnt);
    vax_scan_kernel<<<1, 32, 0, stream>>>(bcnt, blocks);
    vax_decide_kernel<<<blocks, kSelBlock, 0, stream>>>(cls_caller, n, sel, bcnt, dose_caller);
    return cudaGetLastError();
}

// ---- batched contexts: the same selection in every replicate column, each
// from its own state and dose-2 delay, with the same supply.  The class array is
// [caller id][replicate] like the state; the per-column ranking inside the
// threshold class walks caller ids in chunks of kSelChunk (a thread per (chunk,
// column), the columns of a warp side by side so every read is coalesced).
constexpr uint32_t kSelChunk = 256;

__global__ void vax_class_batch_kernel(const KParams P, uint32_t day, uint32_t elderly_bin, StateRef S, uint8_t *cls,
                                       uint32_t *counts)
{
    __shared__ uint32_t h[kVaxClasses][32];
    const uint32_t lane = threadIdx.x, wy = threadIdx.y, B = P.n_rep;
    for (uint32_t q = wy * 32u + lane; q < kVaxClasses * 32u; q += 256u) (&h[0][0])[q] = 0;
    __syncthreads();
    const uint32_t b = blockIdx.y * 32u + lane;
    if (b < B) {
        const uint32_t delay = P.rep[b].dose2_delay;
        for (uint32_t t = 0; t < 8u; ++t) {
            const uint32_t j = blockIdx.x * 64u + t * 8u + wy;
            if (j >= P.n) break;
            const size_t i = (size_t)j * B + b;
            const int st = S.stage[i];
            const uint32_t fl = S.flags[i];
            uint32_t type = 0;
            if (!(st == DEABM_HOSP || st == DEABM_ICU || st == DEABM_DEAD)) {
                if (!(fl & DEABM_FL_DOSE1)) type = 1;
                else if (!(fl & DEABM_FL_DOSE2) && (int64_t)day - (int64_t)S.vd1[i] >= (int64_t)delay) type = 2;
            }
            uint8_t c = 255;
            if (type) {
                c = (uint8_t)vax_key(P.vax_strategy, elderly_bin, P.age[j], type);
                atomicAdd(&h[c][lane], 1u);
            }
            cls[(size_t)(P.orig_id ? P.orig_id[j] : j) * B + b] = c;
        }
    }
    __syncthreads();
    for (uint32_t q = wy * 32u + lane; q < kVaxClasses * 32u; q += 256u) {
        const uint32_t c = q / 32u, l = q % 32u, bb = blockIdx.y * 32u + l;
        if (bb < B && h[c][l]) atomicAdd(&counts[(size_t)bb * kVaxClasses + c], h[c][l]);
    }
}

// a thread per column: threshold class and how many of it are dosed (sel[2b], sel[2b+1])
__global__ void vax_threshold_batch_kernel(const uint32_t *counts, uint32_t B, uint32_t supply, uint32_t *sel)
{
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const uint32_t *cb = counts + (size_t)b * kVaxClasses;
    uint32_t cum = 0, c = 0;
    for (; c < kVaxClasses; ++c) {
        if (cum + cb[c] >= supply) break;
        cum += cb[c];
    }
    sel[2u * b] = c;
    sel[2u * b + 1u] = c < kVaxClasses ? supply - cum : 0u;
}

// per (chunk, column): members of the column's threshold class in the chunk
__global__ void vax_chunk_count_kernel(const uint8_t *cls, uint32_t n, uint32_t B, const uint32_t *sel, uint32_t *ccnt)
{
    const uint32_t b = blockIdx.y * 32u + threadIdx.x, chunk = blockIdx.x * blockDim.y + threadIdx.y;
    const uint32_t chunks = (n + kSelChunk - 1u) / kSelChunk;
    if (b >= B || chunk >= chunks) return;
    const uint32_t cstar = sel[2u * b], o1 = min(n, (chunk + 1u) * kSelChunk);
    uint32_t cnt = 0;
    for (uint32_t o = chunk * kSelChunk; o < o1; ++o) cnt += cls[(size_t)o * B + b] == cstar ? 1u : 0u;
    ccnt[(size_t)chunk * B + b] = cnt;
}

// a thread per column: exclusive scan of its chunk counts, in chunk order (in place)
__global__ void vax_chunk_scan_kernel(uint32_t *ccnt, uint32_t chunks, uint32_t B)
{
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    uint32_t run = 0;
    for (uint32_t c = 0; c < chunks; ++c) {
        const uint32_t v = ccnt[(size_t)c * B + b];
        ccnt[(size_t)c * B + b] = run;
        run += v;
    }
}

// per (chunk, column): the chunk's agents in caller-id order, ranked inside the
// threshold class from the chunk's offset
__global__ void vax_chunk_decide_kernel(const uint8_t *cls, uint32_t n, uint32_t B, const uint32_t *sel,
                                        const uint32_t *coff, uint8_t *dose)
{
    const uint32_t b = blockIdx.y * 32u + threadIdx.x, chunk = blockIdx.x * blockDim.y + threadIdx.y;
    const uint32_t chunks = (n + kSelChunk - 1u) / kSelChunk;
    if (b >= B || chunk >= chunks) return;
    const uint32_t cstar = sel[2u * b], r = sel[2u * b + 1u], o1 = min(n, (chunk + 1u) * kSelChunk);
    uint32_t rank = coff[(size_t)chunk * B + b];
    for (uint32_t o = chunk * kSelChunk; o < o1; ++o) {
        const size_t i = (size_t)o * B + b;
        const uint32_t c = cls[i];
        const bool m = c == cstar;
        dose[i] = (c != 255u && (c < cstar || (m && rank < r))) ? 1 : 0;
        if (m) ++rank;
    }
}

size_t vax_select_batch_scratch_words(uint32_t n, uint32_t B)
{
    return (size_t)B * (kVaxClasses + 2u) + (size_t)((n + kSelChunk - 1u) / kSelChunk) * B;
}

cudaError_t launch_vax_select_batch(const KParams &P, uint32_t day, uint32_t elderly_bin, uint32_t supply,
                                    const StateRef &S, uint8_t *cls, uint8_t *dose, uint32_t *scratch,
                                    cudaStream_t stream)
{
    const uint32_t n = P.n, B = P.n_rep, chunks = (n + kSelChunk - 1u) / kSelChunk;
    uint32_t *counts = scratch, *sel = scratch + (size_t)B * kVaxClasses, *ccnt = sel + 2u * (size_t)B;
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * kVaxClasses * (size_t)B, stream);
    if (e != cudaSuccess) return e;
    const uint32_t cgroups = (B + 31u) / 32u;
    vax_class_batch_kernel<<<dim3((n + 63u) / 64u, cgroups), dim3(32, 8), 0, stream>>>(P, day, elderly_bin, S, cls,
                                                                                      counts);
    vax_threshold_batch_kernel<<<(B + 127u) / 128u, 128, 0, stream>>>(counts, B, supply, sel);
    const dim3 cgrid((chunks + 7u) / 8u, cgroups), cblock(32, 8);
    vax_chunk_count_kernel<<<cgrid, cblock, 0, stream>>>(cls, n, B, sel, ccnt);
    vax_chunk_scan_kernel<<<(B + 127u) / 128u, 128, 0, stream>>>(ccnt, chunks, B);
    vax_chunk_decide_kernel<<<cgrid, cblock, 0, stream>>>(cls, n, B, sel, ccnt, dose);
    return cudaGetLastError();
}

}  // namespace deabm
