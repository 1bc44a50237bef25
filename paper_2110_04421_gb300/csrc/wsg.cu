// wsg.cu -- the day's global random network as a Watts-Strogatz graph (Sec. 3
// "Interaction Networks": one small-world graph, re-initialised every step),
// built on the device before the day kernel, which then gathers along it.
//
// The ring lattice runs over all agents in caller-id order; agent i owns the h
// undirected edges to (i + m) mod n, m = 1..h.  Every day each owned edge is
// rewired with the rewiring probability (always when i + m wraps onto i): its far
// end moves to a uniform other agent.  Edges are undirected, so a destination's
// messages come from its own edges' far ends, from the lattice edges of the h
// agents before it that were not rewired, and from the rewired edges that
// landed on it.  Those last ones are the transpose of a random map, built here
// each day:
//   1. mark: per owner, one Philox block per two edges; the rewired bits go to
//      a byte per agent, each rewired edge's new far end to far[owner h + m - 1],
//      and it is counted at that far end (ends[v + 2]);
//   2. an inclusive prefix sum over ends[0 .. n+3) leaves ends[v + 2] = the end
//      of agent v's landing slots and ends[n + 2] = their total;
//   3. fill: each rewired edge takes the last free slot of its far end by
//      decrementing ends[v + 2], which finishes at the start of v's slots, so
//      afterwards agent v's landings are land[ends[v + 2] .. ends[v + 3]);
//   4. order: each agent's landing owners are sorted ascending (a few per agent),
//      so the day kernel sums them in a fixed order and the result does not
//      depend on the order the atomics ran in (the prefix sum is the two-launch
//      tiled scan of relabel.cu).
#include <cuda_runtime.h>

#include <cstdint>

#include "day_common.cuh"
#include "deabm_device.cuh"
#include "kernels.h"

namespace deabm {

__global__ void wsg_mark_kernel(const KParams P, uint32_t day, uint8_t *rew, uint32_t *far, uint32_t *ends)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const uint32_t h = P.wsg_h;
    uint32_t bits = 0;
    for (uint32_t m = 1; m <= h; m += 2u) {
        const uint4 w = draw_rk(P.nrk, i, day, kStreamWsg, (m - 1u) >> 1);
#pragma unroll
        for (uint32_t u = 0; u < 2u; ++u) {
            const uint32_t e = m + u;
            if (e > h) break;
            const uint32_t coin = u ? w.z : w.x, word = u ? w.w : w.y;
            if (e % P.n == 0u || (uint64_t)coin < P.thr_wsg) {
                uint32_t v = (uint32_t)(((uint64_t)word * (uint64_t)(P.n - 1u)) >> 32);
                v += (v >= i) ? 1u : 0u;
                bits |= 1u << (e - 1u);
                far[i * h + (e - 1u)] = v;
                atomicAdd(ends + v + 2u, 1u);
            }
        }
    }
    rew[i] = (uint8_t)bits;
}

// each rewired edge's owner into a slot of its far end.  Only owners are kept:
// two edges of one owner that land on the same agent carry the same message, so
// the order between them does not change the sum.
__global__ void wsg_fill_kernel(uint32_t n, uint32_t h, const uint8_t *rew, const uint32_t *far, uint32_t *ends,
                                uint32_t *land)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t bits = rew[i];
    while (bits) {
        const uint32_t e = (uint32_t)__ffs(bits) - 1u;
        bits &= bits - 1u;
        land[atomicSub(ends + far[i * h + e] + 2u, 1u) - 1u] = i;
    }
}

// each agent's landing owners in ascending order: up to kSortCap of them loaded
// at once and sorted in registers (odd-even transposition network), more than
// that by insertion in place (rare: the counts are about Poisson(h beta))
constexpr uint32_t kSortCap = 8;
__global__ void wsg_order_kernel(uint32_t n, const uint32_t *start, uint32_t *land)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const uint32_t s0 = start[v], c = start[v + 1u] - s0;
    if (c < 2u) return;
    if (c <= kSortCap) {
        uint32_t k[kSortCap];
#pragma unroll
        for (uint32_t u = 0; u < kSortCap; ++u) k[u] = u < c ? land[s0 + u] : 0xFFFFFFFFu;
#pragma unroll
        for (uint32_t r = 0; r < kSortCap; ++r)
#pragma unroll
            for (uint32_t u = r & 1u; u + 1u < kSortCap; u += 2u) {
                const uint32_t lo = min(k[u], k[u + 1u]), hi = max(k[u], k[u + 1u]);
                k[u] = lo;
                k[u + 1u] = hi;
            }
#pragma unroll
        for (uint32_t u = 0; u < kSortCap; ++u)
            if (u < c) land[s0 + u] = k[u];
        return;
    }
    for (uint32_t a = s0 + 1u; a < s0 + c; ++a) {
        const uint32_t key = land[a];
        uint32_t b = a;
        while (b > s0 && land[b - 1u] > key) {
            land[b] = land[b - 1u];
            --b;
        }
        land[b] = key;
    }
}

size_t wsg_scratch_words(uint32_t n) { return scan_scratch_words((size_t)n + 3u); }

__global__ void wsg_slot_kernel(KParams *kp, uint32_t day)
{
    const uint32_t slot = day % kp->wsg_ring_days;
    kp->wsg_start = kp->wsg_ends_ring + (size_t)slot * ((size_t)kp->n + 3u) + 2u;
    kp->wsg_land = kp->wsg_land_ring + (size_t)slot * kp->n * kp->wsg_h;
}

cudaError_t launch_wsg_slot(KParams *kp_dev, uint32_t day, cudaStream_t s)
{
    wsg_slot_kernel<<<1, 1, 0, s>>>(kp_dev, day);
    return cudaGetLastError();
}

cudaError_t launch_wsg_build(const KParams &P, uint32_t day, const WsgBuffers &B, cudaStream_t s)
{
    const uint32_t n = P.n, h = P.wsg_h;
    cudaError_t e = cudaMemsetAsync(B.ends, 0, sizeof(uint32_t) * ((size_t)n + 3u), s);
    if (e != cudaSuccess) return e;
    const uint32_t blocks = (n + 255u) / 256u;
    wsg_mark_kernel<<<blocks, 256, 0, s>>>(P, day, B.rew, B.far, B.ends);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_scan_inclusive(B.ends, (size_t)n + 3u, B.scratch, s)) != cudaSuccess) return e;
    wsg_fill_kernel<<<blocks, 256, 0, s>>>(n, h, B.rew, B.far, B.ends, B.land);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    wsg_order_kernel<<<blocks, 256, 0, s>>>(n, B.ends + 2, B.land);
    return cudaGetLastError();
}

}  // namespace deabm
