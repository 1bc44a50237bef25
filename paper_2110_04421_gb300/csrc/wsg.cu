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
//      a byte per agent, each rewired edge is counted at its new far end and
//      appended to a list (warp-aggregated append);
//   2. an inclusive prefix sum of the counts (stored one slot up) gives every
//      agent's first landing slot;
//   3. fill: each listed edge takes a slot of its far end (atomic cursor);
//   4. order: each agent's landing owners are sorted ascending (a few per agent),
//      so the day kernel sums them in a fixed order and the result does not
//      depend on the order the atomics ran in.
#include <cuda_runtime.h>

#include <cstdint>

#include "day_common.cuh"
#include "deabm_device.cuh"
#include "kernels.h"

namespace deabm {

__global__ void wsg_mark_kernel(const KParams P, uint32_t day, uint8_t *rew, uint32_t *cnt1, uint32_t *list,
                                uint32_t *list_n)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < P.n;
    const uint32_t h = P.wsg_h, lane = threadIdx.x & 31u;
    uint32_t bits = 0;
    for (uint32_t m = 1; m <= h; m += 2u) {  // every lane runs every block (warp-wide appends)
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (active) w = draw_rk(P.nrk, i, day, kStreamWsg, (m - 1u) >> 1);
#pragma unroll
        for (uint32_t u = 0; u < 2u; ++u) {
            const uint32_t e = m + u;
            if (e > h) break;  // uniform
            const uint32_t coin = u ? w.z : w.x, word = u ? w.w : w.y;
            const bool r = active && (e % P.n == 0u || (uint64_t)coin < P.thr_wsg);
            uint32_t v = 0;
            if (r) {
                v = (uint32_t)(((uint64_t)word * (uint64_t)(P.n - 1u)) >> 32);
                v += (v >= i) ? 1u : 0u;
                bits |= 1u << (e - 1u);
                atomicAdd(cnt1 + v + 1u, 1u);
            }
            const unsigned ball = __ballot_sync(0xFFFFFFFFu, r);
            uint32_t base = 0;
            if (lane == 0 && ball) base = atomicAdd(list_n, (uint32_t)__popc(ball));
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (r) {
                const uint32_t q = base + (uint32_t)__popc(ball & ((1u << lane) - 1u));
                list[2u * q] = v;
                list[2u * q + 1u] = i * h + (e - 1u);  // owner and edge, in ascending order of (owner, m)
            }
        }
    }
    if (active) rew[i] = (uint8_t)bits;
}

__global__ void wsg_fill_kernel(const uint32_t *list, const uint32_t *list_n, const uint32_t *start, uint32_t *fill,
                                uint32_t *land)
{
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= *list_n) return;
    const uint32_t v = list[2u * q];
    land[start[v] + atomicAdd(fill + v, 1u)] = list[2u * q + 1u];
}

// each agent's landing edges in ascending (owner, m) order, then as owners
__global__ void wsg_order_kernel(uint32_t n, uint32_t h, const uint32_t *start, uint32_t *land)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const uint32_t s0 = start[v], s1 = start[v + 1u];
    for (uint32_t a = s0 + 1u; a < s1; ++a) {
        const uint32_t key = land[a];
        uint32_t b = a;
        while (b > s0 && land[b - 1u] > key) {
            land[b] = land[b - 1u];
            --b;
        }
        land[b] = key;
    }
    for (uint32_t a = s0; a < s1; ++a) land[a] /= h;
}

size_t wsg_scratch_words(uint32_t n) { return scan_scratch_words((size_t)n + 1u); }

cudaError_t launch_wsg_build(const KParams &P, uint32_t day, const WsgBuffers &B, cudaStream_t s)
{
    const uint32_t n = P.n;
    cudaError_t e = cudaMemsetAsync(B.cnt1, 0, sizeof(uint32_t) * ((size_t)n + 1u), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(B.fill, 0, sizeof(uint32_t) * n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(B.list_n, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const uint32_t blocks = (n + 255u) / 256u;
    wsg_mark_kernel<<<blocks, 256, 0, s>>>(P, day, B.rew, B.cnt1, B.list, B.list_n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_scan_inclusive(B.cnt1, (size_t)n + 1u, B.scratch, s)) != cudaSuccess) return e;
    const size_t edges = (size_t)n * P.wsg_h;
    wsg_fill_kernel<<<(unsigned)((edges + 255u) / 256u), 256, 0, s>>>(B.list, B.list_n, B.cnt1, B.fill, B.land);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    wsg_order_kernel<<<blocks, 256, 0, s>>>(n, P.wsg_h, B.cnt1, B.land);
    return cudaGetLastError();
}

}  // namespace deabm
