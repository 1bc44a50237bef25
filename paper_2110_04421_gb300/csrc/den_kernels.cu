// den_kernels.cu -- digital exposure notification (Sec. 4.2) on the GPU.
//
// The notification goes from a positive app holder to the app holders that had
// it as an in-contact over the last den_window days.  It runs destination-
// centred, as a gather: after the day's update every eligible app holder j
// walks its own in-contacts of those days -- its stored CSR rows, and the daily
// occupation and random contacts the day kernel recorded for app holders while
// drawing them (a ring of den_window records per agent) -- and looks each
// source up in the day's byte map of positive app holders.
#include <cuda_runtime.h>
#include <cstdint>

#include "day_common.cuh"
#include "deabm_device.cuh"
#include "kernels.h"

namespace deabm {

// was any stored in-neighbour of row j a positive app holder today?
__device__ __forceinline__ bool den_static_hit(const KParams &P, uint32_t j)
{
    for (uint32_t net = 0; net < P.n_nets; ++net) {
        const uint32_t e1 = __ldg(P.row_ptr[net] + j + 1);
        for (uint32_t e = __ldg(P.row_ptr[net] + j); e < e1; ++e)
            if (P.den_src[__ldg(P.col[net] + e)]) return true;
    }
    return false;
}

// the random and occupation in-contacts of row j on day d, from the record the
// day kernel wrote while drawing them
__device__ __forceinline__ bool den_ring_hit(const KParams &P, uint32_t j, uint32_t d)
{
    const uint8_t *src_rand = P.den_src_orig ? P.den_src_orig : P.den_src;
    const uint32_t *rec = P.den_ring + ((size_t)(d % P.den_window) * P.n + j) * P.den_slots;
    const uint32_t h = rec[0], kr = h & 0xFFu, ko = h >> 8;
    for (uint32_t e = 0; e < kr; ++e)
        if (src_rand[rec[1u + e]]) return true;
    for (uint32_t e = 0; e < ko; ++e)
        if (P.den_src[rec[kDenOccAt + e]]) return true;
    return false;
}

__global__ void __launch_bounds__(256) den_kernel(const KParams P, uint32_t day, StateRef S, Counters C)
{
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    bool notified = false;
    // nothing to do on a day without a positive app holder
    if (j < P.n && __ldg(P.den_pos + day) > 0) {
        const uint32_t fl = S.flags[j];
        const int st = S.stage[j];
        if ((fl & DEABM_FL_APP) && (S.qt[j] & 0x0Fu) == 0u && st != DEABM_HOSP && st != DEABM_ICU &&
            st != DEABM_DEAD) {
            bool hit = den_static_hit(P, j);
            const uint32_t d0 = day + 1u > P.den_window ? day + 1u - P.den_window : 0u;
            for (uint32_t d = d0; d <= day && !hit; ++d) hit = den_ring_hit(P, j, d);
            if (hit) {
                notified = true;
                const uint32_t jo = P.orig_id ? __ldg(P.orig_id + j) : j;
                const uint32_t w = draw(seed_key(P.rep[0].seed), jo, day, kStreamDen).x;
                if ((uint64_t)w < P.thr_comp) S.flags[j] = (uint8_t)(fl | DEABM_FL_DEN);
            }
        }
    }
    const unsigned b = __ballot_sync(0xFFFFFFFFu, notified);
    if ((threadIdx.x & 31u) == 0u && b) atomicAdd(&s_cnt, __popc(b));
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd(C.den + day, s_cnt);
}

// app holders, drawn once: word x of (seed, caller id, day word 0xFFFFFFFD, stream 6)
__global__ void den_apps_kernel(const KParams P, StateRef S)
{
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.n) return;
    const uint32_t jo = P.orig_id ? __ldg(P.orig_id + j) : j;
    const uint32_t w = draw(seed_key(P.rep[0].seed), jo, 0xFFFFFFFDu, kStreamDen).x;
    const uint32_t fl = S.flags[j];
    S.flags[j] = (uint8_t)((uint64_t)w < P.thr_adopt ? (fl | DEABM_FL_APP) : (fl & ~DEABM_FL_APP));
}

cudaError_t launch_den_apps(const KParams &P, const StateRef &S, cudaStream_t stream)
{
    den_apps_kernel<<<(P.n + 255u) / 256u, 256, 0, stream>>>(P, S);
    return cudaGetLastError();
}

cudaError_t launch_den(const KParams &P, uint32_t day, const StateRef &S, const Counters &C, cudaStream_t stream)
{
    den_kernel<<<(P.n + 255u) / 256u, 256, 0, stream>>>(P, day, S, C);
    return cudaGetLastError();
}

}  // namespace deabm
