// den_kernels.cu -- digital exposure notification (Sec. 4.2) on the GPU.
//
// The notification goes from a positive app holder to the app holders that had
// it as an in-contact over the last den_window days.  It runs destination-
// centred, as a gather: after the day's update every eligible app holder j
// re-generates its own in-contacts of those days -- the stored CSR rows, and
// the daily occupation and random contacts from the same Philox words the day
// kernels drew them from -- and looks each source up in the day's byte map of
// positive app holders.  Nothing about past days is stored.
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

// the occupation contacts of row j (caller id jo) on day d, as drawn by occ_sum
__device__ __forceinline__ bool den_occ_hit(const KParams &P, uint32_t j, uint32_t jo, uint32_t d)
{
    const uint32_t g = __ldg(P.occ_gid + j);
    const uint32_t beg = __ldg(P.occ_start + g), size = __ldg(P.occ_start + g + 1u) - beg;
    const uint32_t k = size > 1u ? (uint32_t)__ldg(P.occ_k + g) : 0u;
    const uint2 nk = seed_key(P.net_seed);
    for (uint32_t e = 0; e < k; e += 4u) {
        const uint4 w = draw(nk, jo, d, kStreamOcc, e >> 2);
        const uint32_t x[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (uint32_t u = 0; u < 4u; ++u)
            if (e + u < k && P.den_src[beg + occ_place(x[u], size - 1u, j - beg)]) return true;
    }
    return false;
}

// the random contacts of caller id jo on day d, as drawn by random_sum
__device__ __forceinline__ bool den_rand_hit(const KParams &P, uint32_t jo, uint32_t d)
{
    const uint8_t *src = P.den_src_orig ? P.den_src_orig : P.den_src;
    const uint2 nk = seed_key(P.net_seed);
    uint4 w = draw(nk, jo, d, kStreamRnet, 0u);
    uint32_t k = 0;
    while (k < DEABM_POIS_CAP && (uint64_t)w.x >= __ldg(&P.tab->pois[k])) ++k;
    const uint64_t nm1 = (uint64_t)(P.n - 1u);
    for (uint32_t e = 0; e < k; ++e) {
        const uint32_t idx = e + 1u;
        if ((idx & 3u) == 0u) w = draw(nk, jo, d, kStreamRnet, idx >> 2);
        const uint32_t x = (idx & 3u) == 1u ? w.y : (idx & 3u) == 2u ? w.z : (idx & 3u) == 3u ? w.w : w.x;
        uint32_t v = (uint32_t)(((uint64_t)x * nm1) >> 32);
        v += (v >= jo) ? 1u : 0u;
        if (src[v]) return true;
    }
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
            const uint32_t jo = P.orig_id ? __ldg(P.orig_id + j) : j;
            bool hit = den_static_hit(P, j);
            const uint32_t d0 = day + 1u > P.den_window ? day + 1u - P.den_window : 0u;
            for (uint32_t d = d0; d <= day && !hit; ++d) {
                if (P.n_occ) hit = den_occ_hit(P, j, jo, d);
                if (!hit && P.rand_on) hit = den_rand_hit(P, jo, d);
            }
            if (hit) {
                notified = true;
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
