// den_kernels.cu -- digital exposure notification (Sec. 4.2) on the GPU.
//
// The notification goes from a positive app holder to the app holders that had
// it as an in-contact over the last den_window days.  It runs destination-
// centred, as a gather: after the day's update every eligible app holder j
// walks its own in-contacts of those days -- its stored CSR rows, and the daily
// occupation and random contacts the day kernel recorded for app holders while
// drawing them (a ring of den_window records per app holder, stored as word
// planes) -- and looks each
// source up in the day's bit map of positive app holders.  One thread per app
// holder, app holders listed in row order.  Batched contexts run the same
// notification in every replicate column at once (den_batch_* below).
#include <cuda_runtime.h>
#include <cstdint>

#include "day_common.cuh"
#include "deabm_device.cuh"
#include "kernels.h"

namespace deabm {

__device__ __forceinline__ bool bit_of(const uint32_t *map, uint32_t x) { return (__ldg(map + (x >> 5)) >> (x & 31u)) & 1u; }

// Agent jo's (caller id) neighbours in the Watts-Strogatz random network of day d
// (edges undirected: its in-contacts): f(caller id) for each, returning true to
// stop.  Its own edges' far ends and the unrewired lattice edges of the agents
// jo - m come from Philox (stream 10), the rewired edges that landed on jo from
// day d's slot of the kept graphs.  Returns whether f stopped the walk.
template <class F>
__device__ bool den_wsg_for(const KParams &P, uint32_t jo, uint32_t d, F f)
{
    const uint32_t n = P.n, h = P.wsg_h;
    for (uint32_t m = 1; m <= h; m += 2u) {
        const uint4 w = draw_rk(P.nrk, jo, d, kStreamWsg, (m - 1u) >> 1);
        if (f(wsg_far(P, jo, m, w.x, w.y))) return true;
        if (m + 1u <= h && f(wsg_far(P, jo, m + 1u, w.z, w.w))) return true;
    }
    for (uint32_t m = 1; m <= h; ++m) {
        const uint32_t i = (uint32_t)(((uint64_t)jo + (uint64_t)n - (uint64_t)(m % n)) % n);
        const uint4 w = draw_rk(P.nrk, i, d, kStreamWsg, (m - 1u) >> 1);
        const uint32_t coin = ((m - 1u) & 1u) ? w.z : w.x;
        const bool rewired = m % n == 0u || (uint64_t)coin < P.thr_wsg;
        if (!rewired && f(i)) return true;
    }
    const uint32_t slot = d % P.wsg_ring_days;
    const uint32_t *ends = P.wsg_ends_ring + (size_t)slot * ((size_t)n + 3u);
    const uint32_t *land = P.wsg_land_ring + (size_t)slot * n * h;
    const uint32_t s1 = __ldg(ends + jo + 3u);
    for (uint32_t q = __ldg(ends + jo + 2u); q < s1; ++q)
        if (f(__ldg(land + q))) return true;
    return false;
}

// was any stored in-neighbour of row j a positive app holder today?  Each row
// is taken in rounds of four edges: four column loads, then four bit lookups.
__device__ __forceinline__ bool den_static_hit(const KParams &P, uint32_t j)
{
    bool hit = false;
    for (uint32_t net = 0; net < P.n_nets; ++net) {
        const uint32_t e1 = __ldg(P.row_ptr[net] + j + 1);
        for (uint32_t e = __ldg(P.row_ptr[net] + j); e < e1; e += 4u) {
            uint32_t c[4];
#pragma unroll
            for (uint32_t u = 0; u < 4u; ++u) c[u] = e + u < e1 ? __ldg(P.col[net] + e + u) : 0u;
#pragma unroll
            for (uint32_t u = 0; u < 4u; ++u) hit |= (e + u < e1) && bit_of(P.den_bits, c[u]);
        }
    }
    return hit;
}

// The records of four days [c0, c0 + 4) of app holder a (days >= d1 empty):
// headers and first three random contacts, which cover most days' random
// contacts.  Records are word planes over the app holders, so a warp's loads of
// one word are coalesced.
struct RingChunk {
    uint32_t h[4], w1[4], w2[4], w3[4];
};

__device__ __forceinline__ const uint32_t *den_rec(const KParams &P, uint32_t a, uint32_t d)
{
    return P.den_ring + (size_t)(d % P.den_window) * P.den_slots * P.n_app + a;
}

__device__ __forceinline__ RingChunk den_ring_load(const KParams &P, uint32_t a, uint32_t c0, uint32_t d1)
{
    const size_t plane = P.n_app;
    RingChunk c;
#pragma unroll
    for (uint32_t u = 0; u < 4u; ++u) {
        const uint32_t *rec = den_rec(P, a, c0 + u);
        const bool ok = c0 + u < d1;
        c.h[u] = ok ? __ldg(rec) : 0u;
        c.w1[u] = ok ? __ldg(rec + plane) : 0u;
        c.w2[u] = ok ? __ldg(rec + 2 * plane) : 0u;
        c.w3[u] = ok ? __ldg(rec + 3 * plane) : 0u;
    }
    return c;
}

// any positive app holder among the contacts of a loaded chunk (the rest of a
// day's contacts loaded on demand)?
__device__ __forceinline__ bool den_ring_eval(const KParams &P, uint32_t a, uint32_t c0, const RingChunk &c)
{
    const uint32_t *src_rand = P.den_bits_orig ? P.den_bits_orig : P.den_bits;
    const size_t plane = P.n_app;
    bool hit = false;
#pragma unroll
    for (uint32_t u = 0; u < 4u; ++u) {
        const uint32_t kr = c.h[u] & 0xFFu, ko = c.h[u] >> 8;
        hit |= (kr > 0u && bit_of(src_rand, c.w1[u])) | (kr > 1u && bit_of(src_rand, c.w2[u])) |
               (kr > 2u && bit_of(src_rand, c.w3[u]));
        if (kr > 3u || ko) {
            const uint32_t *rec = den_rec(P, a, c0 + u);
            for (uint32_t e = 4u; e <= kr; ++e) hit |= bit_of(src_rand, __ldg(rec + e * plane));
            for (uint32_t e = 0; e < ko; ++e) hit |= bit_of(P.den_bits, __ldg(rec + (kDenOccAt + e) * plane));
        }
    }
    return hit;
}

// 8 blocks per SM (32 registers, some spilled): the pass waits on dependent loads,
// so more resident warps beat fewer spills (day with the pass, N = 2e6: 0.202 ms
// at 48 registers, 0.193 at 6 blocks, 0.190 at 8)
__global__ void __launch_bounds__(256, 8) den_kernel(const KParams P, uint32_t day, StateRef S, Counters C)
{
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const uint32_t a = blockIdx.x * blockDim.x + threadIdx.x;  // one thread per app holder
    bool notified = false;
    // nothing to do on a day without a positive app holder
    if (a < P.n_app && __ldg(P.den_pos + day) > 0) {
        // the first four days' records are requested before the agent's own state
        // and rows, so their latencies overlap
        const uint32_t d0 = day + 1u > P.den_window ? day + 1u - P.den_window : 0u;
        const RingChunk first = den_ring_load(P, a, d0, day + 1u);
        const uint32_t j = __ldg(P.app_rows + a);
        const uint32_t fl = S.flags[j];
        const int st = S.stage[j];
        if ((S.qt[j] & 0x0Fu) == 0u && st != DEABM_HOSP && st != DEABM_ICU && st != DEABM_DEAD) {
            bool hit = den_static_hit(P, j) || den_ring_eval(P, a, d0, first);
            for (uint32_t c0 = d0 + 4u; c0 <= day && !hit; c0 += 4u)
                hit = den_ring_eval(P, a, c0, den_ring_load(P, a, c0, day + 1u));
            if (P.wsg_on && !hit) {  // the Watts-Strogatz neighbours of the window's days
                const uint32_t jo = P.orig_id ? __ldg(P.orig_id + j) : j;
                const uint32_t *src_rand = P.den_bits_orig ? P.den_bits_orig : P.den_bits;
                for (uint32_t d = d0; d <= day && !hit; ++d)
                    hit = den_wsg_for(P, jo, d, [&](uint32_t v) { return bit_of(src_rand, v); });
            }
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

// app holders, drawn once per replicate column: word x of (the column's seed,
// caller id, day word 0xFFFFFFFD, stream 6); one thread per (agent, column)
__global__ void den_apps_kernel(const KParams P, StateRef S)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)P.n * P.n_rep) return;
    const uint32_t j = (uint32_t)(i / P.n_rep), b = (uint32_t)(i % P.n_rep);
    const uint32_t jo = P.orig_id ? __ldg(P.orig_id + j) : j;
    const uint32_t w = draw(seed_key(P.rep[b].seed), jo, 0xFFFFFFFDu, kStreamDen).x;
    const uint32_t fl = S.flags[i];
    S.flags[i] = (uint8_t)((uint64_t)w < P.thr_adopt ? (fl | DEABM_FL_APP) : (fl & ~DEABM_FL_APP));
}

// The in-contacts agent j (internal row; jo its caller id) received on day d
// through the day's generated networks, redrawn from Philox exactly as the day
// kernel drew them: f(0, e, caller id) for random contact e, then f(1, e, row) for
// daily occupation contact e.  Returns the counts, k_rand | k_occ << 8.
template <class F>
__device__ uint32_t den_day_contacts(const KParams &P, uint32_t j, uint32_t jo, uint32_t d, F f)
{
    const uint2 nk = seed_key(P.net_seed);
    uint32_t k_rand = 0, k_occ = 0;
    if (P.rand_on) {
        uint4 w = draw(nk, jo, d, kStreamRnet, 0u);
        const uint64_t *thr = P.rand_by_age ? P.tab->pois_age[__ldg(P.age + j)] : P.tab->pois;
        while (k_rand < DEABM_POIS_CAP && (uint64_t)w.x >= __ldg(thr + k_rand)) ++k_rand;
        const uint64_t nm1 = (uint64_t)(P.n - 1u);
        for (uint32_t e = 0; e < k_rand; ++e) {
            const uint32_t idx = e + 1u;
            if ((idx & 3u) == 0u) w = draw(nk, jo, d, kStreamRnet, idx >> 2);
            const uint32_t x = (idx & 3u) == 1u ? w.y : (idx & 3u) == 2u ? w.z : (idx & 3u) == 3u ? w.w : w.x;
            uint32_t c = (uint32_t)(((uint64_t)x * nm1) >> 32);
            c += (c >= jo) ? 1u : 0u;
            f(0u, e, c);
        }
    }
    if (P.n_occ) {
        const uint32_t g = __ldg(P.occ_gid + j);
        const uint32_t beg = __ldg(P.occ_start + g), size = __ldg(P.occ_start + g + 1u) - beg;
        k_occ = size > 1u ? (uint32_t)__ldg(P.occ_k + g) : 0u;
        const uint32_t own = j - beg;
        for (uint32_t e = 0; e < k_occ; ++e) {
            uint32_t r;
            if (P.occ_lattice) {  // as occ_ws_sum
                const uint4 w = draw(nk, jo, d, kStreamWs, e >> 1);
                const uint32_t m = (e >> 1) + 1u, hop = m < size ? m : m % size;
                const uint32_t coin = (e & 1u) ? w.z : w.x, word = (e & 1u) ? w.w : w.y;
                const uint32_t off = (e & 1u) == 0u ? hop : (hop == 0u ? 0u : size - hop);
                if (off == 0u || (uint64_t)coin < P.thr_rewire) {
                    r = occ_place(word, size - 1u, own);
                } else {
                    r = own + off;
                    r = r >= size ? r - size : r;
                }
            } else {  // as occ_sum
                const uint4 w = draw(nk, jo, d, kStreamOcc, e >> 2);
                const uint32_t x = (e & 3u) == 0u ? w.x : (e & 3u) == 1u ? w.y : (e & 3u) == 2u ? w.z : w.w;
                r = occ_place(x, size - 1u, own);
            }
            f(1u, e, beg + r);
        }
    }
    return k_rand | (k_occ << 8);
}

// One app holder's contact record of day d redrawn from Philox: the random and
// occupation contacts the day kernel drew that day (used when a context resumes
// from a saved state, whose previous days' records it never wrote).
__global__ void den_record_kernel(const KParams P, uint32_t d0, uint32_t d1)
{
    const uint32_t a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= P.n_app) return;
    const uint32_t j = __ldg(P.app_rows + a);
    const uint32_t jo = P.orig_id ? __ldg(P.orig_id + j) : j;
    const size_t plane = P.n_app;
    for (uint32_t d = d0; d < d1; ++d) {
        uint32_t *rec = P.den_ring + (size_t)(d % P.den_window) * P.den_slots * plane + a;
        rec[0] = den_day_contacts(P, j, jo, d, [&](uint32_t kind, uint32_t e, uint32_t v) {
            rec[(size_t)((kind ? kDenOccAt : 1u) + e) * plane] = v;
        });
    }
}

// ---- batched contexts (state [N][B], column b = replicate b)
// The day kernel leaves bit b % 32 of den_bits[row * W + b / 32] set (W = ceil(B /
// 32)) when the row's agent is a positive app holder of column b today.  The
// notification pass is one launch per 256 columns: eight lanes per row OR, word
// by word, the bits of all the row's in-contacts of the last den_window days --
// its stored rows (the same every day) and the random and daily occupation
// contacts of each day, redrawn from Philox (the contacts are the same in every
// column, so no record is kept) -- and then, for each column whose bit is set,
// check that column's own state (app holder, out of quarantine, not in hospital,
// ICU or dead), count the notification and draw the compliance word of the
// column's seed.  Each column reproduces the plain pass of its own run.  Bit
// lookups are whole words (32 columns at once), so a contact costs the same for
// any B <= 256.
constexpr uint32_t kDenHitWords = 8;  // words of columns one launch covers (256 columns)

// Lane g of a row's eight takes the stored in-edges g, g + 8, ... of each row and
// the days d0 + g, d0 + g + 8, ... of the window; the partial ORs are combined by
// shuffles and lane g then works through the columns of word w0 + g.
__global__ void __launch_bounds__(128) den_batch_kernel(const KParams P, uint32_t day, const uint32_t *row_of,
                                                         uint32_t W, uint32_t w0, StateRef S, Counters C,
                                                         uint32_t den_stride, uint32_t den_col0)
{
    __shared__ int s_cnt[kDenHitWords * 32];
    for (uint32_t q = threadIdx.x; q < kDenHitWords * 32u; q += blockDim.x) s_cnt[q] = 0;
    __syncthreads();
    if (__ldg(P.den_pos + day) == 0) return;  // uniform: nobody tested positive today
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x, j = t >> 3, g = t & 7u;
    const uint32_t nw = W - w0 < kDenHitWords ? W - w0 : kDenHitWords;
    uint32_t acc[kDenHitWords];
#pragma unroll
    for (uint32_t u = 0; u < kDenHitWords; ++u) acc[u] = 0u;
    auto add = [&](uint32_t row) {
        const uint32_t *src = P.den_bits + (size_t)row * W + w0;
#pragma unroll
        for (uint32_t u = 0; u < kDenHitWords; ++u)
            if (u < nw) acc[u] |= __ldg(src + u);
    };
    const uint32_t jo = j < P.n ? (P.orig_id ? __ldg(P.orig_id + j) : j) : 0u;
    if (j < P.n) {
        for (uint32_t net = 0; net < P.n_nets; ++net) {
            const uint32_t e1 = __ldg(P.row_ptr[net] + j + 1);
            for (uint32_t e = __ldg(P.row_ptr[net] + j) + g; e < e1; e += 8u) add(__ldg(P.col[net] + e));
        }
        const uint32_t d0 = day + 1u > P.den_window ? day + 1u - P.den_window : 0u;
        for (uint32_t d = d0 + g; d <= day; d += 8u) {
            (void)den_day_contacts(P, j, jo, d, [&](uint32_t kind, uint32_t, uint32_t v) {
                add(kind || !row_of ? v : __ldg(row_of + v));
            });
            if (P.wsg_on)  // the Watts-Strogatz neighbours (caller ids)
                (void)den_wsg_for(P, jo, d, [&](uint32_t v) {
                    add(row_of ? __ldg(row_of + v) : v);
                    return false;
                });
        }
    }
    // (a row's eight lanes are an aligned eighth of one warp; rows past n add nothing)
#pragma unroll
    for (uint32_t u = 0; u < kDenHitWords; ++u) {
        acc[u] |= __shfl_xor_sync(0xFFFFFFFFu, acc[u], 1);
        acc[u] |= __shfl_xor_sync(0xFFFFFFFFu, acc[u], 2);
        acc[u] |= __shfl_xor_sync(0xFFFFFFFFu, acc[u], 4);
    }
    uint32_t hit = 0;
#pragma unroll
    for (uint32_t u = 0; u < kDenHitWords; ++u)
        if (u == g) hit = acc[u];
    if (j < P.n && g < nw) {
        while (hit) {
            const uint32_t bit = __ffs(hit) - 1u;
            hit &= hit - 1u;
            const uint32_t b = (w0 + g) * 32u + bit;
            if (b >= P.n_rep) break;
            const size_t i = (size_t)j * P.n_rep + b;
            const uint32_t fl = S.flags[i];
            const int st = S.stage[i];
            if ((fl & DEABM_FL_APP) && (S.qt[i] & 0x0Fu) == 0u && st != DEABM_HOSP && st != DEABM_ICU &&
                st != DEABM_DEAD) {
                atomicAdd(&s_cnt[g * 32u + bit], 1);
                const uint32_t w = draw(seed_key(P.rep[b].seed), jo, day, kStreamDen).x;
                if ((uint64_t)w < P.thr_comp) S.flags[i] = (uint8_t)(fl | DEABM_FL_DEN);
            }
        }
    }
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < kDenHitWords * 32u; q += blockDim.x)
        if (s_cnt[q]) atomicAdd(C.den + (size_t)day * den_stride + den_col0 + w0 * 32u + q, s_cnt[q]);
}

cudaError_t launch_den_batch(const KParams &P, uint32_t day, const uint32_t *row_of, const StateRef &S,
                             const Counters &C, uint32_t den_stride, uint32_t den_col0, cudaStream_t stream)
{
    const uint32_t W = (P.n_rep + 31u) / 32u;
    const unsigned blocks = (unsigned)(((size_t)P.n * 8u + 127u) / 128u);
    for (uint32_t w0 = 0; w0 < W; w0 += kDenHitWords)
        den_batch_kernel<<<blocks, 128, 0, stream>>>(P, day, row_of, W, w0, S, C, den_stride, den_col0);
    return cudaGetLastError();
}

cudaError_t launch_den_records(const KParams &P, uint32_t d0, uint32_t d1, cudaStream_t stream)
{
    if (P.n_app == 0u || d0 >= d1) return cudaSuccess;
    den_record_kernel<<<(P.n_app + 255u) / 256u, 256, 0, stream>>>(P, d0, d1);
    return cudaGetLastError();
}

cudaError_t launch_den_apps(const KParams &P, const StateRef &S, cudaStream_t stream)
{
    const size_t m = (size_t)P.n * P.n_rep;
    den_apps_kernel<<<(unsigned)((m + 255u) / 256u), 256, 0, stream>>>(P, S);
    return cudaGetLastError();
}

cudaError_t launch_den(const KParams &P, uint32_t day, const StateRef &S, const Counters &C, cudaStream_t stream)
{
    if (P.n_app == 0u) return cudaSuccess;
    den_kernel<<<(P.n_app + 255u) / 256u, 256, 0, stream>>>(P, day, S, C);
    return cudaGetLastError();
}

}  // namespace deabm
