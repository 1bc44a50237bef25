// day_common.cuh -- per-destination infection rate of one day (Eq. 1 summed over
// a destination's interactions): CSR sums in CSR order, the day's occupation
// and random in-contacts generated from Philox, and their combination into lambda.
// Shared by the day kernels.
#pragma once
#include <cstdint>

#include "deabm_device.cuh"

namespace deabm {

// A block of the day's network words (net_seed): from the precomputed round keys
// when the parameters live in the kernel's parameter space (RK), else from the
// seed's key schedule (parameters in shared memory, where the keys would cost
// a load each).
template <bool RK = true>
__device__ __forceinline__ uint4 net_draw(const KParams &P, uint32_t agent, uint32_t day, uint32_t stream, uint32_t blk)
{
    return RK ? draw_rk(P.nrk, agent, day, stream, blk) : draw(seed_key(P.net_seed), agent, day, stream, blk);
}

// Sum of inf over one CSR row, left to right from +0.0f.  The row is taken in
// rounds of kRound edges: all column loads of a round are issued, then all
// gathers, then the adds in order, so a row of up to kRound in-edges costs two
// dependent memory round trips instead of one per edge.
#ifndef DEABM_ROUND
#define DEABM_ROUND 10
#endif
#ifndef DEABM_PLAIN_MINB
#define DEABM_PLAIN_MINB 12
#endif
#ifndef DEABM_ROUND0
#define DEABM_ROUND0 6  // round of the first stored network (households of up to 6: one round; swept 4, 6, 10)
#endif
template <uint32_t kRound = DEABM_ROUND>
__device__ __forceinline__ float csr_sum(const uint32_t *__restrict__ col, const float *__restrict__ inf, uint32_t e,
                                         uint32_t end, uint32_t stride, uint32_t b, float h = 0.0f)
{
    while (e < end) {
        uint32_t c[kRound];
        float v[kRound];
#pragma unroll
        for (uint32_t u = 0; u < kRound; ++u) c[u] = (e + u < end) ? __ldg(col + e + u) : 0u;
#pragma unroll
        for (uint32_t u = 0; u < kRound; ++u) v[u] = (e + u < end) ? __ldg(inf + (size_t)c[u] * stride + b) : 0.0f;
#pragma unroll
        for (uint32_t u = 0; u < kRound; ++u)
            if (e + u < end) h = __fadd_rn(h, v[u]);
        e += kRound;
    }
    return h;
}

// Exposure-notification record of one (day, app holder), kept for the last
// den_window days: word 0 = random count | occupation count << 8, the random
// contacts (caller ids) from word 1, the occupation contacts (internal rows)
// from word kDenOccAt.  Word e of the record at rec lives at rec[e * n_app]
// (one plane per word, app holders side by side).
constexpr uint32_t kDenOccAt = 16;

// Random in-contacts of agent j (the caller's id) on `day`: count from word 0 of
// block 0, contact e from word e+1 (block (e+1)/4, lane (e+1)%4); v uniform on
// the other n-1 agents.  `inf` is indexed by the caller's ids, or (ROWMAP) by
// internal rows through row_of.  REC: also write the contacts to
// rec[1..] when rec is not null.
#ifndef DEABM_RAND_DEFER
#define DEABM_RAND_DEFER 0  // 1: block 0's gathers are added only after the stored networks' sums (more
                            // spills at 40 registers; measured 2 % slower at N = 2e6)
#endif

// The random contacts of block 0 (count word, then contacts 0..2), their
// gathers issued but not yet added.
struct RandHead {
    uint32_t k;
    float v[3];
};

// Block 0 of agent j's random network on `day` (caller id) and the day's
// in-contact count it fixes: K_j = the number of Poisson thresholds (of j's age
// bin's mean when the means are age-stratified) at or below word 0, at most
// DEABM_POIS_CAP.
struct RandBlock0 {
    uint4 w;
    uint32_t k;
};

template <bool RK = true>
__device__ __forceinline__ RandBlock0 random_block0(const KParams &P, uint32_t j, uint32_t day, int age)
{
    RandBlock0 r;
    r.w = net_draw<RK>(P, j, day, kStreamRnet, 0u);
    r.k = poisson_count(P, r.w.x, age);
    return r;
}

template <bool REC, bool ROWMAP>
__device__ __forceinline__ RandHead random_head(const KParams &P, const float *__restrict__ inf, uint32_t j,
                                                const RandBlock0 &r0, uint32_t stride, uint32_t b, uint32_t *rec,
                                                const uint32_t *row_of)
{
    const uint4 w = r0.w;
    RandHead h;
    h.k = r0.k;
    const uint64_t nm1 = (uint64_t)(P.n - 1u);
    const uint32_t x[3] = {w.y, w.z, w.w};
#pragma unroll
    for (uint32_t u = 0; u < 3u; ++u) {
        uint32_t c = (uint32_t)(((uint64_t)x[u] * nm1) >> 32);
        c += (c >= j) ? 1u : 0u;
        if (REC && rec && u < h.k) rec[(size_t)(1u + u) * P.n_app] = c;
        h.v[u] = u < h.k ? __ldg(inf + (size_t)(ROWMAP ? __ldg(row_of + c) : c) * stride + b) : 0.0f;
    }
    return h;
}

// The sum over all k random contacts in draw order: block 0's values from the
// head, then four contacts per further block, each block's gathers together.
template <bool REC, bool ROWMAP, bool RK = true>
__device__ __forceinline__ float random_tail(const KParams &P, const float *__restrict__ inf, uint32_t j,
                                             uint32_t day, uint32_t stride, uint32_t b, const RandHead &h,
                                             uint32_t *rec, const uint32_t *row_of)
{
    float r = 0.0f;
#pragma unroll
    for (uint32_t u = 0; u < 3u; ++u)
        if (u < h.k) r = __fadd_rn(r, h.v[u]);
    const uint64_t nm1 = (uint64_t)(P.n - 1u);
    for (uint32_t e = 3u; e < h.k; e += 4u) {
        const uint4 w = net_draw<RK>(P, j, day, kStreamRnet, (e + 1u) >> 2);
        const uint32_t x[4] = {w.x, w.y, w.z, w.w};
        float v[4];
#pragma unroll
        for (uint32_t u = 0; u < 4u; ++u) {
            uint32_t c = (uint32_t)(((uint64_t)x[u] * nm1) >> 32);
            c += (c >= j) ? 1u : 0u;
            if (REC && rec && e + u < h.k) rec[(size_t)(1u + e + u) * P.n_app] = c;
            v[u] = e + u < h.k ? __ldg(inf + (size_t)(ROWMAP ? __ldg(row_of + c) : c) * stride + b) : 0.0f;
        }
#pragma unroll
        for (uint32_t u = 0; u < 4u; ++u)
            if (e + u < h.k) r = __fadd_rn(r, v[u]);
    }
    return r;
}

// Far end of edge m (1-based) of agent i in the day's Watts-Strogatz random
// network, from its block of stream 10: the lattice neighbour (i + m) mod n, or,
// when rewired (coin below the threshold, or i + m wrapping onto i), the agent
// the word picks among the other n - 1.
__device__ __forceinline__ uint32_t wsg_far(const KParams &P, uint32_t i, uint32_t m, uint32_t coin, uint32_t word)
{
    const uint32_t n = P.n;
    if (m % n == 0u || (uint64_t)coin < P.thr_wsg) {
        uint32_t v = (uint32_t)(((uint64_t)word * (uint64_t)(n - 1u)) >> 32);
        return v + ((v >= i) ? 1u : 0u);
    }
    return (uint32_t)(((uint64_t)i + m) % n);
}

// Agent jo's (caller id) messages in the day's Watts-Strogatz random network,
// summed left to right from +0.0f: its own edges m = 1..h, the unrewired lattice
// edges of agents jo - m, m = 1..h, then the rewired edges that landed on jo, by
// owner ascending.  *k_out = their number.  NEED_SUM = false: the count only.
// Agent c's infectiousness is inf[c * stride + b], or (ROWMAP) inf[row_of[c] *
// stride + b] when the panel is in internal row order.
template <bool NEED_SUM = true, bool RK = true, bool ROWMAP = false>
__device__ __forceinline__ float wsg_sum(const KParams &P, const float *__restrict__ inf, uint32_t jo, uint32_t day,
                                         uint32_t *k_out, uint32_t stride = 1u, uint32_t b = 0u,
                                         const uint32_t *row_of = nullptr)
{
    auto val = [&](uint32_t c) { return __ldg(inf + (size_t)(ROWMAP ? __ldg(row_of + c) : c) * stride + b); };
    const uint32_t n = P.n, h = P.wsg_h;
    float r = 0.0f;
    uint32_t k = h;
    if (NEED_SUM) {
        for (uint32_t m = 1; m <= h; m += 2u) {
            const uint4 w = net_draw<RK>(P, jo, day, kStreamWsg, (m - 1u) >> 1);
            const uint32_t f0 = wsg_far(P, jo, m, w.x, w.y);
            const float v0 = val(f0);
            float v1 = 0.0f;
            if (m + 1u <= h) v1 = val(wsg_far(P, jo, m + 1u, w.z, w.w));
            r = __fadd_rn(r, v0);
            if (m + 1u <= h) r = __fadd_rn(r, v1);
        }
    }
    for (uint32_t m = 1; m <= h; ++m) {
        const uint32_t i = (uint32_t)(((uint64_t)jo + (uint64_t)n - (uint64_t)(m % n)) % n);
        if (!((__ldg(P.wsg_rew + i) >> (m - 1u)) & 1u)) {
            ++k;
            if (NEED_SUM) r = __fadd_rn(r, val(i));
        }
    }
    const uint32_t s0 = __ldg(P.wsg_start + jo), s1 = __ldg(P.wsg_start + jo + 1u);
    k += s1 - s0;
    if (NEED_SUM)
        for (uint32_t q = s0; q < s1; ++q) r = __fadd_rn(r, val(__ldg(P.wsg_land + q)));
    *k_out = k;
    return r;
}

// Place of the member an occupation contact lands on: word x mapped to
// [0, size-1), the agent's own place skipped.
__device__ __forceinline__ uint32_t occ_place(uint32_t x, uint32_t size_m1, uint32_t own)
{
    uint32_t r = (uint32_t)(((uint64_t)x * size_m1) >> 32);
    return r + ((r >= own) ? 1u : 0u);
}

// The day's occupation in-contacts of internal row j (caller id jo): occ_k[g]
// of them (none for a lone member), contact e from word e of stream 4 (block
// e/4, lane e%4).  Taken four at a time: one Philox block gives four rows whose
// gathers are issued together, then added in draw order from +0.0f.
// Watts-Strogatz variant: the member at place `own` of a ring of `size`
// receives in-edge e from the lattice place own + (e/2+1) (e even) or
// own - (e/2+1) (e odd), unless the edge is rewired (coin below the threshold,
// or a lattice offset that is a multiple of the size): then from a uniform
// other member.  Two contacts per Philox block.
template <bool REC = false, bool RK = true>
__device__ __forceinline__ float occ_ws_sum(const KParams &P, const float *__restrict__ inf, uint32_t jo, uint32_t day,
                                            uint32_t stride, uint32_t b, uint32_t beg, uint32_t size, uint32_t own,
                                            uint32_t k, uint32_t *rec)
{
    float h = 0.0f;
    for (uint32_t e = 0; e < k; e += 2u) {
        const uint4 w = net_draw<RK>(P, jo, day, kStreamWs, e >> 1);
        const uint32_t m = (e >> 1) + 1u;
        const uint32_t hop = m < size ? m : m % size;
        const uint32_t coin[2] = {w.x, w.z}, word[2] = {w.y, w.w};
        float v[2];
#pragma unroll
        for (uint32_t u = 0; u < 2u; ++u) {
            const uint32_t off = u == 0u ? hop : (hop == 0u ? 0u : size - hop);
            uint32_t r;
            if (off == 0u || (uint64_t)coin[u] < P.thr_rewire) {
                r = occ_place(word[u], size - 1u, own);
            } else {
                r = own + off;
                r = r >= size ? r - size : r;
            }
            if (REC && rec && e + u < k) rec[(size_t)(kDenOccAt + e + u) * P.n_app] = beg + r;
            v[u] = (e + u < k) ? __ldg(inf + (size_t)(beg + r) * stride + b) : 0.0f;
        }
        h = __fadd_rn(h, v[0]);
        if (e + 1u < k) h = __fadd_rn(h, v[1]);
    }
    return h;
}

template <bool REC = false, bool RK = true>
__device__ __forceinline__ float occ_sum(const KParams &P, const float *__restrict__ inf, uint32_t j, uint32_t jo,
                                         uint32_t day, uint32_t stride, uint32_t b, uint32_t *k_out,
                                         uint32_t *rec = nullptr)
{
    const uint32_t g = __ldg(P.occ_gid + j);
    const uint32_t beg = __ldg(P.occ_start + g), size = __ldg(P.occ_start + g + 1u) - beg;
    const uint32_t k = size > 1u ? (uint32_t)__ldg(P.occ_k + g) : 0u;
    const uint32_t own = j - beg;
    *k_out = k;
    if (P.occ_lattice) return occ_ws_sum<REC, RK>(P, inf, jo, day, stride, b, beg, size, own, k, rec);
    float h = 0.0f;
    for (uint32_t e = 0; e < k; e += 4u) {
        const uint4 w = net_draw<RK>(P, jo, day, kStreamOcc, e >> 2);
        const uint32_t x[4] = {w.x, w.y, w.z, w.w};
        float v[4];
#pragma unroll
        for (uint32_t u = 0; u < 4u; ++u) {
            const uint32_t row = beg + occ_place(x[u], size - 1u, own);
            if (REC && rec && e + u < k) rec[(size_t)(kDenOccAt + e + u) * P.n_app] = row;
            v[u] = (e + u < k) ? __ldg(inf + (size_t)row * stride + b) : 0.0f;
        }
#pragma unroll
        for (uint32_t u = 0; u < 4u; ++u)
            if (e + u < k) h = __fadd_rn(h, v[u]);
    }
    *k_out = k;
    return h;
}

// The number of the day's in-contacts of an agent whose lambda is not needed
// (not susceptible): the random network's count (k_rand, from block 0) and the
// occupation's daily count.  No gathers.
template <bool WSG = false, bool RK = true>
__device__ __forceinline__ uint32_t contact_count(const KParams &P, uint32_t j, uint32_t k_rand, uint32_t jo,
                                                  uint32_t day)
{
    uint32_t k = k_rand;
    if (WSG && P.wsg_on) {
        uint32_t kw;
        (void)wsg_sum<false, RK>(P, nullptr, jo, day, &kw);
        k += kw;
    }
    if (P.n_occ) {
        const uint32_t g = __ldg(P.occ_gid + j);
        if (__ldg(P.occ_start + g + 1u) - __ldg(P.occ_start + g) > 1u) k += __ldg(P.occ_k + g);
    }
    return k;
}

// Row bounds of agent j (internal row) in every stored network.
struct RowBounds {
    uint32_t beg[DEABM_MAX_NETS], end[DEABM_MAX_NETS];
};

__device__ __forceinline__ RowBounds row_bounds(const KParams &P, uint32_t j)
{
    RowBounds rb;
#pragma unroll
    for (uint32_t net = 0; net < DEABM_MAX_NETS; ++net) {
        rb.beg[net] = net < P.n_nets ? __ldg(P.row_ptr[net] + j) : 0u;
        rb.end[net] = net < P.n_nets ? __ldg(P.row_ptr[net] + j + 1) : 0u;
    }
    return rb;
}

// lambda_j of one (agent, replicate) from the state of the day; j = internal row,
// jo = the caller's id of the same agent; rb = its row bounds, r0 = block 0 of
// its random network (unused when the random network is off).  OCC = false
// compiles the daily occupation networks out (for contexts that have none).
// Callers load the row bounds and draw block 0 first, so that the bounds are in
// flight while the Philox rounds run.  REC: the agent's exposure-notification
// record of the day goes to rec (when not null).
template <bool OCC = true, bool REC = false, bool ROWMAP = false, bool WSG = false, bool RK = true>
__device__ __forceinline__ float lambda_at(const KParams &P, const Rep &rp, const InfBuffers &I, uint32_t j, uint32_t jo,
                                           uint32_t day, uint32_t stride, uint32_t b, int age, const RowBounds &rb,
                                           const RandBlock0 &r0, uint32_t *k_out, uint32_t *rec = nullptr)
{
    *k_out = 0;
    const bool rmap = ROWMAP && I.row_of != nullptr;
    const float *rinf = rmap ? I.cur : I.rand_cur;
    RandHead head{0u, {0.0f, 0.0f, 0.0f}};
#if !DEABM_RAND_DEFER
    float r_now = 0.0f;
#endif
    if (P.rand_on) {  // block 0's gathers go out now and are added after the stored networks
        head = rmap ? random_head<REC, true>(P, rinf, jo, r0, stride, b, rec, I.row_of)
                    : random_head<REC, false>(P, rinf, jo, r0, stride, b, rec, nullptr);
#if !DEABM_RAND_DEFER
        r_now = rmap ? random_tail<REC, true, RK>(P, rinf, jo, day, stride, b, head, rec, I.row_of)
                     : random_tail<REC, false, RK>(P, rinf, jo, day, stride, b, head, rec, nullptr);
#endif
    }
    const uint32_t k_rand = head.k;
    *k_out = k_rand;
    uint32_t k_occ = 0;
    float s = 0.0f;
#pragma unroll
    for (uint32_t net = 0; net < DEABM_MAX_NETS; ++net) {
        if (net < P.n_nets) {
            const float h = net == 0 ? csr_sum<DEABM_ROUND0>(P.col[net], I.cur, rb.beg[net], rb.end[net], stride, b)
                                     : csr_sum<DEABM_ROUND>(P.col[net], I.cur, rb.beg[net], rb.end[net], stride, b);
            const float term = __fmul_rn(rp.B_net[net], h);
            s = net == 0 ? term : __fadd_rn(s, term);
        }
    }
    if (OCC && P.n_occ) {
        const float term = __fmul_rn(rp.B_net[P.n_nets], occ_sum<REC, RK>(P, I.cur, j, jo, day, stride, b, &k_occ, rec));
        s = P.n_nets == 0 ? term : __fadd_rn(s, term);
        *k_out += k_occ;
    }
    if (REC && rec) rec[0] = k_rand | (k_occ << 8);
    if (WSG && P.wsg_on) {  // the Watts-Strogatz random network in the random network's place
        uint32_t kw;
        const float w = rmap ? wsg_sum<true, RK, true>(P, rinf, jo, day, &kw, stride, b, I.row_of)
                             : wsg_sum<true, RK, false>(P, rinf, jo, day, &kw, stride, b, nullptr);
        const float term = __fmul_rn(rp.B_rand, w);
        s = (P.n_nets == 0 && (!OCC || P.n_occ == 0)) ? term : __fadd_rn(s, term);
        *k_out += kw;
    }
    if (P.rand_on) {
#if DEABM_RAND_DEFER
        const float r = rmap ? random_tail<REC, true, RK>(P, rinf, jo, day, stride, b, head, rec, I.row_of)
                             : random_tail<REC, false, RK>(P, rinf, jo, day, stride, b, head, rec, nullptr);
#else
        const float r = r_now;
#endif
        const float term = __fmul_rn(rp.B_rand, r);
        s = (P.n_nets == 0 && (!OCC || P.n_occ == 0)) ? term : __fadd_rn(s, term);
    }
    return __fmul_rn(__fmul_rn(rp.cR, rp.S_age[age]), s);
}

// lambda_j with its own bounds and block 0 (see lambda_at).
template <bool OCC = true, bool REC = false, bool ROWMAP = false, bool WSG = false, bool RK = true>
__device__ __forceinline__ float lambda_of(const KParams &P, const Rep &rp, const InfBuffers &I, uint32_t j, uint32_t jo,
                                           uint32_t day, uint32_t stride, uint32_t b, int age, uint32_t *k_out,
                                           uint32_t *rec = nullptr)
{
    const RowBounds rb = row_bounds(P, j);
    RandBlock0 r0{make_uint4(0u, 0u, 0u, 0u), 0u};
    if (P.rand_on) r0 = random_block0<RK>(P, jo, day, age);
    return lambda_at<OCC, REC, ROWMAP, WSG, RK>(P, rp, I, j, jo, day, stride, b, age, rb, r0, k_out, rec);
}

}  // namespace deabm
