// step_kernels.cu -- one simulated day of DeepABM-COVID on the GPU.
//
// A day (Sec. 3 "Infection Transmission", Eq. 1-2) is one kernel launch:
//   for every destination agent j (and replicate b in batched runs)
//     H_{n,j}  = sum of inf_src over the CSR in-edges of j in static network n,
//                in CSR order (left to right from +0.0f, no FMA contraction)
//     O_j      = sum of inf_src over the day's occupation in-contacts of j
//                (optional), generated here from Philox (never stored)
//     Rn_j     = sum of inf_src over the K_j ~ Poisson random in-contacts of
//                the day, generated here from Philox (never stored)
//     lambda_j = (R/I * S_{age_j}) * (B_0 H_0 + B_1 H_1 + ... + B_o O_j + B_r Rn_j)
//     p_j      = 1 - exp(-lambda_j dt), infected iff susceptible and u_j < p_j
//   then the agent's stage/timer machine and interventions, the agent's emitted
//   infectiousness for the next day (written to the other half of a double
//   buffer), and the day's counters (block-aggregated atomics).
// The emitted-infectiousness vector of the day being read (4 B per agent per
// replicate) stays L2-resident; the CSR column stream is the HBM traffic.
#include <cuda_runtime.h>
#include <cstdint>

#include "day_common.cuh"
#include "deabm_device.cuh"
#include "kernels.h"

namespace deabm {

// fl32(1 - exp(-x)) correctly rounded: the decision u < p uses this value.
// expm1f (<= 2 ulp) decides every draw whose u is more than 2^-21 away from
// p; the rest take the FP64 value rounded once to FP32.
__device__ __forceinline__ bool infection_decision(float lam_dt, float u, float *p_out)
{
    const float p = -expm1f(-lam_dt);
    if (fabsf(u - p) > 4.76837158203125e-07f) {  // 2^-21
        *p_out = p;
        return u < p;
    }
    const float pe = (float)(-expm1(-(double)lam_dt));
    *p_out = pe;
    return u < pe;
}

#ifndef DEABM_QUIET_S
#define DEABM_QUIET_S 0  // 1: a susceptible agent with nothing happening today writes nothing (measured at
                         // N = 2e6, days 5..24: 12 MB less DRAM written a day but 1 % slower, 90.2 against
                         // 89.1 us a day)
#endif
#ifndef DEABM_SUSCEPTIBLE_ONLY
#define DEABM_SUSCEPTIBLE_ONLY 1  // 0: lambda (all gathers) for every agent, as the method is written
#endif

// Full day for one (agent j, replicate b) at flat index i = j*stride + b.  Every
// random draw is keyed by the caller's agent id jo, so relabelling the agents
// inside the library changes no result.
// DEN: exposure notification on (plain contexts): an app holder records the day's
// contacts, a positive app holder is marked for the notification pass.  POS:
// only the mark (*notify), for the batched notification pass.
template <bool OCC = true, bool DEN = false, bool ROWMAP = false, bool WSG = false, bool RK = false, bool POS = false>
__device__ __forceinline__ void agent_day(const KParams &P, const Rep &rp, uint32_t day, const InfBuffers &I,
                                          const StateRef &S, uint32_t j, uint32_t stride, uint32_t b, float *lam_out,
                                          float *p_out, int *new_stage, bool *infected, uint32_t *k_out,
                                          uint32_t *kg_out, bool *notify = nullptr)
{
    const size_t i = (size_t)j * stride + b;
    const uint32_t jo = P.orig_id ? __ldg(P.orig_id + j) : j;
    const int age = __ldg(P.age + j);
    uint32_t *rec = nullptr;
    if (DEN && (S.flags[i] & DEABM_FL_APP))
        rec = P.den_ring + (size_t)(day % P.den_window) * P.den_slots * P.n_app + __ldg(P.app_rank + j);
    AgentState a;
    a.st = S.stage[i];
    // Eq. 2 applies to susceptible agents only: the others skip the gathers (their
    // in-contacts are still counted), unless lambda is kept for every agent.  With
    // exposure notification every agent takes the full path: the app holders
    // record their contacts anyway, and one path for all measured faster than the
    // divergent pair there.
    // Block 0 of the random network is drawn once, before the two paths part,
    // so that a warp holding both kinds of agent runs its Philox rounds once.
    const bool full = !DEABM_SUSCEPTIBLE_ONLY || DEN || a.st == DEABM_S || lam_out != nullptr;
    RowBounds rb = {};
    if (full) rb = row_bounds(P, j);
    RandBlock0 r0{make_uint4(0u, 0u, 0u, 0u), 0u};
    if (P.rand_on) r0 = random_block0<RK>(P, jo, day, age);
    float lam = 0.0f;
    if (full) {
        lam = lambda_at<OCC, DEN, ROWMAP, WSG, RK>(P, rp, I, j, jo, day, stride, b, age, rb, r0, k_out, rec);
        uint32_t deg = 0;
#pragma unroll
        for (uint32_t net = 0; net < DEABM_MAX_NETS; ++net) deg += rb.end[net] - rb.beg[net];
        *kg_out = *k_out + deg;
    } else {
        *k_out = contact_count<WSG, RK>(P, j, r0.k, jo, day);
        *kg_out = 0;
    }
    a.tm = S.timer[i];
    a.ti = S.tinf[i];
    a.fl = S.flags[i];
    const uint32_t q = S.qt[i];
    a.qd = q & 0x0Fu;
    a.cd = (q >> 4) & 0x07u;
    if (S.vd1) {
        a.vd1 = S.vd1[i];
        a.vd2 = S.vd2[i];
    }
    const uint2 key = seed_key(rp.seed);
    bool inf_now = false;
    uint32_t inf_y = 0;
    float p = 0.0f;
    // the draw is needed by a susceptible agent with lambda > 0 (p = 0 never infects)
    // and by a quarantined agent (its dropout word); skipping it elsewhere lets
    // whole warps skip the Philox rounds
    const float lam_dt = __fmul_rn(lam, P.dt);
    if ((a.st == DEABM_S && lam_dt > 0.0f) || a.qd > 0u || lam_out != nullptr) {
        const uint4 w = RK ? draw_rk(rp.rk, jo, day, kStreamInf) : draw(key, jo, day, kStreamInf);
        inf_y = w.y;
        const bool hit = infection_decision(lam_dt, unit_float(w.x), &p);
        inf_now = (a.st == DEABM_S) && hit;
    }
    const int16_t d1 = P.vax_on ? __ldg(P.dose1_day + j) : kNever;
#if DEABM_QUIET_S
    // A susceptible agent that is not infected today and has nothing pending (no
    // quarantine, no test result, no notification, no dose or vaccine onset of the
    // static schedule today) keeps its state word for word and emits nothing, so
    // neither its state nor its infectiousness is written: the buffer being
    // written already holds its 0 of two days ago (S is only ever left, and both
    // buffers are cleared whenever a state is installed).
    bool quiet = !DEN && a.st == DEABM_S && !inf_now && a.qd == 0u && a.cd == 0u && !(a.fl & DEABM_FL_DEN);
    if (quiet && P.vax_on) {
        if (P.vax_strategy != 0) {
            quiet = false;
        } else if (d1 != kNever) {
            const int32_t t = (int32_t)day, D1 = d1, D2 = D1 + (int32_t)rp.dose2_delay, on = (int32_t)P.vax_onset;
            quiet = t != D1 && t != D2 && t != D1 + on && t != D2 + on;
        }
    }
    if (quiet) {
        if (lam_out) {
            lam_out[i] = lam;
            p_out[i] = p;
        }
        *new_stage = DEABM_S;
        *infected = false;
        return;
    }
#endif
    advance<RK>(P, rp, key, jo, day, age, d1, inf_now, a, inf_y, (size_t)jo * stride + b);
    if (DEN || POS) {  // a positive app holder notifies its contacts after the day
        const bool v = a.pos_result && (a.fl & DEABM_FL_APP);
        *notify = v;
        if (DEN && v && P.den_bits_orig) atomicOr(P.den_bits_orig + (jo >> 5), 1u << (jo & 31u));
    }
    S.stage[i] = (int8_t)a.st;
    S.timer[i] = (int16_t)a.tm;
    S.tinf[i] = (int16_t)a.ti;
    S.flags[i] = (uint8_t)a.fl;
    S.qt[i] = (uint8_t)((a.qd & 0x0Fu) | ((a.cd & 0x07u) << 4));
    if (S.vd1) {
        S.vd1[i] = (int16_t)a.vd1;
        S.vd2[i] = (int16_t)a.vd2;
    }
    const float v = emitted(P.tab, P.inf_len, a.st, a.ti, a.qd);
    I.next[i] = v;
    if (I.rand_next) I.rand_next[(size_t)jo * stride + b] = v;
    if (lam_out) {
        lam_out[i] = lam;
        p_out[i] = p;
    }
    *new_stage = a.st;
    *infected = inf_now;
}

// block-level aggregation of the day's counters; every thread of the block calls it
#ifndef DEABM_HIST_MATCH
#define DEABM_HIST_MATCH 0  // 1: warp-aggregated (match.any) stage counts; 2: warp-reduced packed counts;
                            // 0: one shared atomic per agent
#endif
__device__ __forceinline__ void count_day(bool active, int st, bool infected, uint32_t k, uint32_t kg, int *s_hist,
                                          int *s_new, unsigned long long *s_msgs, unsigned long long *s_gath)
{
    const unsigned full = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
#if DEABM_HIST_MATCH == 1
    const unsigned act = __ballot_sync(full, active);
    if (active) {
        const unsigned m = __match_any_sync(act, st);
        if (lane == __ffs(m) - 1) atomicAdd(&s_hist[st], __popc(m));
    }
#elif DEABM_HIST_MATCH == 2
    // the warp's 11 stage counts (each <= 32) packed 6 bits apiece into three
    // words, summed by three warp reductions; lane s adds stage s's count
    const uint32_t one = active ? 1u : 0u;
    const uint32_t r0 = __reduce_add_sync(full, st < 5 ? one << (6 * st) : 0u);
    const uint32_t r1 = __reduce_add_sync(full, (st >= 5 && st < 10) ? one << (6 * (st - 5)) : 0u);
    const uint32_t r2 = __reduce_add_sync(full, st == 10 ? one : 0u);
    if (lane < DEABM_N_STAGE) {
        const uint32_t word = lane < 5 ? r0 : lane < 10 ? r1 : r2;
        const int c = (int)((word >> (6 * (lane % 5))) & 63u);
        if (c) atomicAdd(&s_hist[lane], c);
    }
#else
    if (active) atomicAdd(&s_hist[st], 1);
#endif
    const unsigned nb = __ballot_sync(full, infected);
    if (lane == 0 && nb) atomicAdd(s_new, __popc(nb));
    const unsigned ks = __reduce_add_sync(full, active ? k : 0u);
    if (lane == 0 && ks) atomicAdd(s_msgs, (unsigned long long)ks);
    const unsigned kgs = __reduce_add_sync(full, active ? kg : 0u);
    if (lane == 0 && kgs) atomicAdd(s_gath, (unsigned long long)kgs);
}

#ifndef DEABM_PLAIN_BLOCK
#define DEABM_PLAIN_BLOCK 128
#endif
#ifndef DEABM_OCC_MINB
#define DEABM_OCC_MINB 10  // resident blocks per SM asked of the daily-occupation variant (swept: 8, 10, 12)
#endif
template <bool KEEP, bool OCC, bool DEN, bool WSG>
__global__ void __launch_bounds__(DEABM_PLAIN_BLOCK, OCC ? DEABM_OCC_MINB : DEABM_PLAIN_MINB) step_plain_kernel(const KParams P, uint32_t day, const InfBuffers I, StateRef S,
                                                         Counters C, float *lam_out, float *p_out)
{
    __shared__ int s_hist[DEABM_N_STAGE];
    __shared__ int s_new;
    __shared__ unsigned long long s_msgs, s_gath;
#ifndef DEABM_REP_SMEM
#define DEABM_REP_SMEM 0  // 1: stage the replicate parameters in shared memory once per block
#endif
#if DEABM_REP_SMEM
    __shared__ Rep s_rep;
    for (uint32_t q = threadIdx.x; q < sizeof(Rep) / 4; q += blockDim.x)
        ((uint32_t *)&s_rep)[q] = ((const uint32_t *)P.rep)[q];
#endif
    if (threadIdx.x < DEABM_N_STAGE) s_hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) { s_new = 0; s_msgs = 0ull; s_gath = 0ull; }
    __syncthreads();
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = j < P.n;
    int st = 0;
    bool infected = false, notify = false;
    uint32_t k = 0, kg = 0;
    if (active) {
#ifndef DEABM_REP_PARAM
#define DEABM_REP_PARAM 1  // 1: replicate 0 from the kernel's parameter space; 0: through the rep pointer
#endif
#if DEABM_REP_SMEM
        const Rep &rp = s_rep;
#elif DEABM_REP_PARAM
        const Rep &rp = P.rep0;
#else
        const Rep &rp = P.rep[0];
#endif
        agent_day<OCC, DEN, false, WSG, DEABM_REP_PARAM != 0>(P, rp, day, I, S, j, 1u, 0u, KEEP ? lam_out : nullptr,
                                                             p_out, &st, &infected, &k, &kg, &notify);
    }
    if (DEN) {  // the day's positive app holders as a bit map over rows: one word per warp
        const unsigned bits = __ballot_sync(0xFFFFFFFFu, notify);
        if ((threadIdx.x & 31u) == 0u && j < P.n) {
            P.den_bits[j >> 5] = bits;
            if (bits) atomicAdd(P.den_pos + day, __popc(bits));
        }
    }
    count_day(active, st, infected, k, kg, s_hist, &s_new, &s_msgs, &s_gath);
    __syncthreads();
    if (threadIdx.x < DEABM_N_STAGE && s_hist[threadIdx.x])
        atomicAdd(&C.hist[(size_t)day * DEABM_N_STAGE + threadIdx.x], s_hist[threadIdx.x]);
    if (threadIdx.x == 0) {
        if (s_new) atomicAdd(&C.new_inf[day], s_new);
        if (s_msgs) atomicAdd(&C.msgs[day], s_msgs);
        if (s_gath) atomicAdd(&C.gath[day], s_gath);
    }
}

// Batched panel: block (32 x 8) covers 8 agents x 32 replicates; lane = replicate.
// The 32 lanes of a warp read the same CSR entries (one broadcast load) and
// gather one contiguous 128 B run of the [N][B] infectiousness panel per edge.
// DEN: the warp's positive app holders go to word blockIdx.y of the row's
// ceil(B/32) words in den_bits (one ballot; every word is written every day).
template <bool KEEP, bool WSG, bool DEN = false>
__global__ void __launch_bounds__(256) step_batch_kernel(const KParams P, uint32_t day, const InfBuffers I, StateRef S,
                                                         Counters C, float *lam_out, float *p_out)
{
    // per (stage or new-infection, replicate lane) counts of the block's 8 agent rows
    __shared__ int s_cnt[DEABM_N_STAGE + 1][32];
    __shared__ unsigned long long s_msgs;
    const uint32_t lane = threadIdx.x, wy = threadIdx.y, tid = wy * 32u + lane;
    const uint32_t j = blockIdx.x * 8u + wy;
    const uint32_t b = blockIdx.y * 32u + lane;
    for (uint32_t q = tid; q < (DEABM_N_STAGE + 1) * 32u; q += 256u) (&s_cnt[0][0])[q] = 0;
    if (tid == 0) s_msgs = 0ull;
    __syncthreads();
    const bool active = (j < P.n) && (b < P.n_rep);
    int st = 0;
    bool infected = false, notify = false;
    uint32_t k = 0;
    if (active) {
        const Rep &rp = P.rep[b];
        uint32_t kg;
        agent_day<true, false, true, WSG, false, DEN>(P, rp, day, I, S, j, P.n_rep, b, KEEP ? lam_out : nullptr, p_out,
                                                      &st, &infected, &k, &kg, &notify);
        atomicAdd(&s_cnt[st][lane], 1);
        if (infected) atomicAdd(&s_cnt[DEABM_N_STAGE][lane], 1);
    }
    if (DEN) {
        const unsigned bits = __ballot_sync(0xFFFFFFFFu, notify);
        if (lane == 0 && j < P.n) {
            P.den_bits[(size_t)j * gridDim.y + blockIdx.y] = bits;
            if (bits) atomicAdd(P.den_pos + day, __popc(bits));
        }
    }
    // messages are counted once per agent row (lane 0 of the first replicate panel)
    if (lane == 0 && blockIdx.y == 0 && j < P.n && k) atomicAdd(&s_msgs, (unsigned long long)k);
    __syncthreads();
    for (uint32_t q = tid; q < (DEABM_N_STAGE + 1) * 32u; q += 256u) {
        const uint32_t s = q / 32u, l = q % 32u, bb = blockIdx.y * 32u + l;
        const int v = s_cnt[s][l];
        if (v && bb < P.n_rep) {
            if (s < DEABM_N_STAGE) atomicAdd(&C.hist[((size_t)day * P.n_rep + bb) * DEABM_N_STAGE + s], v);
            else atomicAdd(&C.new_inf[(size_t)day * P.n_rep + bb], v);
        }
    }
    if (tid == 0 && s_msgs) atomicAdd(&C.msgs[day], s_msgs);
}

// Ragged batch of independent populations in one launch (OCC: some population
// draws its occupation contacts daily): CTAs stay resident and
// pull tiles (rows of one population) from the day's atomic queue until none is
// left, so populations of 10^4 and 10^6 agents share the GPU without one
// launch each.  Every row runs the plain day on its population's local ids,
// giving exactly the single-population result.
// 6 blocks per SM asked (swept at 64 populations, autotuned tiling: no minimum
// 0.533 ms a day at 64 registers, 6 blocks 0.472, 8 blocks 0.480)
template <bool OCC, bool WSG, bool VAX, bool DEN>
__global__ void __launch_bounds__(256, 6) step_ragged_kernel(const PopDesc *__restrict__ pops, const Tile *__restrict__ tiles,
                                                          uint32_t n_tiles, uint32_t *queue, uint32_t day,
                                                          const float *inf_cur, float *inf_next, StateRef S,
                                                          Counters C, uint32_t n_pops)
{
    __shared__ PopDesc sp;
    __shared__ uint32_t s_tile;
    __shared__ int s_hist[DEABM_N_STAGE];
    __shared__ int s_new;
    __shared__ unsigned long long s_msgs, s_gath;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(queue + day, 1u);
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= n_tiles) break;
        const Tile tl = tiles[t];
        {
            const uint32_t *src = (const uint32_t *)(pops + tl.pop);
            uint32_t *dst = (uint32_t *)&sp;
            for (uint32_t q = threadIdx.x; q < sizeof(PopDesc) / 4; q += blockDim.x) dst[q] = src[q];
        }
        if (threadIdx.x < DEABM_N_STAGE) s_hist[threadIdx.x] = 0;
        if (threadIdx.x == 0) { s_new = 0; s_msgs = 0ull; s_gath = 0ull; }
        __syncthreads();
        InfBuffers I;
        I.cur = inf_cur + sp.base;
        I.next = inf_next + sp.base;
        I.rand_cur = I.cur;
        I.rand_next = nullptr;
        I.row_of = sp.row_of;  // random contacts (caller ids) reach rows through the map
        StateRef Sp;
        Sp.stage = S.stage + sp.base;
        Sp.timer = S.timer + sp.base;
        Sp.tinf = S.tinf + sp.base;
        Sp.flags = S.flags + sp.base;
        Sp.qt = S.qt + sp.base;
        Sp.vd1 = VAX ? S.vd1 + sp.base : nullptr;  // dose days (some population under a priority strategy)
        Sp.vd2 = VAX ? S.vd2 + sp.base : nullptr;
        for (uint32_t r0 = tl.begin; r0 < tl.end; r0 += blockDim.x) {
            const uint32_t j = r0 + threadIdx.x;
            const bool active = j < tl.end;
            int st = 0;
            bool infected = false, notify = false;
            uint32_t k = 0, kg = 0;
            if (active)
                // the population's parameters are in shared memory: keys from the seeds (RK = false)
                agent_day<OCC, false, true, WSG, false, DEN>(sp.kp, sp.rep, day, I, Sp, j, 1u, 0u, nullptr, nullptr,
                                                             &st, &infected, &k, &kg, &notify);
            if (DEN && active && sp.kp.den_on) {  // the population's positive app holders: one word per row
                sp.kp.den_bits[j] = notify ? 1u : 0u;
                if (notify) atomicAdd(sp.kp.den_pos + day, 1);
            }
            count_day(active, st, infected, k, kg, s_hist, &s_new, &s_msgs, &s_gath);
        }
        __syncthreads();
        if (threadIdx.x < DEABM_N_STAGE && s_hist[threadIdx.x])
            atomicAdd(&C.hist[((size_t)day * n_pops + tl.pop) * DEABM_N_STAGE + threadIdx.x], s_hist[threadIdx.x]);
        if (threadIdx.x == 0) {
            if (s_new) atomicAdd(&C.new_inf[(size_t)day * n_pops + tl.pop], s_new);
            if (s_msgs) atomicAdd(&C.msgs[day], s_msgs);
            if (s_gath) atomicAdd(&C.gath[day], s_gath);
        }
        __syncthreads();
    }
}

cudaError_t launch_step_ragged(const PopDesc *pops, const Tile *tiles, uint32_t n_tiles, uint32_t *queue, uint32_t day,
                               const float *inf_cur, float *inf_next, const StateRef &S, const Counters &C,
                               uint32_t n_pops, uint32_t grid, bool occ, bool wsg, bool den, cudaStream_t stream)
{
    // compiled with the daily-occupation, the Watts-Strogatz, the dose-day and the
    // notification paths only when some population needs them
    const int v = (den ? 8 : 0) | (occ ? 4 : 0) | (wsg ? 2 : 0) | (S.vd1 ? 1 : 0);
    switch (v) {
#define DEABM_RAGGED_CASE(c, O, W, V, D)                                                                        \
    case c: step_ragged_kernel<O, W, V, D><<<grid, 256, 0, stream>>>(pops, tiles, n_tiles, queue, day, inf_cur, inf_next, S, C, n_pops); break;
        DEABM_RAGGED_CASE(0, false, false, false, false)
        DEABM_RAGGED_CASE(1, false, false, true, false)
        DEABM_RAGGED_CASE(2, false, true, false, false)
        DEABM_RAGGED_CASE(3, false, true, true, false)
        DEABM_RAGGED_CASE(4, true, false, false, false)
        DEABM_RAGGED_CASE(5, true, false, true, false)
        DEABM_RAGGED_CASE(6, true, true, false, false)
        DEABM_RAGGED_CASE(7, true, true, true, false)
        DEABM_RAGGED_CASE(8, false, false, false, true)
        DEABM_RAGGED_CASE(9, false, false, true, true)
        DEABM_RAGGED_CASE(10, false, true, false, true)
        DEABM_RAGGED_CASE(11, false, true, true, true)
        DEABM_RAGGED_CASE(12, true, false, false, true)
        DEABM_RAGGED_CASE(13, true, false, true, true)
        DEABM_RAGGED_CASE(14, true, true, false, true)
        DEABM_RAGGED_CASE(15, true, true, true, true)
#undef DEABM_RAGGED_CASE
    }
    return cudaGetLastError();
}

// Batched panel, four replicates per thread (n_rep a multiple of 4): a warp owns
// one agent row and 128 consecutive replicates, so each in-edge costs one
// broadcast column load and one 16-byte gather per lane, and the row's random
// contacts are generated once for 128 replicates.  Each replicate's sums are
// still left to right in CSR order, so results equal the one-replicate kernels.
constexpr uint32_t kRepPerThread = 4;
#ifndef DEABM_B4_UNROLL
#define DEABM_B4_UNROLL 1   // unroll factor of the per-replicate state update (swept: 1 0.548 ms, 2 0.553,
                            // 4 0.574 a day at N = 1e5, B = 256)
#endif
constexpr int kB4Unroll = DEABM_B4_UNROLL;

__device__ __forceinline__ void add4(float4 &h, const float4 v)
{
    h.x = __fadd_rn(h.x, v.x);
    h.y = __fadd_rn(h.y, v.y);
    h.z = __fadd_rn(h.z, v.z);
    h.w = __fadd_rn(h.w, v.w);
}

// DEN: the positive app holders of the warp's 128 replicates go to four words of
// the row's ceil(B/32) in den_bits (every word is written every day).
template <bool KEEP, bool DEN = false>
#ifndef DEABM_B4_MINB
#define DEABM_B4_MINB 6  // resident blocks per SM asked of the four-replicate kernel: 40 registers with
                         // some spilled (swept at N = 1e5, B = 256: 1 block 105 registers, 38 % slower;
                         // 3 0.634 ms, 4 0.544, 5 0.517, 6 0.512, 7 and 8 0.700 a day)
#endif
__global__ void __launch_bounds__(256, DEABM_B4_MINB) step_batch4_kernel(const KParams P, uint32_t day, const InfBuffers I, StateRef S,
                                                          Counters C, float *lam_out, float *p_out)
{
    __shared__ int s_cnt[DEABM_N_STAGE + 1][32 * kRepPerThread];
    __shared__ unsigned long long s_msgs;
    const uint32_t lane = threadIdx.x, wy = threadIdx.y, tid = wy * 32u + lane;
    const uint32_t j = blockIdx.x * 8u + wy;
    const uint32_t B = P.n_rep;
    const uint32_t b0 = blockIdx.y * (32u * kRepPerThread) + lane * kRepPerThread;
    for (uint32_t q = tid; q < (DEABM_N_STAGE + 1) * 32u * kRepPerThread; q += 256u) (&s_cnt[0][0])[q] = 0;
    if (tid == 0) s_msgs = 0ull;
    __syncthreads();
    uint32_t k = 0, pos4 = 0;  // pos4 bit v: replicate b0 + v is a positive app holder today (DEN)
    if (j < P.n && b0 < B) {
        const uint32_t jo = P.orig_id ? __ldg(P.orig_id + j) : j;
        const int age = __ldg(P.age + j);
        // static networks: per replicate sums in CSR order
        float s4[kRepPerThread] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (uint32_t net = 0; net < P.n_nets; ++net) {
            float4 h = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            const uint32_t e1 = __ldg(P.row_ptr[net] + j + 1);
            for (uint32_t e = __ldg(P.row_ptr[net] + j); e < e1; ++e) {
                const uint32_t c = __ldg(P.col[net] + e);
                add4(h, __ldg((const float4 *)(I.cur + (size_t)c * B + b0)));
            }
            const float hv[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
            for (uint32_t v = 0; v < kRepPerThread; ++v) {
                const float term = __fmul_rn(P.rep[b0 + v].B_net[net], hv[v]);
                s4[v] = net == 0 ? term : __fadd_rn(s4[v], term);
            }
        }
        if (P.n_occ) {
            // the day's occupation contacts, drawn once for the warp's 128 replicates
            const uint32_t g = __ldg(P.occ_gid + j);
            const uint32_t beg = __ldg(P.occ_start + g), size = __ldg(P.occ_start + g + 1u) - beg;
            const uint32_t ko = size > 1u ? (uint32_t)__ldg(P.occ_k + g) : 0u;
            float4 h = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (P.occ_lattice) {  // Watts-Strogatz contacts, two per Philox block (as occ_ws_sum)
                const uint32_t own = j - beg;
                for (uint32_t e = 0; e < ko; e += 2u) {
                    const uint4 w = draw_rk(P.nrk, jo, day, kStreamWs, e >> 1);
                    const uint32_t m = (e >> 1) + 1u;
                    const uint32_t hop = m < size ? m : m % size;
                    const uint32_t coin[2] = {w.x, w.z}, word[2] = {w.y, w.w};
                    float4 v[2];
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
                        v[u] = (e + u < ko) ? __ldg((const float4 *)(I.cur + (size_t)(beg + r) * B + b0))
                                            : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    }
                    add4(h, v[0]);
                    if (e + 1u < ko) add4(h, v[1]);
                }
            } else {
                for (uint32_t e = 0; e < ko; e += 4u) {
                    const uint4 w = draw_rk(P.nrk, jo, day, kStreamOcc, e >> 2);
                    const uint32_t x[4] = {w.x, w.y, w.z, w.w};
                    float4 v[4];
#pragma unroll
                    for (uint32_t u = 0; u < 4u; ++u)
                        v[u] = (e + u < ko) ? __ldg((const float4 *)(I.cur + (size_t)(beg + occ_place(x[u], size - 1u, j - beg)) * B + b0))
                                            : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
                    for (uint32_t u = 0; u < 4u; ++u)
                        if (e + u < ko) add4(h, v[u]);
                }
            }
            const float hv[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
            for (uint32_t v = 0; v < kRepPerThread; ++v) {
                const float term = __fmul_rn(P.rep[b0 + v].B_net[P.n_nets], hv[v]);
                s4[v] = P.n_nets == 0 ? term : __fadd_rn(s4[v], term);
            }
            k = ko;
        }
        if (P.rand_on) {
            uint4 w = draw_rk(P.nrk, jo, day, kStreamRnet, 0u);
            const uint32_t kr = poisson_count(P, w.x, age);
            float4 r = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            const uint64_t nm1 = (uint64_t)(P.n - 1u);
            const float *panel = I.row_of ? I.cur : I.rand_cur;
            // as random_sum: contacts 0..2 from block 0, then four per block,
            // each block's gathers issued together and added in draw order
            for (uint32_t e = 0; e < kr; e += (e == 0u ? 3u : 4u)) {
                if (e) w = draw_rk(P.nrk, jo, day, kStreamRnet, (e + 1u) >> 2);
                const uint32_t x[4] = {w.x, w.y, w.z, w.w};
                const uint32_t u0 = e == 0u ? 1u : 0u;  // block 0 starts at word 1
                float4 v[4];
#pragma unroll
                for (uint32_t u = 0; u < 4u; ++u) {
                    const uint32_t c = e + u - u0;  // contact index of word u
                    uint32_t src = (uint32_t)(((uint64_t)x[u] * nm1) >> 32);
                    src += (src >= jo) ? 1u : 0u;
                    const bool ok = u >= u0 && c < kr;
                    v[u] = ok ? __ldg((const float4 *)(panel + (size_t)(I.row_of ? __ldg(I.row_of + src) : src) * B + b0))
                              : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                }
#pragma unroll
                for (uint32_t u = 0; u < 4u; ++u)
                    if (u >= u0 && e + u - u0 < kr) add4(r, v[u]);
            }
            const float rv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (uint32_t v = 0; v < kRepPerThread; ++v) {
                const float term = __fmul_rn(P.rep[b0 + v].B_rand, rv[v]);
                s4[v] = (P.n_nets == 0 && P.n_occ == 0) ? term : __fadd_rn(s4[v], term);
            }
            k += kr;
        }
        // state of the four replicates (vector loads)
        const size_t i0 = (size_t)j * B + b0;
        const char4 st4 = *(const char4 *)(S.stage + i0);
        const short4 tm4 = *(const short4 *)(S.timer + i0);
        const short4 ti4 = *(const short4 *)(S.tinf + i0);
        const uchar4 fl4 = *(const uchar4 *)(S.flags + i0);
        const uchar4 qt4 = *(const uchar4 *)(S.qt + i0);
        const int8_t st_in[4] = {st4.x, st4.y, st4.z, st4.w};
        const int16_t tm_in[4] = {tm4.x, tm4.y, tm4.z, tm4.w}, ti_in[4] = {ti4.x, ti4.y, ti4.z, ti4.w};
        const uint8_t fl_in[4] = {fl4.x, fl4.y, fl4.z, fl4.w}, qt_in[4] = {qt4.x, qt4.y, qt4.z, qt4.w};
        int8_t st_out[4];
        int16_t tm_out[4], ti_out[4];
        uint8_t fl_out[4], qt_out[4];
        float inf_out[4];
        const int16_t d1 = P.vax_on ? __ldg(P.dose1_day + j) : kNever;
#pragma unroll kB4Unroll
        for (uint32_t v = 0; v < kRepPerThread; ++v) {
            const Rep &rp = P.rep[b0 + v];
            const float lam = __fmul_rn(__fmul_rn(rp.cR, rp.S_age[age]), s4[v]);
            AgentState a;
            a.st = st_in[v];
            a.tm = tm_in[v];
            a.ti = ti_in[v];
            a.fl = fl_in[v];
            a.qd = qt_in[v] & 0x0Fu;
            a.cd = (qt_in[v] >> 4) & 0x07u;
            const uint2 key = seed_key(rp.seed);
            bool inf_now = false;
            uint32_t inf_y = 0;
            float p = 0.0f;
            const float lam_dt = __fmul_rn(lam, P.dt);
            if ((a.st == DEABM_S && lam_dt > 0.0f) || a.qd > 0u || KEEP) {
                const uint4 w = draw(key, jo, day, kStreamInf);
                inf_y = w.y;
                const bool hit = infection_decision(lam_dt, unit_float(w.x), &p);
                inf_now = (a.st == DEABM_S) && hit;
            }
            advance(P, rp, key, jo, day, age, d1, inf_now, a, inf_y, (size_t)jo * B + b0 + v);
            if (DEN && a.pos_result && (a.fl & DEABM_FL_APP)) pos4 |= 1u << v;
            st_out[v] = (int8_t)a.st;
            tm_out[v] = (int16_t)a.tm;
            ti_out[v] = (int16_t)a.ti;
            fl_out[v] = (uint8_t)a.fl;
            qt_out[v] = (uint8_t)((a.qd & 0x0Fu) | ((a.cd & 0x07u) << 4));
            inf_out[v] = emitted(P.tab, P.inf_len, a.st, a.ti, a.qd);
            if (KEEP) {
                lam_out[i0 + v] = lam;
                p_out[i0 + v] = p;
            }
            atomicAdd(&s_cnt[a.st][lane * kRepPerThread + v], 1);
            if (inf_now) atomicAdd(&s_cnt[DEABM_N_STAGE][lane * kRepPerThread + v], 1);
        }
        *(char4 *)(S.stage + i0) = make_char4(st_out[0], st_out[1], st_out[2], st_out[3]);
        *(short4 *)(S.timer + i0) = make_short4(tm_out[0], tm_out[1], tm_out[2], tm_out[3]);
        *(short4 *)(S.tinf + i0) = make_short4(ti_out[0], ti_out[1], ti_out[2], ti_out[3]);
        *(uchar4 *)(S.flags + i0) = make_uchar4(fl_out[0], fl_out[1], fl_out[2], fl_out[3]);
        *(uchar4 *)(S.qt + i0) = make_uchar4(qt_out[0], qt_out[1], qt_out[2], qt_out[3]);
        const float4 iv = make_float4(inf_out[0], inf_out[1], inf_out[2], inf_out[3]);
        *(float4 *)(I.next + i0) = iv;
        if (I.rand_next) *(float4 *)(I.rand_next + (size_t)jo * B + b0) = iv;
    }
    if (DEN) {  // lanes 8q .. 8q + 7 hold the 32 replicates of word 4 blockIdx.y + q
        uint32_t v = pos4 << ((lane & 7u) * 4u);
        v |= __shfl_xor_sync(0xFFFFFFFFu, v, 1);
        v |= __shfl_xor_sync(0xFFFFFFFFu, v, 2);
        v |= __shfl_xor_sync(0xFFFFFFFFu, v, 4);
        const uint32_t W = (B + 31u) / 32u, w = blockIdx.y * 4u + (lane >> 3);
        if ((lane & 7u) == 0u && j < P.n && w < W) {
            P.den_bits[(size_t)j * W + w] = v;
            if (v) atomicAdd(P.den_pos + day, __popc(v));
        }
    }
    if (lane == 0 && blockIdx.y == 0 && j < P.n && k) atomicAdd(&s_msgs, (unsigned long long)k);
    __syncthreads();
    for (uint32_t q = tid; q < (DEABM_N_STAGE + 1) * 32u * kRepPerThread; q += 256u) {
        const uint32_t s = q / (32u * kRepPerThread), l = q % (32u * kRepPerThread);
        const uint32_t bb = blockIdx.y * (32u * kRepPerThread) + l;
        const int v = s_cnt[s][l];
        if (v && bb < B) {
            if (s < DEABM_N_STAGE) atomicAdd(&C.hist[((size_t)day * B + bb) * DEABM_N_STAGE + s], v);
            else atomicAdd(&C.new_inf[(size_t)day * B + bb], v);
        }
    }
    if (tid == 0 && s_msgs) atomicAdd(&C.msgs[day], s_msgs);
}

cudaError_t launch_step(const KParams &P, uint32_t day, const InfBuffers &I, const StateRef &S, const Counters &C,
                        float *lam_out, float *p_out, cudaStream_t stream)
{
    if (P.n_rep == 1) {
        const dim3 grid((P.n + DEABM_PLAIN_BLOCK - 1u) / DEABM_PLAIN_BLOCK);
        const int v = (P.wsg_on ? 8 : 0) | (lam_out ? 4 : 0) | (P.n_occ ? 2 : 0) | (P.den_on ? 1 : 0);
        switch (v) {
#define DEABM_PLAIN_CASE(c, K, O, D, W)                                                                      \
    case c: step_plain_kernel<K, O, D, W><<<grid, DEABM_PLAIN_BLOCK, 0, stream>>>(P, day, I, S, C, lam_out, p_out); break;
            DEABM_PLAIN_CASE(0, false, false, false, false)
            DEABM_PLAIN_CASE(1, false, false, true, false)
            DEABM_PLAIN_CASE(2, false, true, false, false)
            DEABM_PLAIN_CASE(3, false, true, true, false)
            DEABM_PLAIN_CASE(4, true, false, false, false)
            DEABM_PLAIN_CASE(5, true, false, true, false)
            DEABM_PLAIN_CASE(6, true, true, false, false)
            DEABM_PLAIN_CASE(7, true, true, true, false)
            DEABM_PLAIN_CASE(8, false, false, false, true)
            DEABM_PLAIN_CASE(9, false, false, true, true)
            DEABM_PLAIN_CASE(10, false, true, false, true)
            DEABM_PLAIN_CASE(11, false, true, true, true)
            DEABM_PLAIN_CASE(12, true, false, false, true)
            DEABM_PLAIN_CASE(13, true, false, true, true)
            DEABM_PLAIN_CASE(14, true, true, false, true)
            DEABM_PLAIN_CASE(15, true, true, true, true)
#undef DEABM_PLAIN_CASE
        }
    } else if (P.n_rep % kRepPerThread == 0 && P.vax_strategy == 0 && !P.wsg_on) {
        // (priority strategies and the Watts-Strogatz random network: the general panel)
        const dim3 grid((P.n + 7u) / 8u, (P.n_rep + 32u * kRepPerThread - 1u) / (32u * kRepPerThread));
        const dim3 block(32, 8);
        if (P.den_on) {
            if (lam_out) step_batch4_kernel<true, true><<<grid, block, 0, stream>>>(P, day, I, S, C, lam_out, p_out);
            else step_batch4_kernel<false, true><<<grid, block, 0, stream>>>(P, day, I, S, C, nullptr, nullptr);
        } else {
            if (lam_out) step_batch4_kernel<true><<<grid, block, 0, stream>>>(P, day, I, S, C, lam_out, p_out);
            else step_batch4_kernel<false><<<grid, block, 0, stream>>>(P, day, I, S, C, nullptr, nullptr);
        }
    } else {
        const dim3 grid((P.n + 7u) / 8u, (P.n_rep + 31u) / 32u);
        const dim3 block(32, 8);
        if (P.wsg_on && P.den_on) {
            if (lam_out) step_batch_kernel<true, true, true><<<grid, block, 0, stream>>>(P, day, I, S, C, lam_out, p_out);
            else step_batch_kernel<false, true, true><<<grid, block, 0, stream>>>(P, day, I, S, C, nullptr, nullptr);
        } else if (P.wsg_on) {
            if (lam_out) step_batch_kernel<true, true><<<grid, block, 0, stream>>>(P, day, I, S, C, lam_out, p_out);
            else step_batch_kernel<false, true><<<grid, block, 0, stream>>>(P, day, I, S, C, nullptr, nullptr);
        } else if (P.den_on) {
            if (lam_out) step_batch_kernel<true, false, true><<<grid, block, 0, stream>>>(P, day, I, S, C, lam_out, p_out);
            else step_batch_kernel<false, false, true><<<grid, block, 0, stream>>>(P, day, I, S, C, nullptr, nullptr);
        } else {
            if (lam_out) step_batch_kernel<true, false><<<grid, block, 0, stream>>>(P, day, I, S, C, lam_out, p_out);
            else step_batch_kernel<false, false><<<grid, block, 0, stream>>>(P, day, I, S, C, nullptr, nullptr);
        }
    }
    return cudaGetLastError();
}

}  // namespace deabm
