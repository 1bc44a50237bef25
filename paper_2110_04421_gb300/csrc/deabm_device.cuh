// deabm_device.cuh -- device-side pieces shared by the step kernels of libdeabm.
//
// Philox4x32-10, the per-context parameter block, and the per-agent state
// machine (Sec. 3 "Disease Progression", Sec. 4 interventions) of DeepABM-COVID.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "deabm.h"

namespace deabm {

// Philox counter word 2 ("stream") layout; counter = (agent, day, stream, block)
enum : uint32_t {
    kStreamInf = 0,    // x: infection uniform, y: quarantine dropout
    kStreamProg = 1,   // x: asymptomatic?, y: stage duration, z: severe?, w: secondary branch
    kStreamRnet = 3,   // random network: word 0 = contact count, words 1.. = contacts
    kStreamOcc = 4,    // daily occupation network: word e = contact e
    kStreamTest = 5,   // x: test positive?, y: result delay
    kStreamDen = 6,    // x: complies with a notification; day word 0xFFFFFFFD: x = holds the app
    kStreamVax = 7,    // x: vaccine response (day word fixed at 0)
    kStreamGumbel = 8, // relaxed draw noise
    kStreamWs = 9,     // Watts-Strogatz occupation contacts: block e/2, lanes 2(e%2), 2(e%2)+1 = coin, place
    kStreamWsg = 10,   // Watts-Strogatz global random network: edge m of an agent in block (m-1)/2, lanes
                       // 2((m-1)%2), 2((m-1)%2)+1 = rewire coin, new far end
};
constexpr uint32_t kSeedDay = 0xFFFFFFFFu;  // day word of the infections before day 0
constexpr int16_t kNever = 0x7FFF;

// ---------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}
__device__ __forceinline__ uint2 seed_key(uint64_t s) { return make_uint2((uint32_t)s, (uint32_t)(s >> 32)); }

// The same generator with its ten round keys given: rk[2r], rk[2r+1] = the key
// after r bumps (k + r (0x9E3779B9, 0xBB67AE85)), computed once on the host.  When
// rk lives in the kernel's parameter space the round keys are operands of the
// XORs, and the two adds of each round disappear.
#ifndef DEABM_PHILOX_WIDE
#define DEABM_PHILOX_WIDE 0  // 1: each round's products as one 64-bit product per word
#endif
__device__ __forceinline__ uint4 philox_rk(uint4 c, const uint32_t *rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#if DEABM_PHILOX_WIDE
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0, hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#else
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#endif
        c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
    }
    return c;
}
__device__ __forceinline__ uint4 draw_rk(const uint32_t *rk, uint32_t agent, uint32_t day, uint32_t stream,
                                         uint32_t blk = 0)
{
    return philox_rk(make_uint4(agent, day, stream, blk), rk);
}
__device__ __forceinline__ uint4 draw(uint2 key, uint32_t agent, uint32_t day, uint32_t stream, uint32_t blk = 0)
{
    return philox(make_uint4(agent, day, stream, blk), key);
}
// 24-bit uniform in [0,1), exact in FP32
__device__ __forceinline__ float unit_float(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }
__device__ __forceinline__ uint32_t uniform_int(uint32_t w, uint32_t lo, uint32_t hi)
{
    return lo + (uint32_t)(((uint64_t)w * (uint64_t)(hi - lo + 1u)) >> 32);
}

// ---------------------------------------------------------------- parameter blocks
// Tables with per-thread dynamic indices live in device global memory (L1-resident).
struct Tables {
    float infT[DEABM_N_CLASS][DEABM_MAX_INF_LEN];  // A_class folded in: A_c * infT_c[t]
    uint64_t pois[DEABM_POIS_CAP];
    uint64_t pois_age[DEABM_N_AGE][DEABM_POIS_CAP];  // rand_by_age: the thresholds of each age bin's mean
    uint64_t thr_asym[DEABM_N_AGE], thr_sev[DEABM_N_AGE];
    uint64_t thr_branch[8][DEABM_N_AGE];   // by stage: SEV->HOSP, HOSP->ICU, ICU->DEAD
    uint8_t dur_lo[8][DEABM_N_AGE], dur_hi[8][DEABM_N_AGE];
};

// per replicate (n_rep entries; plain runs have one)
struct Rep {
    float cR;                    // R * inv_Ibar (FP32 product)
    float B_net[DEABM_MAX_NETS];
    float B_rand;
    float S_age[DEABM_N_AGE];
    uint32_t dose2_delay;
    uint64_t seed;
    uint32_t rk[20];             // Philox round keys of seed (philox_rk)
};

// by-value kernel argument
struct KParams {
    uint32_t n, n_nets, n_rep, inf_len;
    float dt;
    uint32_t rand_on;
    const uint32_t *row_ptr[DEABM_MAX_NETS];
    const uint32_t *col[DEABM_MAX_NETS];
    uint64_t net_seed;
    uint32_t test_on, test_lo, test_hi, quar_on, quar_days;
    uint64_t thr_sens, thr_qdrop;
    uint32_t vax_on, vax_onset;
    uint64_t thr_eff1, thr_eff2;
    const Tables *tab;
    const Rep *rep;
    const uint8_t *age;        // by internal id
    const int16_t *dose1_day;  // by internal id
    const uint32_t *orig_id;   // internal id -> caller's agent id (nullptr: the same)
    uint32_t vax_strategy;     // 0 static schedule; 1..3 priority strategies with a shared supply
    uint32_t vax_nonsterile;   // 1: immunity leaves the agent susceptible (flag), infections asymptomatic
    const uint8_t *dose_today; // priority strategies: 1 = dosed today, [caller id][replicate] (nullptr: none)
    // daily occupation networks (n_occ = 0: none).  Internal rows are in
    // occupation order, members of one occupation consecutive and in ascending
    // caller id, so the member in place r of occupation g is row occ_start[g] + r.
    uint32_t n_occ;
    const uint32_t *occ_gid;    // [n] occupation of each internal row
    const uint32_t *occ_start;  // [n_occ + 1] first internal row of each occupation
    const uint8_t *occ_k;       // [n_occ] daily in-contacts of a member
    uint32_t occ_lattice;       // 1: Watts-Strogatz ring lattice, rewired daily
    uint64_t thr_rewire;
    // digital exposure notification (den_on = 0: none).  Bit r of den_bits is
    // set when row r is an app holder whose positive result landed today; the
    // same by caller id in den_bits_orig (nullptr when the ids are not
    // relabelled; cleared before each day).
    uint32_t den_on, den_window;
    uint64_t thr_comp, thr_adopt;
    uint32_t *den_bits, *den_bits_orig;
    int32_t *den_pos;           // [day] positive app holders of the day
    // the app holders: their rows in ascending order, and each row's rank among
    // them; each app holder's in-contacts of the last den_window days: word e of
    // the record of (day d, rank a) at den_ring[((d % den_window) * den_slots + e)
    // * n_app + a]
    uint32_t n_app;
    const uint32_t *app_rows, *app_rank;
    uint32_t *den_ring;
    uint32_t den_slots;
    // The random network's Poisson CDF thresholds (Tables::pois) as 32-bit words:
    // thresholds from index pois_fin on are 2^32, which no word reaches.
    uint32_t pois32[DEABM_POIS_CAP];
    uint32_t pois_fin;
    uint32_t nrk[20];  // Philox round keys of net_seed (philox_rk)
    // replicate 0's parameters by value: plain contexts read them from the
    // kernel's parameter space (uniform across the grid) instead of through `rep`
    Rep rep0;
    // the global random network as a daily Watts-Strogatz graph (wsg_on; then
    // rand_on = 0): h = k/2 owned edges per agent, rewiring threshold; the day's
    // graph built before the day kernel, by caller id: bit m-1 of wsg_rew[i] = edge
    // m of agent i rewired; the owners of the rewired edges that landed on agent v
    // at wsg_land[wsg_start[v] .. wsg_start[v+1]), ascending
    uint32_t wsg_on, wsg_h;
    uint64_t thr_wsg;
    const uint8_t *wsg_rew;
    const uint32_t *wsg_start;
    const uint32_t *wsg_land;
    uint32_t rand_by_age;  // 1: agent j's random-contact count from tab->pois_age[age_j] (age-stratified means)
    // with exposure notification, the Watts-Strogatz graphs of the last
    // wsg_ring_days days (day d in slot d % wsg_ring_days): landing slot ends
    // [slot][n + 3] (agent v's landings at [ends[v + 2], ends[v + 3]) of the slot's
    // owners [slot][n wsg_h])
    const uint32_t *wsg_ends_ring;
    const uint32_t *wsg_land_ring;
    uint32_t wsg_ring_days;
};

// K_j of the random network from word 0 of its block 0: the number of Poisson
// thresholds at or below w, which (the thresholds being non-decreasing) is the
// first index whose threshold exceeds w.  The first eight compares are unrolled
// against the parameter-space thresholds; beyond them (P(K >= 8) < 0.2 % at the
// mean of 2) a loop finishes the count.
#ifndef DEABM_POIS32
#define DEABM_POIS32 1
#endif
__device__ __forceinline__ uint32_t poisson_count(const KParams &P, uint32_t w, int age)
{
    if (P.rand_by_age) {  // age-stratified means: the bin's thresholds from the table (L1)
        const uint64_t *thr = P.tab->pois_age[age];
        uint32_t c = 0;
        while (c < DEABM_POIS_CAP && (uint64_t)w >= __ldg(thr + c)) ++c;
        return c;
    }
#if !DEABM_POIS32
    uint32_t c = 0;
    while (c < DEABM_POIS_CAP && (uint64_t)w >= __ldg(&P.tab->pois[c])) ++c;
    return c;
#endif
    uint32_t k = 0;
#pragma unroll
    for (uint32_t t = 0; t < 8u; ++t) k += (t < P.pois_fin && w >= P.pois32[t]) ? 1u : 0u;
    if (k == 8u)
        for (uint32_t t = 8u; t < P.pois_fin && w >= P.pois32[t]; ++t) ++k;
    return k;
}

// Infectiousness buffers of a day.  Static-network gathers read `cur` (internal
// ids); random-network gathers read `rand_cur`, indexed by the caller's agent ids
// (the same array when the ids are not relabelled).
struct InfBuffers {
    const float *cur;
    float *next;
    const float *rand_cur;
    float *rand_next;  // nullptr when not relabelled
    // caller id -> internal row (batched contexts when relabelled): random
    // contacts then read `cur` through it and there is no copy by caller id
    const uint32_t *row_of;
};

struct StateRef {
    int8_t *stage;
    int16_t *timer, *tinf;
    uint8_t *flags, *qt;
    int16_t *vd1, *vd2;  // dose days under a priority strategy (nullptr otherwise)
};

// One population of a ragged batch: a KParams view whose CSR, age and dose-day
// pointers are already offset to the population's slice (local ids), its
// replicate parameters, and the offset of its agents in the concatenated state.
struct PopDesc {
    KParams kp;
    Rep rep;
    const uint32_t *row_of;  // the population's caller id -> local row (nullptr: not renumbered)
    uint32_t base;
    uint32_t pad_[3];
};

// A unit of work of the ragged day kernel: rows [begin, end) of population pop.
struct Tile {
    uint32_t pop, begin, end, pad_;
};

struct Counters {
    int32_t *new_inf;          // [day][n_rep]
    int32_t *hist;             // [day][n_rep][11]
    unsigned long long *msgs;  // [day] random in-contacts (static edges added on the host)
    unsigned long long *gath;  // [day] in-contacts (stored, occupation, random) of the destinations that gathered
    int32_t *den;              // [day] agents notified (exposure notification)
};

// ---------------------------------------------------------------- state machine
struct AgentState {
    int st, tm, ti;
    uint32_t fl, qd, cd;
    int vd1 = kNever, vd2 = kNever;
    bool pos_result = false;  // a positive test result landed in this update
};

__device__ __forceinline__ int infector_class(int st)
{
    // asymptomatic -> 0; presymptomatic/symptomatic mild -> 1; severe -> 2; others none
    return st == DEABM_ASYM ? 0
         : (st == DEABM_PRE_MILD || st == DEABM_MILD) ? 1
         : (st == DEABM_PRE_SEV || st == DEABM_SEV) ? 2 : -1;
}

// infectiousness an agent emits on a day: A_c * infT_c[tinf], zero when quarantined
__device__ __forceinline__ float emitted(const Tables *tab, uint32_t L, int st, int ti, uint32_t qd)
{
    const int c = infector_class(st);
    if (c < 0 || qd != 0u || ti < 0 || (uint32_t)ti >= L) return 0.0f;
    return __ldg(&tab->infT[c][ti]);
}

__device__ __forceinline__ void new_infection(const Tables *tab, int age, uint4 w, AgentState &a)
{
    if (a.fl & DEABM_FL_IMMUNE) a.st = DEABM_ASYM;  // vaccinated, non-sterilising: asymptomatic infection
    else if ((uint64_t)w.x < __ldg(&tab->thr_asym[age])) a.st = DEABM_ASYM;
    else if ((uint64_t)w.z < __ldg(&tab->thr_sev[age])) a.st = DEABM_PRE_SEV;
    else a.st = DEABM_PRE_MILD;
    a.tm = (int)uniform_int(w.y, __ldg(&tab->dur_lo[a.st][age]), __ldg(&tab->dur_hi[a.st][age]));
    a.ti = 1;
}

// One day's update of one agent (everything after the infection draw).
// `infected` = the draw succeeded this day; `day` is the day index.
template <bool RK = false>
__device__ __forceinline__ void advance(const KParams &P, const Rep &rp, uint2 key, uint32_t j, uint32_t day,
                                        int age, int16_t d1, bool infected, AgentState &a, uint32_t inf_y,
                                        size_t dsel)
{
    // the replicate's draws: from its round keys (RK: rp in parameter or shared
    // space) or from the seed's key schedule
    auto draw_rep = [&](uint32_t dday, uint32_t stream) {
        return RK ? draw_rk(rp.rk, j, dday, stream) : draw(key, j, dday, stream);
    };
    bool onset = false;
    // one draw site for a new infection and for the end of a stage, so that a
    // warp holding both runs the Philox rounds once
    const bool in_course = !infected && a.st >= DEABM_ASYM && a.st <= DEABM_ICU;
    if (in_course) {
        a.ti = a.ti < 32767 ? a.ti + 1 : 32767;
        a.tm -= 1;
    }
    const bool stage_ends = in_course && a.tm <= 0;
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    if (infected || stage_ends) w = draw_rep(day, kStreamProg);
    if (infected) {
        new_infection(P.tab, age, w, a);
    } else if (stage_ends) {
        int nx;
        switch (a.st) {
        case DEABM_PRE_MILD: nx = DEABM_MILD; onset = true; break;
        case DEABM_PRE_SEV: nx = DEABM_SEV; onset = true; break;
        case DEABM_SEV: nx = (uint64_t)w.w < __ldg(&P.tab->thr_branch[DEABM_SEV][age]) ? DEABM_HOSP : DEABM_REC; break;
        case DEABM_HOSP: nx = (uint64_t)w.w < __ldg(&P.tab->thr_branch[DEABM_HOSP][age]) ? DEABM_ICU : DEABM_REC; break;
        case DEABM_ICU: nx = (uint64_t)w.w < __ldg(&P.tab->thr_branch[DEABM_ICU][age]) ? DEABM_DEAD : DEABM_REC; break;
        default: nx = DEABM_REC; break;  // asymptomatic, mild
        }
        a.st = nx;
        a.tm = (nx >= DEABM_ASYM && nx <= DEABM_ICU)
                   ? (int)uniform_int(w.y, __ldg(&P.tab->dur_lo[nx][age]), __ldg(&P.tab->dur_hi[nx][age]))
                   : 0;
    }
    // quarantine in progress: daily dropout, else one day served (Sec. 4.1)
    if (a.qd > 0u) {
        if ((uint64_t)inf_y < P.thr_qdrop) a.qd = 0u;
        else a.qd -= 1u;
    }
    // pending test result, or a test at symptom onset or after yesterday's
    // exposure notification (Sec. 4.3, 4.2); only an infected agent in the
    // community (stages 1..5) can test positive
    if (a.cd > 0u) {
        a.cd -= 1u;
        if (a.cd == 0u) {
            if (a.fl & DEABM_FL_POS) {
                if (P.quar_on) a.qd = P.quar_days;
                a.pos_result = true;
            }
            a.fl &= ~DEABM_FL_POS;
        }
    } else if ((onset || (a.fl & DEABM_FL_DEN)) && P.test_on && a.qd == 0u) {
        const uint4 w = draw_rep(day, kStreamTest);
        if (a.st >= DEABM_ASYM && a.st <= DEABM_SEV && (uint64_t)w.x < P.thr_sens) a.fl |= DEABM_FL_POS;
        else a.fl &= ~DEABM_FL_POS;
        a.cd = uniform_int(w.y, P.test_lo, P.test_hi);
    }
    a.fl &= ~DEABM_FL_DEN;  // a notification is acted on the next day or not at all
    // two-dose vaccination (Sec. 4.4, Sec. 5)
    if (P.vax_on && P.vax_strategy != 0) {
        // priority strategies: today's doses were selected before the day from its starting state
        if (P.dose_today && P.dose_today[dsel]) {  // dsel: the agent's (caller id, replicate) slot
            if (!(a.fl & DEABM_FL_DOSE1)) { a.fl |= DEABM_FL_DOSE1; a.vd1 = (int)day; }
            else { a.fl |= DEABM_FL_DOSE2; a.vd2 = (int)day; }
        }
        if (a.st == DEABM_S && !infected) {
            const bool on1 = (a.fl & DEABM_FL_DOSE1) && (int64_t)day == (int64_t)a.vd1 + (int64_t)P.vax_onset;
            const bool on2 = (a.fl & DEABM_FL_DOSE2) && (int64_t)day == (int64_t)a.vd2 + (int64_t)P.vax_onset;
            if (on1 || on2) {
                const uint32_t v = draw_rep(0u, kStreamVax).x;
                if ((on1 && (uint64_t)v < P.thr_eff1) || (on2 && (uint64_t)v < P.thr_eff2)) {
                    if (P.vax_nonsterile) a.fl |= DEABM_FL_IMMUNE;
                    else a.st = DEABM_VAX;
                }
            }
        }
    } else if (P.vax_on && d1 != kNever) {
        const int64_t t = day, D1 = d1, D2 = D1 + (int64_t)rp.dose2_delay;
        const bool elig = !(a.st == DEABM_HOSP || a.st == DEABM_ICU || a.st == DEABM_DEAD);
        if (t == D1 && elig) a.fl |= DEABM_FL_DOSE1;
        if ((a.fl & DEABM_FL_DOSE1) && t == D2 && elig) a.fl |= DEABM_FL_DOSE2;
        if (a.st == DEABM_S && !infected) {
            const bool on1 = (a.fl & DEABM_FL_DOSE1) && t == D1 + (int64_t)P.vax_onset;
            const bool on2 = (a.fl & DEABM_FL_DOSE2) && t == D2 + (int64_t)P.vax_onset;
            if (on1 || on2) {
                const uint32_t v = draw_rep(0u, kStreamVax).x;
                if ((on1 && (uint64_t)v < P.thr_eff1) || (on2 && (uint64_t)v < P.thr_eff2)) {
                    if (P.vax_nonsterile) a.fl |= DEABM_FL_IMMUNE;
                    else a.st = DEABM_VAX;
                }
            }
        }
    }
}

}  // namespace deabm
