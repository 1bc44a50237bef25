// deabm_api.cu -- the C ABI of libdeabm (declared in include/deabm.h): context
// creation and validation, device memory ownership, the day loop, readback.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "deabm.h"
#include "deabm_device.cuh"
#include "kernels.h"

using namespace deabm;

struct deabm_ctx {
    cudaStream_t stream = nullptr;
    uint32_t n = 0, n_nets = 0, n_rep = 1, max_steps = 0, day = 0;
    uint64_t static_edges = 0;
    bool keep_lambda = false;
    std::vector<void *> allocs;               // device blocks owned by the context (freed at destroy)
    // the context's arrays are carved out of a few large device blocks (one
    // cudaMalloc and one cudaFree each instead of one per array)
    char *arena = nullptr;
    size_t arena_used = 0, arena_size = 0, arena_chunk = 0;
    uint32_t *row_ptr[DEABM_MAX_NETS] = {};
    uint32_t *col[DEABM_MAX_NETS] = {};
    WsgBuffers wsg{};                         // the day's Watts-Strogatz random network (rand_ws)
    uint8_t *age = nullptr;
    int16_t *dose1 = nullptr;
    StateRef S{};
    float *inf[2] = {nullptr, nullptr};
    float *inf_rand[2] = {nullptr, nullptr};  // by caller id: plain contexts, relabelled, random network on
    uint32_t *row_of = nullptr;               // caller id -> row: batched contexts, relabelled
    int cur = 0;
    bool relabel = false;
    std::vector<uint32_t> new2orig;           // internal id -> caller id (relabelled only)
    uint32_t *orig_id = nullptr;
    void *perm_scratch = nullptr;             // caller-order copies for the readbacks (relabelled only)
    uint32_t *orig_local = nullptr, *row_local = nullptr;  // ragged: per population, local ids
    // daily occupation networks (internal rows in occupation order)
    uint32_t n_occ = 0;
    uint32_t *occ_gid = nullptr, *occ_start = nullptr;
    uint8_t *occ_k = nullptr;
    // exposure notification: today's positive app holders (internal rows, caller ids;
    // batched: [n][ceil(B/32)] words by rows), per-day counts
    uint32_t *den_bits = nullptr, *den_bits_orig = nullptr;
    int32_t *den_pos = nullptr;
    uint32_t *den_ring = nullptr;  // [den_window][slots][n_app] contact records of the app holders
    size_t den_ring_cap = 0;       // app holders the ring has room for
    uint32_t *app_rows = nullptr, *app_rank = nullptr;
    float *lam = nullptr, *p = nullptr;
    Tables *tab = nullptr;
    Rep *rep = nullptr;
    Counters C{};
    KParams kp{};
    StateRef S0{};                 // initial state as given at create (before the initial cases)
    uint32_t *seed_ids = nullptr;  // initial cases, internal ids
    uint32_t n_seed = 0;
    deabm_params base{};
    // ragged batch of populations (n_rep counts the populations for the counters)
    bool ragged = false;
    bool ragged_occ = false;  // some population of the ragged batch draws daily occupation contacts
    bool ragged_wsg = false;  // some population of the ragged batch has a Watts-Strogatz random network
    std::vector<std::pair<uint32_t, WsgBuffers>> ragged_wsg_bufs;  // (population, its day's graph)
    std::vector<uint32_t> ragged_den;  // the populations with exposure notification
    std::vector<PopDesc> pops;         // host copies, KParams pointers already offset
    PopDesc *d_pops = nullptr;
    Tile *d_tiles = nullptr;
    uint32_t n_tiles = 0, max_tiles = 0, rows_per_tile = 1024, grid = 0, sm_count = 0;
    uint32_t *queue = nullptr;         // [max_steps] tile counters, one per day
    std::vector<std::vector<uint32_t>> pop_seeds;
    std::vector<uint32_t *> d_pop_seeds;
    cudaStream_t own_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    uint32_t graph_day0 = 0, graph_T = 0;
    // vaccination priority strategies: today's classes and doses by caller id, selection scratch
    uint8_t *vax_cls = nullptr, *vax_dose = nullptr;
    uint32_t *vax_scratch = nullptr;
    uint32_t vax_supply = 0;
    // ragged batches: the populations under a priority strategy (their index,
    // daily supply, first day, dose-2 delay and first "65+" bin)
    struct RaggedVax {
        uint32_t q, supply, start, delay, elderly;
    };
    std::vector<RaggedVax> ragged_vax;
    std::string err;
};

static thread_local std::string g_err;

static int fail(deabm_ctx *ctx, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    g_err = buf;
    return code;
}

#define CU(ctx, call)                                                                                    \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? DEABM_ENOMEM : DEABM_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                             \
    } while (0)

// Allocation-failure injection for the tests (deabm_inject_alloc_failure): the
// number of device allocations of simulation contexts still to succeed before
// one fails; 0 = off.
static std::atomic<uint32_t> g_alloc_fault{0};

static bool injected_alloc_failure()
{
    uint32_t c = g_alloc_fault.load();
    while (c != 0u)
        if (g_alloc_fault.compare_exchange_weak(c, c - 1u)) return c == 1u;
    return false;
}

extern "C" void deabm_inject_alloc_failure(uint32_t after) { g_alloc_fault.store(after); }

template <class T>
static int dalloc(deabm_ctx *ctx, T **out, size_t count)
{
    const size_t bytes = count ? count * sizeof(T) : sizeof(T);
    const size_t rounded = (bytes + 255u) & ~(size_t)255u;  // every array 256-byte aligned
    const size_t chunk = ctx->arena_chunk ? ctx->arena_chunk : (size_t)1 << 20;
    const bool own_block = rounded > chunk / 4;  // large arrays get a block of their own
    if (!own_block && ctx->arena && ctx->arena_used + rounded <= ctx->arena_size) {
        *out = (T *)(ctx->arena + ctx->arena_used);
        ctx->arena_used += rounded;
        return DEABM_OK;
    }
    void *ptr = nullptr;
    const size_t block = own_block ? rounded : chunk;
    cudaError_t e = injected_alloc_failure() ? cudaErrorMemoryAllocation : cudaMalloc(&ptr, block);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ctx, DEABM_ENOMEM, "cudaMalloc of %zu bytes failed: %s", block, cudaGetErrorString(e));
    }
    ctx->allocs.push_back(ptr);
    if (!own_block) {
        ctx->arena = (char *)ptr;
        ctx->arena_size = block;
        ctx->arena_used = rounded;
    }
    *out = (T *)ptr;
    return DEABM_OK;
}

// Block size for the context's small arrays: about what a context of n agents x
// n_rep replicates keeps, between 1 MB and 256 MB.
static void arena_plan(deabm_ctx *ctx, uint64_t n, uint64_t n_rep)
{
    const uint64_t want = n * n_rep * 32u + n * 16u;
    ctx->arena_chunk = (size_t)std::min<uint64_t>(std::max<uint64_t>(want, 1u << 20), 256ull << 20);
}

static uint64_t threshold(double p)
{
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return (uint64_t)1 << 32;
    return (uint64_t)std::floor(p * 4294967296.0);
}

// Poisson(m) CDF thresholds: t_0 = exp(-m), t_k = (t_{k-1} * m) / k, c_k = c_{k-1} + t_k
static void poisson_thresholds(double m, uint64_t *thr)
{
    volatile double t = std::exp(-m), c = t;
    thr[0] = threshold(c);
    for (int k = 1; k < DEABM_POIS_CAP; ++k) {
        t = (t * m) / (double)k;
        c = c + t;
        thr[k] = threshold(c);
    }
}

// the Poisson random network is on: a positive mean (of some age bin when the
// means are age-stratified), and not replaced by the Watts-Strogatz graph
static bool poisson_on(const deabm_graph *g)
{
    if (g->rand_ws) return false;
    if (!g->rand_by_age) return g->rand_mean > 0.0f;
    for (int a = 0; a < DEABM_N_AGE; ++a)
        if (g->rand_mean_age[a] > 0.0f) return true;
    return false;
}

// both Poisson tables of a context's graph (the single mean, and each age bin's)
static void poisson_tables(const deabm_graph *g, Tables &T)
{
    poisson_thresholds((double)g->rand_mean, T.pois);
    for (int a = 0; a < DEABM_N_AGE; ++a)
        poisson_thresholds(g->rand_by_age ? (double)g->rand_mean_age[a] : (double)g->rand_mean, T.pois_age[a]);
}

// Before a state is installed (create, reset, restore): the infectiousness
// buffers the next day writes start at 0, since the day kernels leave a quiet
// susceptible agent's entry untouched (it emits nothing).
static cudaError_t clear_next_buffers(deabm_ctx *ctx, size_t count)
{
    cudaError_t e = cudaMemsetAsync(ctx->inf[1], 0, sizeof(float) * count, ctx->stream);
    if (e == cudaSuccess && ctx->inf_rand[1]) e = cudaMemsetAsync(ctx->inf_rand[1], 0, sizeof(float) * count, ctx->stream);
    return e;
}

// Philox4x32-10 round keys of a 64-bit seed: the key (low, high word) after r
// bumps by the Weyl constants 0x9E3779B9, 0xBB67AE85, r = 0..9 (philox_rk)
static void round_keys(uint64_t seed, uint32_t *rk)
{
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k0;
        rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// the Poisson thresholds as the day kernels' 32-bit words (KParams::pois32)
static void set_pois32(KParams &K, const uint64_t *pois)
{
    K.pois_fin = 0;
    for (int k = 0; k < DEABM_POIS_CAP; ++k) {
        K.pois32[k] = pois[k] < ((uint64_t)1 << 32) ? (uint32_t)pois[k] : 0xFFFFFFFFu;
        if (pois[k] < ((uint64_t)1 << 32)) K.pois_fin = (uint32_t)k + 1u;
    }
}

static bool prob_ok(double p) { return p >= 0.0 && p <= 1.0; }

// ---------------------------------------------------------------- validation
// The first row in [0, n) for which bad(row) holds, or n: rows split over host
// threads (validation of a graph of tens of millions of edges is otherwise the
// largest host cost of create).
template <class F>
static uint32_t first_bad_row(uint32_t n, const F &bad)
{
    const uint32_t hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const uint32_t T = n < (1u << 16) ? 1u : hw;
    std::vector<uint32_t> found(T, n);
    auto work = [&](uint32_t t) {
        const uint32_t r0 = (uint32_t)((uint64_t)n * t / T), r1 = (uint32_t)((uint64_t)n * (t + 1) / T);
        for (uint32_t j = r0; j < r1; ++j)
            if (bad(j)) {
                found[t] = j;
                return;
            }
    };
    if (T == 1) {
        work(0);
    } else {
        std::vector<std::thread> th;
        th.reserve(T);
        for (uint32_t t = 0; t < T; ++t) th.emplace_back(work, t);
        for (auto &x : th) x.join();
    }
    return *std::min_element(found.begin(), found.end());
}

// fn(begin, end, t) over [0, n) split into contiguous chunks on host threads
template <class F>
static void parallel_chunks(uint32_t n, uint32_t T, const F &fn)
{
    if (T <= 1) {
        fn(0u, n, 0u);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(T);
    for (uint32_t t = 0; t < T; ++t)
        th.emplace_back(fn, (uint32_t)((uint64_t)n * t / T), (uint32_t)((uint64_t)n * (t + 1) / T), t);
    for (auto &x : th) x.join();
}

static uint32_t host_threads(uint32_t n)
{
    return n < (1u << 16) ? 1u : std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
}

// Every per-row check of create's inputs runs in one pass over the rows on host
// threads (each thread a contiguous range), recording per thread the first bad
// row of each check; validate() then reports errors in a fixed order.  A row's
// edges are read only when rp[q] <= rp[q+1] <= rp[n], i.e. inside col; NULL
// arrays are skipped (validate reports them).  Needs g, a non-NULL and
// 0 < n_agents < 2^31, n_nets <= DEABM_MAX_NETS.
struct RowFirsts {
    uint32_t dec[DEABM_MAX_NETS], col[DEABM_MAX_NETS], occ, age, stage, qt;
};

static std::vector<RowFirsts> scan_rows(const deabm_graph *g, const deabm_agents *a)
{
    const uint32_t n = g->n_agents;
    const bool occ_arrays = g->n_occ && g->n_occ < (1u << 31) && g->occ_group && g->occ_k;
    using Firsts = RowFirsts;
    const uint32_t T = host_threads(n);
    std::vector<Firsts> found(T);
    parallel_chunks(n, T, [&](uint32_t b, uint32_t e, uint32_t t) {
        Firsts f;
        for (uint32_t k = 0; k < DEABM_MAX_NETS; ++k) f.dec[k] = f.col[k] = n;
        f.occ = f.age = f.stage = f.qt = n;
        for (uint32_t k = 0; k < g->n_nets; ++k) {
            const uint32_t *rp = g->row_ptr[k], *col = g->col[k];
            if (!rp) continue;
            const uint32_t last = rp[n];
            const bool cols = col != nullptr || last == 0;
            for (uint32_t q = b; q < e; ++q) {
                const uint32_t lo = rp[q], hi = rp[q + 1];
                if (hi < lo) {
                    if (f.dec[k] == n) f.dec[k] = q;
                    continue;
                }
                if (!cols || hi > last || f.col[k] < n) continue;
                uint32_t bad = 0;
                for (uint32_t x = lo; x < hi; ++x) bad |= (uint32_t)(col[x] >= n) | (uint32_t)(col[x] == q);
                if (bad) f.col[k] = q;
            }
        }
        for (uint32_t q = b; q < e; ++q) {
            if (occ_arrays && f.occ == n && g->occ_group[q] >= g->n_occ) f.occ = q;
            if (a->age_bin && f.age == n && a->age_bin[q] >= DEABM_N_AGE) f.age = q;
            if (a->stage && f.stage == n && (a->stage[q] < 0 || a->stage[q] >= DEABM_N_STAGE)) f.stage = q;
            if (a->qt && f.qt == n && (a->qt[q] & 0x80u) != 0) f.qt = q;
        }
        found[t] = f;
    });
    return found;
}

// Host validation of create's inputs, before they are used: DEABM_OK or the
// first error in a fixed order.  scanned: the rows already scanned by scan_rows
// (create runs the scan on its own thread while the CSR goes up), else scanned here.
static int validate(deabm_ctx *ctx, const deabm_graph *g, const deabm_agents *a, const deabm_params *p,
                    uint32_t n_rep, const float *rep_params, const std::vector<RowFirsts> *scanned = nullptr)
{
    if (!g || !a || !p) return fail(ctx, DEABM_EINVAL, "graph, agents and params are required");
    const uint32_t n = g->n_agents;
    if (n == 0 || n >= (1u << 31)) return fail(ctx, DEABM_EINVAL, "n_agents must be in [1, 2^31)");
    if (g->n_nets > DEABM_MAX_NETS) return fail(ctx, DEABM_EINVAL, "n_nets > %d", DEABM_MAX_NETS);
    if (!(g->rand_mean >= 0.0f) || g->rand_mean > 1e3f) return fail(ctx, DEABM_EINVAL, "rand_mean out of range");
    if (g->rand_by_age > 1) return fail(ctx, DEABM_EINVAL, "rand_by_age must be 0 or 1");
    if (g->rand_by_age)
        for (int q = 0; q < DEABM_N_AGE; ++q)
            if (!(g->rand_mean_age[q] >= 0.0f) || g->rand_mean_age[q] > 1e3f)
                return fail(ctx, DEABM_EINVAL, "rand_mean_age[%d] out of range", q);
    if (poisson_on(g) && n < 2) return fail(ctx, DEABM_EINVAL, "the random network needs >= 2 agents");
    if ((uint64_t)n * n_rep >= (1ull << 40)) return fail(ctx, DEABM_EINVAL, "n_agents * n_rep too large");
    if (g->rand_ws) {
        if (g->rand_ws != 1) return fail(ctx, DEABM_EINVAL, "rand_ws must be 0 or 1");
        if (g->rand_ws_k < 2 || g->rand_ws_k > 16 || g->rand_ws_k % 2)
            return fail(ctx, DEABM_EINVAL, "rand_ws_k must be even, 2..16");
        if (!(g->rand_ws_beta >= 0.0f && g->rand_ws_beta <= 1.0f))
            return fail(ctx, DEABM_EINVAL, "rand_ws_beta must be in [0,1]");
        if (n < 2) return fail(ctx, DEABM_EINVAL, "the random network needs >= 2 agents");
        if ((uint64_t)n * (g->rand_ws_k / 2) >= (1ull << 31))
            return fail(ctx, DEABM_EINVAL, "n_agents * rand_ws_k / 2 must be < 2^31");
    }
    using Firsts = RowFirsts;
    const std::vector<Firsts> found = scanned ? *scanned : scan_rows(g, a);
    auto first = [&](uint32_t Firsts::*m) {
        uint32_t v = n;
        for (const Firsts &f : found) v = std::min(v, f.*m);
        return v;
    };
    for (uint32_t k = 0; k < g->n_nets; ++k) {
        const uint32_t *rp = g->row_ptr[k], *col = g->col[k];
        if (!rp) return fail(ctx, DEABM_EINVAL, "row_ptr[%u] is NULL", k);
        if (rp[0] != 0) return fail(ctx, DEABM_EINVAL, "row_ptr[%u][0] != 0", k);
        uint32_t j = n;
        for (const Firsts &f : found) j = std::min(j, f.dec[k]);
        if (j < n) return fail(ctx, DEABM_EINVAL, "row_ptr[%u] decreases at row %u", k, j);
        if (rp[n] > 0 && !col) return fail(ctx, DEABM_EINVAL, "col[%u] is NULL", k);
        for (const Firsts &f : found) j = std::min(j, f.col[k]);
        if (j < n)
            for (uint32_t e = rp[j]; e < rp[j + 1]; ++e) {
                if (col[e] >= n) return fail(ctx, DEABM_EINVAL, "col[%u][%u] = %u >= n_agents", k, e, col[e]);
                if (col[e] == j) return fail(ctx, DEABM_EINVAL, "self-loop at row %u of network %u", j, k);
            }
    }
    if (g->n_occ) {
        if (g->n_nets >= DEABM_MAX_NETS)
            return fail(ctx, DEABM_EINVAL, "daily occupation networks take weight B_net[n_nets]: n_nets must be <= %d",
                        DEABM_MAX_NETS - 1);
        if (!g->occ_group || !g->occ_k) return fail(ctx, DEABM_EINVAL, "occ_group and occ_k are required when n_occ > 0");
        if (g->n_occ >= (1u << 31)) return fail(ctx, DEABM_EINVAL, "n_occ too large");
        if (g->occ_lattice > 1) return fail(ctx, DEABM_EINVAL, "occ_lattice must be 0 or 1");
        if (!(g->occ_rewire >= 0.0f && g->occ_rewire <= 1.0f))
            return fail(ctx, DEABM_EINVAL, "occ_rewire must be in [0,1]");
        for (uint32_t q = 0; q < g->n_occ; ++q)
            if (g->occ_k[q] > DEABM_POIS_CAP)
                return fail(ctx, DEABM_EINVAL, "occ_k[%u] = %u > %d", q, g->occ_k[q], DEABM_POIS_CAP);
        const uint32_t j = first(&Firsts::occ);
        if (j < n) return fail(ctx, DEABM_EINVAL, "occ_group[%u] = %u >= n_occ", j, g->occ_group[j]);
    }
    if (!a->age_bin) return fail(ctx, DEABM_EINVAL, "age_bin is required");
    uint32_t jb = first(&Firsts::age);
    if (jb < n) return fail(ctx, DEABM_EINVAL, "age_bin[%u] = %u > 8", jb, a->age_bin[jb]);
    jb = first(&Firsts::stage);
    if (jb < n) return fail(ctx, DEABM_EINVAL, "stage[%u] = %d is not a stage code", jb, a->stage[jb]);
    jb = first(&Firsts::qt);
    if (jb < n) return fail(ctx, DEABM_EINVAL, "qt[%u] has bit 7 set", jb);
    if (a->n_seed && !a->seed_ids) return fail(ctx, DEABM_EINVAL, "seed_ids is NULL");
    for (uint32_t q = 0; q < a->n_seed; ++q)
        if (a->seed_ids[q] >= n) return fail(ctx, DEABM_EINVAL, "seed_ids[%u] >= n_agents", q);
    if (p->inf_len == 0 || p->inf_len > DEABM_MAX_INF_LEN) return fail(ctx, DEABM_EINVAL, "inf_len must be 1..64");
    for (int c = 0; c < DEABM_N_CLASS; ++c)
        if (!(p->inf_shape[c] > 0.0) || !(p->inf_scale[c] > 0.0))
            return fail(ctx, DEABM_EINVAL, "gamma shape and scale must be > 0");
    if (!(p->dt >= 0.0f)) return fail(ctx, DEABM_EINVAL, "dt must be >= 0");
    for (int q = 0; q < DEABM_N_AGE; ++q)
        if (!prob_ok(p->p_asym[q]) || !prob_ok(p->p_sev[q]) || !prob_ok(p->p_hosp[q]) || !prob_ok(p->p_icu[q]) ||
            !prob_ok(p->p_death[q]))
            return fail(ctx, DEABM_EINVAL, "branch probabilities must be in [0,1]");
    for (int st = DEABM_ASYM; st <= DEABM_ICU; ++st)
        for (int q = 0; q < DEABM_N_AGE; ++q)
            if (p->dur_lo[st][q] < 1 || p->dur_hi[st][q] < p->dur_lo[st][q])
                return fail(ctx, DEABM_EINVAL, "stage %d durations need 1 <= lo <= hi", st);
    if (p->test_lo < 1 || p->test_hi > 7 || p->test_lo > p->test_hi)
        return fail(ctx, DEABM_EINVAL, "test delays need 1 <= test_lo <= test_hi <= 7");
    if (p->quar_days > 15) return fail(ctx, DEABM_EINVAL, "quar_days must be <= 15");
    if (!prob_ok(p->test_sens) || !prob_ok(p->q_dropout) || !prob_ok(p->vax_eff1) || !prob_ok(p->vax_eff2) ||
        !(p->vax_rate >= 0.0 && p->vax_rate <= 1.0))
        return fail(ctx, DEABM_EINVAL, "probabilities and rates must be in [0,1]");
    if (p->vax_on && (p->vax_onset < 1 || p->dose2_delay < 1))
        return fail(ctx, DEABM_EINVAL, "vax_onset and dose2_delay must be >= 1");
    if (p->vax_strategy > 3 || p->elderly_bin > 9)
        return fail(ctx, DEABM_EINVAL, "vax_strategy must be 0..3 and elderly_bin 0..9");
    if (p->den_on) {
        if (!p->test_on) return fail(ctx, DEABM_EINVAL, "exposure notification needs test_on");
        if (p->den_window < 1 || p->den_window > 64) return fail(ctx, DEABM_EINVAL, "den_window must be 1..64");
        if (!prob_ok(p->den_adoption) || !prob_ok(p->den_compliance))
            return fail(ctx, DEABM_EINVAL, "den_adoption and den_compliance must be in [0,1]");
    }
    if (n_rep < 1 || n_rep > 1024) return fail(ctx, DEABM_EINVAL, "n_rep must be in 1..1024");
    if (rep_params)
        for (uint32_t b = 0; b < n_rep; ++b) {
            const float d = rep_params[b * DEABM_N_REP_PARAMS + 13];
            if (!(d >= 1.0f && d <= 30000.0f) || d != std::floor(d))
                return fail(ctx, DEABM_EINVAL, "replicate %u: dose2_delay must be a whole number of days >= 1", b);
        }
    return DEABM_OK;
}

// ---------------------------------------------------------------- locality order
// Device scratch freed when the creating call returns, on every path.
struct DevScratch {
    std::vector<void *> ptrs;
    ~DevScratch()
    {
        for (void *q : ptrs) (void)cudaFree(q);
    }
};

template <class T>
static int scratch_alloc(deabm_ctx *ctx, DevScratch &sc, T **out, size_t count)
{
    void *ptr = nullptr;
    const cudaError_t e =
        injected_alloc_failure() ? cudaErrorMemoryAllocation : cudaMalloc(&ptr, (count ? count : 1) * sizeof(T));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ctx, DEABM_ENOMEM, "cudaMalloc of %zu scratch bytes failed: %s", count * sizeof(T),
                    cudaGetErrorString(e));
    }
    sc.ptrs.push_back(ptr);
    *out = (T *)ptr;
    return DEABM_OK;
}

// The internal order on the host (row -> caller id), read back from the device on
// first use: only the readbacks of host-side gathers need it.
static int host_order(deabm_ctx *ctx)
{
    if (!ctx->relabel || !ctx->new2orig.empty()) return DEABM_OK;
    std::vector<uint32_t> v(ctx->n);
    CU(ctx, cudaMemcpyAsync(v.data(), ctx->orig_id, sizeof(uint32_t) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->new2orig.swap(v);
    return DEABM_OK;
}

// Rounds of min-label propagation that fix the locality order (even).
constexpr uint32_t kLocalityRounds = 8;

// ---------------------------------------------------------------- occupation order
// Occupations in id order, the members of each in ascending caller id: the
// member in place r of occupation g is internal row start[g] + r, which is how
// the day kernels map a drawn place to a row.
static void occupation_order(const deabm_graph *g, std::vector<uint32_t> &order, std::vector<uint32_t> &start)
{
    const uint32_t n = g->n_agents, G = g->n_occ;
    start.assign((size_t)G + 1, 0);
    for (uint32_t j = 0; j < n; ++j) start[g->occ_group[j] + 1]++;
    for (uint32_t q = 0; q < G; ++q) start[q + 1] += start[q];
    std::vector<uint32_t> fill(start.begin(), start.end() - 1);
    order.resize(n);
    for (uint32_t j = 0; j < n; ++j) order[fill[g->occ_group[j]]++] = j;
}

// per-replicate parameter blocks: rep_params rows override the base parameters
static void build_reps(const deabm_params *p, uint32_t n_rep, const float *rep_params, const uint64_t *rep_seeds,
                       std::vector<Rep> &reps)
{
    reps.assign(n_rep, Rep{});
    for (uint32_t b = 0; b < n_rep; ++b) {
        Rep &R = reps[b];
        float Rv = p->R, Bn[DEABM_MAX_NETS], Br = p->B_rand, Sa[DEABM_N_AGE];
        uint32_t delay = p->dose2_delay;
        for (int k = 0; k < DEABM_MAX_NETS; ++k) Bn[k] = p->B_net[k];
        for (int q = 0; q < DEABM_N_AGE; ++q) Sa[q] = p->S_age[q];
        if (rep_params) {
            const float *rp = rep_params + (size_t)b * DEABM_N_REP_PARAMS;
            Rv = rp[0]; Bn[0] = rp[1]; Bn[1] = rp[2]; Br = rp[3];
            for (int q = 0; q < DEABM_N_AGE; ++q) Sa[q] = rp[4 + q];
            delay = (uint32_t)rp[13];
        }
        volatile float rv = Rv, ib = p->inv_Ibar;  // one FP32 product, no contraction
        R.cR = rv * ib;
        for (int k = 0; k < DEABM_MAX_NETS; ++k) R.B_net[k] = Bn[k];
        R.B_rand = Br;
        for (int q = 0; q < DEABM_N_AGE; ++q) R.S_age[q] = Sa[q];
        R.dose2_delay = delay;
        R.seed = rep_seeds ? rep_seeds[b] : p->seed;
        round_keys(R.seed, R.rk);
    }
}

// ---------------------------------------------------------------- exposure notification
// The contact ring (den_window days x den_slots words per app holder) is sized
// to the app holders drawn: at creation, and again at a reset whose seed draws
// more of them than it has room for.
static int den_ring_reserve(deabm_ctx *ctx, KParams &K)
{
    if (ctx->den_ring && K.n_app <= ctx->den_ring_cap) {
        K.den_ring = ctx->den_ring;
        return DEABM_OK;
    }
    if (ctx->den_ring) {  // too small for this draw: replaced (nothing in flight reads it)
        CU(ctx, cudaStreamSynchronize(ctx->stream));
        auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), (void *)ctx->den_ring);
        if (it != ctx->allocs.end()) ctx->allocs.erase(it);
        (void)cudaFree(ctx->den_ring);
        ctx->den_ring = nullptr;
        ctx->den_ring_cap = 0;
        K.den_ring = nullptr;
    }
    const size_t cap = K.n_app;
    const size_t bytes = std::max<size_t>(1, (size_t)K.den_window * K.den_slots * cap) * sizeof(uint32_t);
    void *ptr = nullptr;
    cudaError_t e = injected_alloc_failure() ? cudaErrorMemoryAllocation : cudaMalloc(&ptr, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ctx, DEABM_ENOMEM, "cudaMalloc of %zu bytes (contact ring) failed: %s", bytes, cudaGetErrorString(e));
    }
    ctx->allocs.push_back(ptr);
    ctx->den_ring = (uint32_t *)ptr;
    ctx->den_ring_cap = cap;
    K.den_ring = ctx->den_ring;
    return DEABM_OK;
}

// The app holders drawn on the device, listed in row order with each row's rank
// (for the notification pass and the contact ring); sets K.n_app.
static int den_list_apps(deabm_ctx *ctx, KParams &K)
{
    const uint32_t n = ctx->n;
    std::vector<uint8_t> fl(n);
    CU(ctx, cudaMemcpyAsync(fl.data(), ctx->S.flags, n, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<uint32_t> rows, rank(n, 0xFFFFFFFFu);
    rows.reserve(n);
    for (uint32_t j = 0; j < n; ++j)
        if (fl[j] & DEABM_FL_APP) {
            rank[j] = (uint32_t)rows.size();
            rows.push_back(j);
        }
    K.n_app = (uint32_t)rows.size();
    if (int r = den_ring_reserve(ctx, K)) return r;
    if (K.n_app)
        CU(ctx, cudaMemcpyAsync(ctx->app_rows, rows.data(), sizeof(uint32_t) * K.n_app, cudaMemcpyHostToDevice,
                                ctx->stream));
    CU(ctx, cudaMemcpyAsync(ctx->app_rank, rank.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));  // the staging vectors go out of scope
    return DEABM_OK;
}

// ---------------------------------------------------------------- creation
static int create_impl(const deabm_graph *g, const deabm_agents *a, const deabm_params *p, uint32_t n_rep,
                       const float *rep_params, const uint64_t *rep_seeds, void *stream, deabm_ctx **out)
{
    if (!out) return fail(nullptr, DEABM_EINVAL, "out is NULL");
    *out = nullptr;
    deabm_ctx *ctx = new (std::nothrow) deabm_ctx();
    if (!ctx) return fail(nullptr, DEABM_ENOMEM, "host allocation failed");
    // The row scan of the inputs (most of validation) runs on its own host thread
    // while the stored networks go up to the device; the scan is reported before
    // anything reads the inputs on the host or the device.  Inputs too broken to
    // size the uploads are validated first, in full.
    bool overlap = g && a && p && g->n_agents > 0 && g->n_agents < (1u << 31) && g->n_nets <= DEABM_MAX_NETS;
    for (uint32_t k = 0; overlap && k < g->n_nets; ++k)
        overlap = g->row_ptr[k] && (g->col[k] || g->row_ptr[k][g->n_agents] == 0);
    std::vector<RowFirsts> scanned;
    struct Joined {
        std::thread t;
        ~Joined()
        {
            if (t.joinable()) t.join();
        }
    } scan;
    if (overlap) scan.t = std::thread([&] { scanned = scan_rows(g, a); });
    auto validated = [&]() -> int {
        if (scan.t.joinable()) scan.t.join();
        return validate(ctx, g, a, p, n_rep, rep_params, &scanned);
    };
    int rc = overlap ? DEABM_OK : validate(ctx, g, a, p, n_rep, rep_params);
    if (rc == DEABM_OK) {
        rc = [&]() -> int {
            ctx->stream = (cudaStream_t)stream;
            const uint32_t n = g->n_agents;
            const size_t nb = (size_t)n * n_rep;
            ctx->n = n;
            arena_plan(ctx, n, n_rep);
            ctx->n_nets = g->n_nets;
            ctx->n_rep = n_rep;
            ctx->max_steps = p->max_steps ? p->max_steps : 1024u;
            ctx->keep_lambda = p->keep_lambda != 0;
            cudaStream_t s = ctx->stream;
            int r;
            ctx->relabel = (p->locality_order != 0 && g->n_nets > 0) || g->n_occ > 0;
            // the stored networks go to the device as given: in place when the
            // numbering stays, else into scratch to be renumbered there
            DevScratch sc;
            uint32_t *src_rp[DEABM_MAX_NETS] = {}, *src_col[DEABM_MAX_NETS] = {};
            uint32_t best = 0;
            for (uint32_t k = 0; k < g->n_nets; ++k) {
                const uint32_t E = g->row_ptr[k][n];
                ctx->static_edges += E;
                if (E > g->row_ptr[best][n]) best = k;
                if ((r = dalloc(ctx, &ctx->row_ptr[k], (size_t)n + 1))) return r;
                if ((r = dalloc(ctx, &ctx->col[k], E))) return r;
                src_rp[k] = ctx->row_ptr[k];
                src_col[k] = ctx->col[k];
                if (ctx->relabel) {
                    if ((r = scratch_alloc(ctx, sc, &src_rp[k], (size_t)n + 1))) return r;
                    if ((r = scratch_alloc(ctx, sc, &src_col[k], E))) return r;
                }
                CU(ctx, cudaMemcpyAsync(src_rp[k], g->row_ptr[k], sizeof(uint32_t) * ((size_t)n + 1),
                                        cudaMemcpyHostToDevice, s));
                if (E) CU(ctx, cudaMemcpyAsync(src_col[k], g->col[k], sizeof(uint32_t) * E, cudaMemcpyHostToDevice, s));
            }
            if (overlap && (r = validated())) return r;  // the uploads above read nothing else
            std::vector<uint32_t> occ_start;
            uint32_t *d_o2n = nullptr;
            if (ctx->relabel) {
                if ((r = dalloc(ctx, &ctx->orig_id, n))) return r;
                if ((r = scratch_alloc(ctx, sc, &d_o2n, n))) return r;
            }
            if (g->n_occ) {
                occupation_order(g, ctx->new2orig, occ_start);
                CU(ctx, cudaMemcpyAsync(ctx->orig_id, ctx->new2orig.data(), sizeof(uint32_t) * n,
                                        cudaMemcpyHostToDevice, s));
            } else if (ctx->relabel) {
                // groups by the smallest id reaching them along the densest network's
                // in-edges, ids ascending inside a group: labels and order on the device
                uint32_t *label, *tmp, *changed;
                if ((r = scratch_alloc(ctx, sc, &label, n))) return r;
                if ((r = scratch_alloc(ctx, sc, &tmp, std::max<size_t>(n, order_scratch_words(n))))) return r;
                if ((r = scratch_alloc(ctx, sc, &changed, 1))) return r;
                CU(ctx, launch_locality_labels(src_rp[best], src_col[best], n, kLocalityRounds, label, tmp, changed, s));
                CU(ctx, launch_order_by_label(label, n, ctx->orig_id, tmp, s));
            }
            if (ctx->relabel) {
                uint32_t *d_scan;
                if ((r = scratch_alloc(ctx, sc, &d_scan, scan_scratch_words((size_t)n + 1)))) return r;
                CU(ctx, launch_invert(ctx->orig_id, n, d_o2n, s));
                // rows in internal order, each row's edges kept in the caller's order
                for (uint32_t k = 0; k < g->n_nets; ++k)
                    CU(ctx, launch_csr_renumber(src_rp[k], src_col[k], ctx->orig_id, d_o2n, n, ctx->row_ptr[k],
                                                ctx->col[k], d_scan, s));
            }
            if (ctx->relabel && (poisson_on(g) || g->rand_ws) && n_rep > 1) {  // batched: caller id -> row map
                if ((r = dalloc(ctx, &ctx->row_of, n))) return r;
                CU(ctx, cudaMemcpyAsync(ctx->row_of, d_o2n, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
            }
            CU(ctx, cudaStreamSynchronize(s));  // host staging and device scratch end here
            if (g->n_occ) {
                ctx->n_occ = g->n_occ;
                std::vector<uint32_t> gid(n);
                for (uint32_t q = 0; q < n; ++q) gid[q] = g->occ_group[ctx->new2orig[q]];
                if ((r = dalloc(ctx, &ctx->occ_gid, n))) return r;
                if ((r = dalloc(ctx, &ctx->occ_start, (size_t)g->n_occ + 1))) return r;
                if ((r = dalloc(ctx, &ctx->occ_k, g->n_occ))) return r;
                CU(ctx, cudaMemcpyAsync(ctx->occ_gid, gid.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice, s));
                CU(ctx, cudaMemcpyAsync(ctx->occ_start, occ_start.data(), sizeof(uint32_t) * ((size_t)g->n_occ + 1),
                                        cudaMemcpyHostToDevice, s));
                CU(ctx, cudaMemcpyAsync(ctx->occ_k, g->occ_k, g->n_occ, cudaMemcpyHostToDevice, s));
                CU(ctx, cudaStreamSynchronize(s));  // gid is a local staging vector
            }
            if ((r = dalloc(ctx, &ctx->age, n))) return r;
            if ((r = dalloc(ctx, &ctx->dose1, n))) return r;
            if ((r = dalloc(ctx, &ctx->S.stage, nb))) return r;
            if ((r = dalloc(ctx, &ctx->S.timer, nb))) return r;
            if ((r = dalloc(ctx, &ctx->S.tinf, nb))) return r;
            if ((r = dalloc(ctx, &ctx->S.flags, nb))) return r;
            if ((r = dalloc(ctx, &ctx->S.qt, nb))) return r;
            if ((r = dalloc(ctx, &ctx->inf[0], nb))) return r;
            if ((r = dalloc(ctx, &ctx->inf[1], nb))) return r;
            if (ctx->relabel && (poisson_on(g) || g->rand_ws) && n_rep == 1) {
                if ((r = dalloc(ctx, &ctx->inf_rand[0], nb))) return r;
                if ((r = dalloc(ctx, &ctx->inf_rand[1], nb))) return r;
            }
            if (ctx->keep_lambda) {
                if ((r = dalloc(ctx, &ctx->lam, nb))) return r;
                if ((r = dalloc(ctx, &ctx->p, nb))) return r;
                CU(ctx, cudaMemsetAsync(ctx->lam, 0, sizeof(float) * nb, s));
                CU(ctx, cudaMemsetAsync(ctx->p, 0, sizeof(float) * nb, s));
            }
            if ((r = dalloc(ctx, &ctx->tab, 1))) return r;
            if ((r = dalloc(ctx, &ctx->rep, n_rep))) return r;
            const size_t days = ctx->max_steps;
            if ((r = dalloc(ctx, &ctx->C.new_inf, days * n_rep))) return r;
            if ((r = dalloc(ctx, &ctx->C.hist, days * n_rep * DEABM_N_STAGE))) return r;
            if ((r = dalloc(ctx, &ctx->C.msgs, days))) return r;
        if ((r = dalloc(ctx, &ctx->C.gath, days))) return r;
            if ((r = dalloc(ctx, &ctx->C.den, days * n_rep))) return r;
            CU(ctx, cudaMemsetAsync(ctx->C.den, 0, sizeof(int32_t) * days * n_rep, s));
            if (p->den_on) {
                if ((r = dalloc(ctx, &ctx->den_pos, days))) return r;
                CU(ctx, cudaMemsetAsync(ctx->den_pos, 0, sizeof(int32_t) * days, s));
                if (n_rep == 1) {
                    if ((r = dalloc(ctx, &ctx->den_bits, ((size_t)n + 31) / 32))) return r;
                    if (ctx->relabel && (r = dalloc(ctx, &ctx->den_bits_orig, ((size_t)n + 31) / 32))) return r;
                    if ((r = dalloc(ctx, &ctx->app_rows, n))) return r;
                    if ((r = dalloc(ctx, &ctx->app_rank, n))) return r;
                } else {  // positives of the day: one word per (row, 32 columns)
                    if ((r = dalloc(ctx, &ctx->den_bits, (size_t)n * ((n_rep + 31) / 32)))) return r;
                }
            }
            CU(ctx, cudaMemsetAsync(ctx->C.new_inf, 0, sizeof(int32_t) * days * n_rep, s));
            CU(ctx, cudaMemsetAsync(ctx->C.hist, 0, sizeof(int32_t) * days * n_rep * DEABM_N_STAGE, s));
            CU(ctx, cudaMemsetAsync(ctx->C.msgs, 0, sizeof(unsigned long long) * days, s));
        CU(ctx, cudaMemsetAsync(ctx->C.gath, 0, sizeof(unsigned long long) * days, s));

            // agents: [N] -> [N][n_rep] in internal order, each agent's initial state
            // repeated per replicate.  Caller arrays go up as given and are put in
            // place on the device; absent ones are zero.
            uint16_t *d_in = nullptr;  // caller-order staging, n 2-byte words
            if ((r = scratch_alloc(ctx, sc, &d_in, n))) return r;
            const uint32_t *perm = ctx->relabel ? ctx->orig_id : nullptr;
            auto put = [&](void *dst, const void *src, uint32_t elem, uint32_t reps) -> int {
                if (!src) {
                    CU(ctx, cudaMemsetAsync(dst, 0, (size_t)n * reps * elem, s));
                } else if (!perm && reps == 1) {
                    CU(ctx, cudaMemcpyAsync(dst, src, (size_t)n * elem, cudaMemcpyHostToDevice, s));
                } else {
                    CU(ctx, cudaMemcpyAsync(d_in, src, (size_t)n * elem, cudaMemcpyHostToDevice, s));
                    CU(ctx, launch_from_caller(dst, d_in, perm, n, reps, elem, false, s));
                }
                return DEABM_OK;
            };
            if ((r = put(ctx->age, a->age_bin, 1, 1))) return r;
            if ((r = put(ctx->S.stage, a->stage, 1, n_rep))) return r;
            if ((r = put(ctx->S.timer, a->timer, 2, n_rep))) return r;
            if ((r = put(ctx->S.tinf, a->tinf, 2, n_rep))) return r;
            if ((r = put(ctx->S.flags, a->flags, 1, n_rep))) return r;
            if ((r = put(ctx->S.qt, a->qt, 1, n_rep))) return r;
            // keep the initial state for deabm_reset
            if ((r = dalloc(ctx, &ctx->S0.stage, nb))) return r;
            if ((r = dalloc(ctx, &ctx->S0.timer, nb))) return r;
            if ((r = dalloc(ctx, &ctx->S0.tinf, nb))) return r;
            if ((r = dalloc(ctx, &ctx->S0.flags, nb))) return r;
            if ((r = dalloc(ctx, &ctx->S0.qt, nb))) return r;
            CU(ctx, cudaMemcpyAsync(ctx->S0.stage, ctx->S.stage, nb, cudaMemcpyDeviceToDevice, s));
            CU(ctx, cudaMemcpyAsync(ctx->S0.timer, ctx->S.timer, nb * 2, cudaMemcpyDeviceToDevice, s));
            CU(ctx, cudaMemcpyAsync(ctx->S0.tinf, ctx->S.tinf, nb * 2, cudaMemcpyDeviceToDevice, s));
            CU(ctx, cudaMemcpyAsync(ctx->S0.flags, ctx->S.flags, nb, cudaMemcpyDeviceToDevice, s));
            CU(ctx, cudaMemcpyAsync(ctx->S0.qt, ctx->S.qt, nb, cudaMemcpyDeviceToDevice, s));
            ctx->base = *p;
            if (p->vax_strategy != 0) {
                std::vector<int16_t> d1(nb, kNever), d2(nb, kNever);
                if ((a->dose1_day || a->dose2_day) && (r = host_order(ctx))) return r;
                auto orig_of = [&](uint32_t q) { return ctx->relabel ? ctx->new2orig[q] : q; };
                for (uint32_t q = 0; q < n; ++q)  // the caller's dose days, the same in every replicate
                    for (uint32_t b = 0; b < n_rep; ++b) {
                        if (a->dose1_day) d1[(size_t)q * n_rep + b] = a->dose1_day[orig_of(q)];
                        if (a->dose2_day) d2[(size_t)q * n_rep + b] = a->dose2_day[orig_of(q)];
                    }
                if ((r = dalloc(ctx, &ctx->S.vd1, nb))) return r;
                if ((r = dalloc(ctx, &ctx->S.vd2, nb))) return r;
                if ((r = dalloc(ctx, &ctx->S0.vd1, nb))) return r;
                if ((r = dalloc(ctx, &ctx->S0.vd2, nb))) return r;
                if ((r = dalloc(ctx, &ctx->vax_cls, nb))) return r;
                if ((r = dalloc(ctx, &ctx->vax_dose, nb))) return r;
                if ((r = dalloc(ctx, &ctx->vax_scratch, n_rep > 1 ? vax_select_batch_scratch_words(n, n_rep)
                                                                    : vax_select_scratch_words(n))))
                    return r;
                CU(ctx, cudaMemcpyAsync(ctx->S0.vd1, d1.data(), nb * 2, cudaMemcpyHostToDevice, s));
                CU(ctx, cudaMemcpyAsync(ctx->S0.vd2, d2.data(), nb * 2, cudaMemcpyHostToDevice, s));
                CU(ctx, cudaMemcpyAsync(ctx->S.vd1, d1.data(), nb * 2, cudaMemcpyHostToDevice, s));
                CU(ctx, cudaMemcpyAsync(ctx->S.vd2, d2.data(), nb * 2, cudaMemcpyHostToDevice, s));
                CU(ctx, cudaStreamSynchronize(s));
                ctx->vax_supply = (uint32_t)std::floor(p->vax_rate * (double)n);
            }

            // per-replicate parameters
            std::vector<Rep> reps;
            build_reps(p, n_rep, rep_params, rep_seeds, reps);
            CU(ctx, cudaMemcpyAsync(ctx->rep, reps.data(), sizeof(Rep) * n_rep, cudaMemcpyHostToDevice, s));

            // host-side integer tables (thresholds are exact: p * 2^32 then floor)
            Tables T;
            std::memset(&T, 0, sizeof T);
            poisson_tables(g, T);
            for (int q = 0; q < DEABM_N_AGE; ++q) {
                T.thr_asym[q] = threshold(p->p_asym[q]);
                T.thr_sev[q] = threshold(p->p_sev[q]);
                T.thr_branch[DEABM_SEV][q] = threshold(p->p_hosp[q]);
                T.thr_branch[DEABM_HOSP][q] = threshold(p->p_icu[q]);
                T.thr_branch[DEABM_ICU][q] = threshold(p->p_death[q]);
            }
            std::memcpy(T.dur_lo, p->dur_lo, sizeof T.dur_lo);
            std::memcpy(T.dur_hi, p->dur_hi, sizeof T.dur_hi);
            CU(ctx, cudaMemcpyAsync(ctx->tab, &T, sizeof T, cudaMemcpyHostToDevice, s));
            CU(ctx, cudaStreamSynchronize(s));  // host staging buffers above go out of scope

            // device-built tables: infectiousness (FP64 integrals), vaccination days
            double *d_gamma;
            float *d_A;
            uint32_t *d_scratch, *d_ids = nullptr;
            if ((r = dalloc(ctx, &d_gamma, 6))) return r;
            if ((r = dalloc(ctx, &d_A, 3))) return r;
            if ((r = dalloc(ctx, &d_scratch, dose1_scratch_words(n)))) return r;
            const double gs[6] = {p->inf_shape[0], p->inf_shape[1], p->inf_shape[2],
                                  p->inf_scale[0], p->inf_scale[1], p->inf_scale[2]};
            CU(ctx, cudaMemcpyAsync(d_gamma, gs, sizeof gs, cudaMemcpyHostToDevice, s));
            CU(ctx, cudaMemcpyAsync(d_A, p->A_class, sizeof(float) * 3, cudaMemcpyHostToDevice, s));
            CU(ctx, launch_inf_table(ctx->tab, d_gamma, d_A, p->inf_len, s));
            // the priority order is by the caller's ids: rank in caller order, then relabel
            const uint32_t per_day = p->vax_on ? (uint32_t)std::floor(p->vax_rate * (double)n) : 0u;
            if (ctx->relabel) {
                uint8_t *d_age_orig;
                int16_t *d_dose_orig;
                if ((r = dalloc(ctx, &d_age_orig, n))) return r;
                if ((r = dalloc(ctx, &d_dose_orig, n))) return r;
                CU(ctx, cudaMemcpyAsync(d_age_orig, a->age_bin, n, cudaMemcpyHostToDevice, s));
                CU(ctx, launch_dose1_days(d_age_orig, n, p->vax_start, per_day, d_dose_orig, d_scratch, s));
                CU(ctx, launch_gather_i16(ctx->dose1, d_dose_orig, ctx->orig_id, n, s));
            } else {
                CU(ctx, launch_dose1_days(ctx->age, n, p->vax_start, per_day, ctx->dose1, d_scratch, s));
            }

            KParams &K = ctx->kp;
            K.n = n;
            K.n_nets = g->n_nets;
            K.n_rep = n_rep;
            K.inf_len = p->inf_len;
            K.dt = p->dt;
            K.rand_on = poisson_on(g) ? 1u : 0u;
            K.rand_by_age = g->rand_by_age ? 1u : 0u;
            if (g->rand_ws) {  // the day's Watts-Strogatz random network, rebuilt before each day kernel
                K.wsg_on = 1;
                K.wsg_h = g->rand_ws_k / 2u;
                K.thr_wsg = threshold((double)g->rand_ws_beta);
                WsgBuffers &W = ctx->wsg;
                const size_t edges = (size_t)n * K.wsg_h;
                // with exposure notification the graphs of the look-back window are
                // kept (a ring of den_window days), one day's otherwise
                const uint32_t days_kept = p->den_on ? p->den_window : 1u;
                if ((r = dalloc(ctx, &W.rew, n))) return r;
                if ((r = dalloc(ctx, &W.far, edges))) return r;
                if ((r = dalloc(ctx, &W.ends, ((size_t)n + 3) * days_kept))) return r;
                if ((r = dalloc(ctx, &W.land, edges * days_kept))) return r;
                if ((r = dalloc(ctx, &W.scratch, wsg_scratch_words(n)))) return r;
                K.wsg_rew = W.rew;
                K.wsg_start = W.ends + 2;
                K.wsg_land = W.land;
                K.wsg_ends_ring = W.ends;
                K.wsg_land_ring = W.land;
                K.wsg_ring_days = days_kept;
            }
            for (uint32_t k = 0; k < DEABM_MAX_NETS; ++k) {
                K.row_ptr[k] = ctx->row_ptr[k];
                K.col[k] = ctx->col[k];
            }
            K.net_seed = p->net_seed;
            round_keys(p->net_seed, K.nrk);
            K.test_on = p->test_on;
            K.test_lo = p->test_lo;
            K.test_hi = p->test_hi;
            K.quar_on = p->quar_on;
            K.quar_days = p->quar_days;
            K.thr_sens = threshold(p->test_sens);
            K.thr_qdrop = threshold(p->q_dropout);
            K.vax_on = p->vax_on;
            K.vax_onset = p->vax_onset;
            K.thr_eff1 = threshold(p->vax_eff1);
            K.thr_eff2 = threshold(p->vax_eff2);
            K.tab = ctx->tab;
            K.rep = ctx->rep;
            set_pois32(K, T.pois);
            K.rep0 = reps[0];
            K.age = ctx->age;
            K.dose1_day = ctx->dose1;
            K.orig_id = ctx->relabel ? ctx->orig_id : nullptr;
            K.vax_strategy = p->vax_strategy;
            K.vax_nonsterile = p->vax_nonsterile ? 1u : 0u;
            K.dose_today = nullptr;
            K.n_occ = ctx->n_occ;
            K.occ_gid = ctx->occ_gid;
            K.occ_start = ctx->occ_start;
            K.occ_k = ctx->occ_k;
            K.occ_lattice = g->n_occ ? g->occ_lattice : 0u;
            K.thr_rewire = threshold((double)g->occ_rewire);
            K.den_on = p->den_on ? 1u : 0u;
            K.den_window = p->den_window;
            K.thr_comp = threshold(p->den_compliance);
            K.thr_adopt = threshold(p->den_adoption);
            K.den_bits = ctx->den_bits;
            K.den_bits_orig = ctx->den_bits_orig;
            K.den_pos = ctx->den_pos;
            K.den_slots = g->n_occ ? 32u : 16u;
            K.app_rows = ctx->app_rows;
            K.app_rank = ctx->app_rank;
            if (K.den_on) {  // app holders, part of the initial state kept for deabm_reset
                CU(ctx, launch_den_apps(K, ctx->S, s));
                CU(ctx, cudaMemcpyAsync(ctx->S0.flags, ctx->S.flags, nb, cudaMemcpyDeviceToDevice, s));
                if (n_rep == 1 && (r = den_list_apps(ctx, K))) return r;
            }

            if (a->n_seed) {
                if ((r = dalloc(ctx, &d_ids, a->n_seed))) return r;
                CU(ctx, cudaMemcpyAsync(d_ids, a->seed_ids, sizeof(uint32_t) * a->n_seed, cudaMemcpyHostToDevice, s));
                if (ctx->relabel) CU(ctx, launch_map_ids(d_ids, a->n_seed, d_o2n, s));
                CU(ctx, launch_seed(K, d_ids, a->n_seed, ctx->S, s));
                CU(ctx, cudaStreamSynchronize(s));
                ctx->seed_ids = d_ids;
                ctx->n_seed = a->n_seed;
            }
            CU(ctx, clear_next_buffers(ctx, nb));
            CU(ctx, launch_emit(K, ctx->S, ctx->inf[0], ctx->inf_rand[0], s));
            CU(ctx, cudaStreamSynchronize(s));
            return DEABM_OK;
        }();
        // a failure during the uploads, before the scan was reported: an invalid
        // input is the error to report
        if (rc != DEABM_OK && scan.t.joinable()) {
            const int v = validated();
            if (v != DEABM_OK) rc = v;
        }
    }
    if (rc != DEABM_OK) {
        std::string msg = ctx->err;
        deabm_destroy(ctx);
        g_err = msg;
        return rc;
    }
    *out = ctx;
    return DEABM_OK;
}

extern "C" int deabm_create(const deabm_graph *graph, const deabm_agents *agents, const deabm_params *params,
                            void *cuda_stream, deabm_ctx **out)
{
    return create_impl(graph, agents, params, 1u, nullptr, nullptr, cuda_stream, out);
}

extern "C" int deabm_create_batch(const deabm_graph *graph, const deabm_agents *agents, const deabm_params *base,
                                  uint32_t n_rep, const float *rep_params, const uint64_t *rep_seeds,
                                  void *cuda_stream, deabm_ctx **out)
{
    if (!rep_params || !rep_seeds) return fail(nullptr, DEABM_EINVAL, "rep_params and rep_seeds are required");
    return create_impl(graph, agents, base, n_rep, rep_params, rep_seeds, cuda_stream, out);
}

// ---------------------------------------------------------------- the day loop
// One day of a ragged batch (infectiousness buffer c read): the day's dose
// selection of each population under a priority strategy, then the day kernel.
static cudaError_t ragged_day(deabm_ctx *ctx, uint32_t day, int c)
{
    for (const auto &rv : ctx->ragged_vax) {
        if (day < rv.start) continue;
        const PopDesc &pd = ctx->pops[rv.q];
        StateRef Sp{ctx->S.stage + pd.base, ctx->S.timer + pd.base, ctx->S.tinf + pd.base,
                    ctx->S.flags + pd.base, ctx->S.qt + pd.base, ctx->S.vd1 + pd.base, ctx->S.vd2 + pd.base};
        cudaError_t e = launch_vax_select(pd.kp, day, rv.delay, rv.elderly, rv.supply, Sp, ctx->vax_cls + pd.base,
                                          ctx->vax_dose + pd.base, ctx->vax_scratch, ctx->stream);
        if (e != cudaSuccess) return e;
    }
    for (const auto &qw : ctx->ragged_wsg_bufs) {  // the day's Watts-Strogatz graph of each population that has one
        const KParams &kp = ctx->pops[qw.first].kp;
        WsgBuffers W = qw.second;
        cudaError_t e = cudaSuccess;
        if (kp.wsg_ring_days > 1) {  // with exposure notification: a ring of the window's graphs
            const uint32_t slot = day % kp.wsg_ring_days;
            W.ends += (size_t)slot * ((size_t)kp.n + 3);
            W.land += (size_t)slot * kp.n * kp.wsg_h;
            e = launch_wsg_slot(&ctx->d_pops[qw.first].kp, day, ctx->stream);
            if (e != cudaSuccess) return e;
        }
        e = launch_wsg_build(kp, day, W, ctx->stream);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = launch_step_ragged(ctx->d_pops, ctx->d_tiles, ctx->n_tiles, ctx->queue, day, ctx->inf[c],
                                       ctx->inf[c ^ 1], ctx->S, ctx->C, ctx->n_rep, ctx->grid, ctx->ragged_occ,
                                       ctx->ragged_wsg, !ctx->ragged_den.empty(), ctx->stream);
    // the notification pass of each population that has one, on its own slice
    // (one replicate column; its count goes to column q of [day][population])
    for (uint32_t q : ctx->ragged_den) {
        if (e != cudaSuccess) return e;
        const PopDesc &pd = ctx->pops[q];
        StateRef Sp{ctx->S.stage + pd.base, ctx->S.timer + pd.base, ctx->S.tinf + pd.base, ctx->S.flags + pd.base,
                    ctx->S.qt + pd.base};
        e = launch_den_batch(pd.kp, day, pd.row_of, Sp, ctx->C, ctx->n_rep, q, ctx->stream);
    }
    return e;
}

// The Watts-Strogatz graph of `day` built into its slot of the ring, and the
// day kernel's view of it (kp.wsg_start, kp.wsg_land) pointed there.
static cudaError_t wsg_day(deabm_ctx *ctx, KParams &kp, uint32_t day)
{
    const uint32_t slot = day % kp.wsg_ring_days;
    WsgBuffers W = ctx->wsg;
    W.ends += (size_t)slot * ((size_t)kp.n + 3);
    W.land += (size_t)slot * kp.n * kp.wsg_h;
    kp.wsg_start = W.ends + 2;
    kp.wsg_land = W.land;
    return launch_wsg_build(kp, day, W, ctx->stream);
}

extern "C" int deabm_step(deabm_ctx *ctx, uint32_t n_steps)
{
    if (!ctx) return fail(nullptr, DEABM_EINVAL, "ctx is NULL");
    if ((uint64_t)ctx->day + n_steps > ctx->max_steps)
        return fail(ctx, DEABM_ESTATE, "day %u + %u steps exceeds max_steps %u", ctx->day, n_steps, ctx->max_steps);
    if (ctx->ragged) {
        for (uint32_t q = 0; q < n_steps; ++q) {
            CU(ctx, ragged_day(ctx, ctx->day, ctx->cur));
            ctx->cur ^= 1;
            ctx->day += 1;
        }
        return DEABM_OK;
    }
    for (uint32_t s = 0; s < n_steps; ++s) {
        const int c = ctx->cur;
        KParams kp = ctx->kp;
        if (kp.vax_strategy != 0 && kp.vax_on && ctx->day >= ctx->base.vax_start) {
            if (ctx->n_rep > 1)
                CU(ctx, launch_vax_select_batch(kp, ctx->day, ctx->base.elderly_bin, ctx->vax_supply, ctx->S,
                                                ctx->vax_cls, ctx->vax_dose, ctx->vax_scratch, ctx->stream));
            else
                CU(ctx, launch_vax_select(kp, ctx->day, ctx->base.dose2_delay, ctx->base.elderly_bin, ctx->vax_supply,
                                          ctx->S, ctx->vax_cls, ctx->vax_dose, ctx->vax_scratch, ctx->stream));
            kp.dose_today = ctx->vax_dose;
        }
        InfBuffers I;
        I.cur = ctx->inf[c];
        I.next = ctx->inf[c ^ 1];
        I.rand_cur = ctx->inf_rand[c] ? ctx->inf_rand[c] : ctx->inf[c];
        I.rand_next = ctx->inf_rand[c ^ 1];
        I.row_of = ctx->row_of;
        if (kp.den_bits_orig)
            CU(ctx, cudaMemsetAsync(kp.den_bits_orig, 0, sizeof(uint32_t) * (((size_t)ctx->n + 31) / 32), ctx->stream));
        if (kp.wsg_on) CU(ctx, wsg_day(ctx, kp, ctx->day));
        CU(ctx, launch_step(kp, ctx->day, I, ctx->S, ctx->C, ctx->keep_lambda ? ctx->lam : nullptr, ctx->p,
                            ctx->stream));
        if (kp.den_on) {
            if (ctx->n_rep == 1) CU(ctx, launch_den(kp, ctx->day, ctx->S, ctx->C, ctx->stream));
            else CU(ctx, launch_den_batch(kp, ctx->day, ctx->row_of, ctx->S, ctx->C, ctx->n_rep, 0u, ctx->stream));
        }
        ctx->cur ^= 1;
        ctx->day += 1;
    }
    return DEABM_OK;
}

extern "C" int deabm_get_counters(deabm_ctx *ctx, uint32_t day_count, int32_t *new_inf, int32_t *hist,
                                  uint64_t *messages)
{
    if (!ctx) return fail(nullptr, DEABM_EINVAL, "ctx is NULL");
    if (day_count > ctx->day) return fail(ctx, DEABM_EINVAL, "only %u days have run", ctx->day);
    const size_t B = ctx->n_rep;
    if (new_inf && day_count)
        CU(ctx, cudaMemcpyAsync(new_inf, ctx->C.new_inf, sizeof(int32_t) * day_count * B, cudaMemcpyDeviceToHost,
                                ctx->stream));
    if (hist && day_count)
        CU(ctx, cudaMemcpyAsync(hist, ctx->C.hist, sizeof(int32_t) * day_count * B * DEABM_N_STAGE,
                                cudaMemcpyDeviceToHost, ctx->stream));
    if (messages && day_count)
        CU(ctx, cudaMemcpyAsync(messages, ctx->C.msgs, sizeof(uint64_t) * day_count, cudaMemcpyDeviceToHost,
                                ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    if (messages)
        for (uint32_t d = 0; d < day_count; ++d) messages[d] += ctx->static_edges;
    return DEABM_OK;
}

extern "C" int deabm_get_gathered(deabm_ctx *ctx, uint32_t day_count, uint64_t *gathered)
{
    if (!ctx || !gathered) return fail(ctx, DEABM_EINVAL, "ctx and gathered are required");
    if (day_count > ctx->day) return fail(ctx, DEABM_EINVAL, "only %u days have run", ctx->day);
    if (day_count == 0) return DEABM_OK;
    if (!ctx->ragged && ctx->n_rep > 1) {
        // the batched kernels gather every agent's in-contacts for every replicate
        return deabm_get_counters(ctx, day_count, nullptr, nullptr, gathered);
    }
    CU(ctx, cudaMemcpyAsync(gathered, ctx->C.gath, sizeof(uint64_t) * day_count, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return DEABM_OK;
}

// T ragged days as one CUDA graph (captured once per starting day and length, then replayed)
static int run_ragged_graph(deabm_ctx *ctx, uint32_t T)
{
    if ((uint64_t)ctx->day + T > ctx->max_steps)
        return fail(ctx, DEABM_ESTATE, "day %u + %u steps exceeds max_steps %u", ctx->day, T, ctx->max_steps);
    const uint32_t d0 = ctx->day;
    const int cur0 = ctx->cur;
    if (!(ctx->graph && ctx->graph_day0 == d0 && ctx->graph_T == T && cur0 == (int)(d0 & 1u))) {
        if (ctx->graph) {
            CU(ctx, cudaGraphExecDestroy(ctx->graph));
            ctx->graph = nullptr;
        }
        cudaGraph_t g;
        CU(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        int c = cur0;
        for (uint32_t q = 0; q < T; ++q) {
            cudaError_t e = ragged_day(ctx, d0 + q, c);
            if (e != cudaSuccess) {
                cudaStreamEndCapture(ctx->stream, &g);
                return fail(ctx, DEABM_ECUDA, "capture: %s", cudaGetErrorString(e));
            }
            c ^= 1;
        }
        CU(ctx, cudaStreamEndCapture(ctx->stream, &g));
        cudaError_t e = cudaGraphInstantiate(&ctx->graph, g, 0);
        (void)cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(ctx, DEABM_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        ctx->graph_day0 = d0;
        ctx->graph_T = T;
    }
    CU(ctx, cudaGraphLaunch(ctx->graph, ctx->stream));
    ctx->day += T;
    if (T & 1u) ctx->cur ^= 1;
    return DEABM_OK;
}

extern "C" int deabm_run(deabm_ctx *ctx, uint32_t T, int32_t *new_inf, int32_t *hist)
{
    if (!ctx) return fail(nullptr, DEABM_EINVAL, "ctx is NULL");
    const uint32_t d0 = ctx->day;
    int rc = ctx->ragged && T > 0 ? run_ragged_graph(ctx, T) : deabm_step(ctx, T);
    if (rc) return rc;
    const size_t B = ctx->n_rep;
    if (new_inf && T)
        CU(ctx, cudaMemcpyAsync(new_inf, ctx->C.new_inf + (size_t)d0 * B, sizeof(int32_t) * T * B,
                                cudaMemcpyDeviceToHost, ctx->stream));
    if (hist && T)
        CU(ctx, cudaMemcpyAsync(hist, ctx->C.hist + (size_t)d0 * B * DEABM_N_STAGE,
                                sizeof(int32_t) * T * B * DEABM_N_STAGE, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return DEABM_OK;
}

// device scratch of n * n_rep * 4 bytes for caller-order readbacks (relabelled contexts)
// Touches every page of the caller's output buffers on host threads before the
// device copies into them.  A copy into pages the process has never touched
// faults them in one by one during the transfer, which was measured several
// times slower than the copy itself (14 MB of state: 2.5-15 ms against 0.6 ms).
struct HostBuf {
    void *ptr;
    size_t bytes;
};

static void prefault(const HostBuf *bufs, size_t count)
{
    constexpr size_t kPage = 4096;
    size_t pages = 0;
    for (size_t q = 0; q < count; ++q) pages += bufs[q].ptr ? (bufs[q].bytes + kPage - 1) / kPage : 0;
    if (pages == 0) return;
    const uint32_t T = pages < 256 ? 1u : std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    parallel_chunks((uint32_t)pages, T, [&](uint32_t b, uint32_t e, uint32_t) {
        size_t first = 0;  // global index of the current buffer's first page
        for (size_t q = 0; q < count && b < e; ++q) {
            if (!bufs[q].ptr) continue;
            const size_t np = (bufs[q].bytes + kPage - 1) / kPage;
            for (; b < e && b < first + np; ++b)
                static_cast<volatile char *>(bufs[q].ptr)[(b - first) * kPage] = 0;
            first += np;
        }
    });
}

static int perm_scratch_ready(deabm_ctx *ctx)
{
    if (!ctx->relabel || ctx->perm_scratch) return DEABM_OK;
    uint32_t *p;
    int r = dalloc(ctx, &p, (size_t)ctx->n * (ctx->ragged ? 1u : ctx->n_rep));
    if (r) return r;
    ctx->perm_scratch = p;
    return DEABM_OK;
}

extern "C" int deabm_get_state(deabm_ctx *ctx, int8_t *stage, int16_t *timer, int16_t *tinf, uint8_t *flags,
                               uint8_t *qt, float *lambda, float *p)
{
    if (!ctx) return fail(nullptr, DEABM_EINVAL, "ctx is NULL");
    if ((lambda || p) && !ctx->keep_lambda) return fail(ctx, DEABM_ESTATE, "created without keep_lambda");
    const size_t nb = ctx->ragged ? (size_t)ctx->n : (size_t)ctx->n * ctx->n_rep;
    cudaStream_t s = ctx->stream;
    // device arrays are in internal order: when relabelled, a kernel puts each
    // agent back at its caller id in device scratch, which is then copied out
    int r;
    if ((r = perm_scratch_ready(ctx))) return r;
    const HostBuf outs[] = {{stage, nb}, {timer, 2 * nb}, {tinf, 2 * nb}, {flags, nb},
                            {qt, nb},    {lambda, 4 * nb}, {p, 4 * nb}};
    prefault(outs, sizeof outs / sizeof outs[0]);
    auto fetch = [&](void *dst, const void *src, size_t elem) -> int {
        if (!dst) return DEABM_OK;
        if (ctx->relabel) {
            CU(ctx, launch_to_caller(ctx->perm_scratch, src, ctx->orig_id, ctx->n, ctx->ragged ? 1u : ctx->n_rep,
                                     (uint32_t)elem, s));
            src = ctx->perm_scratch;
        }
        CU(ctx, cudaMemcpyAsync(dst, src, nb * elem, cudaMemcpyDeviceToHost, s));
        return DEABM_OK;
    };
    if ((r = fetch(stage, ctx->S.stage, 1))) return r;
    if ((r = fetch(timer, ctx->S.timer, 2))) return r;
    if ((r = fetch(tinf, ctx->S.tinf, 2))) return r;
    if ((r = fetch(flags, ctx->S.flags, 1))) return r;
    if ((r = fetch(qt, ctx->S.qt, 1))) return r;
    if ((r = fetch(lambda, ctx->lam, 4))) return r;
    if ((r = fetch(p, ctx->p, 4))) return r;
    CU(ctx, cudaStreamSynchronize(s));
    return DEABM_OK;
}

extern "C" int deabm_get_dose_days(deabm_ctx *ctx, int16_t *dose1_day, int16_t *dose2_day)
{
    if (!ctx) return fail(nullptr, DEABM_EINVAL, "ctx is NULL");
    if (!ctx->S.vd1) return fail(ctx, DEABM_ESTATE, "no vaccination priority strategy in this context");
    if (ctx->ragged) {  // populations in order, each agent at its caller position (as deabm_get_state)
        int r;
        if ((r = perm_scratch_ready(ctx))) return r;
        const HostBuf outs[] = {{dose1_day, 2ull * ctx->n}, {dose2_day, 2ull * ctx->n}};
        prefault(outs, 2);
        const int16_t *src[2] = {ctx->S.vd1, ctx->S.vd2};
        int16_t *dst[2] = {dose1_day, dose2_day};
        for (int q = 0; q < 2; ++q) {
            if (!dst[q]) continue;
            const void *from = src[q];
            if (ctx->relabel) {
                CU(ctx, launch_to_caller(ctx->perm_scratch, from, ctx->orig_id, ctx->n, 1u, 2u, ctx->stream));
                from = ctx->perm_scratch;
            }
            CU(ctx, cudaMemcpyAsync(dst[q], from, 2ull * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
        }
        CU(ctx, cudaStreamSynchronize(ctx->stream));
        return DEABM_OK;
    }
    const uint32_t B = ctx->n_rep;
    const size_t nb = (size_t)ctx->n * B;
    std::vector<int16_t> t1(nb), t2(nb);
    CU(ctx, cudaMemcpyAsync(t1.data(), ctx->S.vd1, nb * 2, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaMemcpyAsync(t2.data(), ctx->S.vd2, nb * 2, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    int r = host_order(ctx);
    if (r) return r;
    for (uint32_t q = 0; q < ctx->n; ++q) {
        const size_t o = (size_t)(ctx->relabel ? ctx->new2orig[q] : q) * B;
        for (uint32_t b = 0; b < B; ++b) {
            if (dose1_day) dose1_day[o + b] = t1[(size_t)q * B + b];
            if (dose2_day) dose2_day[o + b] = t2[(size_t)q * B + b];
        }
    }
    return DEABM_OK;
}

extern "C" int deabm_get_tables(deabm_ctx *ctx, float *inf_table, uint64_t *poisson_thr, int16_t *dose1_day)
{
    if (!ctx) return fail(nullptr, DEABM_EINVAL, "ctx is NULL");
    Tables T;
    CU(ctx, cudaMemcpyAsync(&T, ctx->tab, sizeof T, cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<int16_t> d1(dose1_day ? ctx->n : 0);
    if (dose1_day) CU(ctx, cudaMemcpyAsync(d1.data(), ctx->dose1, 2ull * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    if (dose1_day) {
        int r = host_order(ctx);
        if (r) return r;
        for (uint32_t q = 0; q < ctx->n; ++q) dose1_day[ctx->relabel ? ctx->new2orig[q] : q] = d1[q];
    }
    if (inf_table)
        for (int c = 0; c < DEABM_N_CLASS; ++c)
            std::memcpy(inf_table + (size_t)c * ctx->kp.inf_len, T.infT[c], sizeof(float) * ctx->kp.inf_len);
    if (poisson_thr) std::memcpy(poisson_thr, T.pois, sizeof T.pois);
    return DEABM_OK;
}

// ---------------------------------------------------------------- ragged batches
// tiles of rows_per_tile rows that never cross a population boundary
static std::vector<Tile> make_tiles(const std::vector<PopDesc> &pops, uint32_t rows_per_tile)
{
    std::vector<Tile> t;
    for (uint32_t p = 0; p < pops.size(); ++p)
        for (uint32_t b = 0; b < pops[p].kp.n; b += rows_per_tile)
            t.push_back(Tile{p, b, std::min(pops[p].kp.n, b + rows_per_tile), 0u});
    return t;
}

static int set_tiling(deabm_ctx *ctx, uint32_t rows_per_tile, uint32_t blocks_per_sm)
{
    std::vector<Tile> t = make_tiles(ctx->pops, rows_per_tile);
    if (t.size() > ctx->max_tiles) return fail(ctx, DEABM_EINVAL, "rows_per_tile %u is too small", rows_per_tile);
    CU(ctx, cudaMemcpyAsync(ctx->d_tiles, t.data(), sizeof(Tile) * t.size(), cudaMemcpyHostToDevice, ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->n_tiles = (uint32_t)t.size();
    ctx->rows_per_tile = rows_per_tile;
    ctx->grid = std::max(1u, std::min(ctx->n_tiles, ctx->sm_count * blocks_per_sm));
    if (ctx->graph) {
        CU(ctx, cudaGraphExecDestroy(ctx->graph));
        ctx->graph = nullptr;
    }
    return DEABM_OK;
}

extern "C" int deabm_create_ragged(uint32_t n_pops, const deabm_graph *graphs, const deabm_agents *agents,
                                   const deabm_params *params, void *cuda_stream, deabm_ctx **out)
{
    if (!out) return fail(nullptr, DEABM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_pops < 1 || n_pops > 4096 || !graphs || !agents || !params)
        return fail(nullptr, DEABM_EINVAL, "1 <= n_pops <= 4096 populations with graphs, agents, params required");
    deabm_ctx *ctx = new (std::nothrow) deabm_ctx();
    if (!ctx) return fail(nullptr, DEABM_ENOMEM, "host allocation failed");
    int rc = [&]() -> int {
        uint64_t total = 0;
        uint32_t max_steps = 0;
        for (uint32_t q = 0; q < n_pops; ++q) {
            int r = validate(ctx, &graphs[q], &agents[q], &params[q], 1u, nullptr);
            if (r) return fail(ctx, r, "population %u: %s", q, ctx->err.c_str());
            total += graphs[q].n_agents;
            max_steps = std::max(max_steps, params[q].max_steps ? params[q].max_steps : 1024u);
            if (params[q].keep_lambda) return fail(ctx, DEABM_EINVAL, "keep_lambda is not available for ragged batches");
        }
        if (total >= (1ull << 31)) return fail(ctx, DEABM_EINVAL, "too many agents in total");
        ctx->ragged = true;
        ctx->n = (uint32_t)total;
        arena_plan(ctx, total, 1);
        ctx->n_rep = n_pops;  // counters are [day][population]
        ctx->max_steps = max_steps;
        ctx->base = params[0];
        if (cuda_stream) {
            ctx->stream = (cudaStream_t)cuda_stream;
        } else {  // graph capture needs a stream other than the legacy default stream
            CU(ctx, cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking));
            ctx->stream = ctx->own_stream;
        }
        cudaStream_t s = ctx->stream;
        int dev = 0, sms = 0;
        CU(ctx, cudaGetDevice(&dev));
        CU(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        ctx->sm_count = (uint32_t)sms;
        int r;
        const size_t N = total;
        if ((r = dalloc(ctx, &ctx->age, N))) return r;
        if ((r = dalloc(ctx, &ctx->dose1, N))) return r;
        StateRef *sets[2] = {&ctx->S, &ctx->S0};
        for (StateRef *st : sets) {
            if ((r = dalloc(ctx, &st->stage, N))) return r;
            if ((r = dalloc(ctx, &st->timer, N))) return r;
            if ((r = dalloc(ctx, &st->tinf, N))) return r;
            if ((r = dalloc(ctx, &st->flags, N))) return r;
            if ((r = dalloc(ctx, &st->qt, N))) return r;
        }
        if ((r = dalloc(ctx, &ctx->inf[0], N))) return r;
        if ((r = dalloc(ctx, &ctx->inf[1], N))) return r;
        if ((r = dalloc(ctx, &ctx->tab, n_pops))) return r;
        if ((r = dalloc(ctx, &ctx->rep, n_pops))) return r;
        const size_t days = ctx->max_steps;
        if ((r = dalloc(ctx, &ctx->C.new_inf, days * n_pops))) return r;
        if ((r = dalloc(ctx, &ctx->C.hist, days * n_pops * DEABM_N_STAGE))) return r;
        if ((r = dalloc(ctx, &ctx->C.msgs, days))) return r;
        if ((r = dalloc(ctx, &ctx->C.gath, days))) return r;
        if ((r = dalloc(ctx, &ctx->queue, days))) return r;
        if ((r = dalloc(ctx, &ctx->C.den, days * n_pops))) return r;  // notified, [day][population]
        bool any_den = false;
        for (uint32_t q = 0; q < n_pops; ++q) any_den |= params[q].den_on != 0;
        if (any_den) {  // positives of the day (one word per row) and their count, [population][day]
            if ((r = dalloc(ctx, &ctx->den_bits, N))) return r;
            if ((r = dalloc(ctx, &ctx->den_pos, days * n_pops))) return r;
        }
        uint32_t max_n = 0;
        for (uint32_t q = 0; q < n_pops; ++q) max_n = std::max(max_n, graphs[q].n_agents);
        bool any_strategy = false;
        for (uint32_t q = 0; q < n_pops; ++q) any_strategy |= params[q].vax_strategy && params[q].vax_on;
        if (any_strategy) {  // dose days (none yet), the day's classes and doses by caller id, selection scratch
            StateRef *vsets[2] = {&ctx->S, &ctx->S0};
            for (StateRef *st : vsets) {
                if ((r = dalloc(ctx, &st->vd1, N))) return r;
                if ((r = dalloc(ctx, &st->vd2, N))) return r;
            }
            if ((r = dalloc(ctx, &ctx->vax_cls, N))) return r;
            if ((r = dalloc(ctx, &ctx->vax_dose, N))) return r;
            if ((r = dalloc(ctx, &ctx->vax_scratch, vax_select_scratch_words(max_n)))) return r;
            const std::vector<int16_t> never(N, kNever);
            CU(ctx, cudaMemcpyAsync(ctx->S0.vd1, never.data(), N * 2, cudaMemcpyHostToDevice, s));
            CU(ctx, cudaMemcpyAsync(ctx->S0.vd2, never.data(), N * 2, cudaMemcpyHostToDevice, s));
            CU(ctx, cudaStreamSynchronize(s));
        }
        uint32_t *d_scratch;
        double *d_gamma;
        float *d_A;
        if ((r = dalloc(ctx, &d_scratch, dose1_scratch_words(max_n)))) return r;
        if ((r = dalloc(ctx, &d_gamma, 6 * (size_t)n_pops))) return r;
        if ((r = dalloc(ctx, &d_A, 3 * (size_t)n_pops))) return r;
        ctx->pops.resize(n_pops);
        ctx->pop_seeds.resize(n_pops);
        ctx->d_pop_seeds.assign(n_pops, nullptr);
        uint32_t base = 0;
        if ((r = dalloc(ctx, &ctx->orig_local, N))) return r;
        if ((r = dalloc(ctx, &ctx->row_local, N))) return r;
        for (uint32_t q = 0; q < n_pops; ++q) {
            const deabm_graph &g = graphs[q];
            const deabm_agents &a = agents[q];
            const deabm_params &p = params[q];
            const uint32_t n = g.n_agents;
            PopDesc &pd = ctx->pops[q];
            std::memset(&pd, 0, sizeof pd);
            pd.base = base;
            KParams &K = pd.kp;
            K.n = n;
            K.n_nets = g.n_nets;
            K.n_rep = 1;
            K.inf_len = p.inf_len;
            K.dt = p.dt;
            K.rand_on = poisson_on(&g) ? 1u : 0u;
            K.rand_by_age = g.rand_by_age ? 1u : 0u;
            // the population's stored networks; renumbered on the device like a
            // plain context's when locality_order asks for it, or in occupation
            // order (members of an occupation adjacent) when it draws daily
            // occupation contacts
            const bool occ_q = g.n_occ > 0;
            const bool relabel_q = (p.locality_order != 0 && g.n_nets > 0) || occ_q;
            std::vector<uint32_t> occ_order, occ_start;  // host staging, kept to the population's sync
            DevScratch sc;
            uint32_t *src_rp[DEABM_MAX_NETS] = {}, *src_col[DEABM_MAX_NETS] = {};
            uint32_t best = 0;
            for (uint32_t k = 0; k < g.n_nets; ++k) {
                const uint32_t E = g.row_ptr[k][n];
                if (E > g.row_ptr[best][n]) best = k;
                uint32_t *rp, *cl;
                if ((r = dalloc(ctx, &rp, (size_t)n + 1))) return r;
                if ((r = dalloc(ctx, &cl, E))) return r;
                src_rp[k] = rp;
                src_col[k] = cl;
                if (relabel_q) {
                    if ((r = scratch_alloc(ctx, sc, &src_rp[k], (size_t)n + 1))) return r;
                    if ((r = scratch_alloc(ctx, sc, &src_col[k], E))) return r;
                }
                CU(ctx, cudaMemcpyAsync(src_rp[k], g.row_ptr[k], 4ull * (n + 1), cudaMemcpyHostToDevice, s));
                if (E) CU(ctx, cudaMemcpyAsync(src_col[k], g.col[k], 4ull * E, cudaMemcpyHostToDevice, s));
                K.row_ptr[k] = rp;
                K.col[k] = cl;
                ctx->static_edges += E;
            }
            if (relabel_q) {  // this population's numbering (local ids)
                uint32_t *d_scan;
                if ((r = scratch_alloc(ctx, sc, &d_scan, scan_scratch_words((size_t)n + 1)))) return r;
                if (occ_q) {
                    occupation_order(&g, occ_order, occ_start);
                    CU(ctx, cudaMemcpyAsync(ctx->orig_local + base, occ_order.data(), 4ull * n, cudaMemcpyHostToDevice, s));
                } else {  // by label propagation on the device
                    uint32_t *label, *tmp, *changed;
                    if ((r = scratch_alloc(ctx, sc, &label, n))) return r;
                    if ((r = scratch_alloc(ctx, sc, &tmp, std::max<size_t>(n, order_scratch_words(n))))) return r;
                    if ((r = scratch_alloc(ctx, sc, &changed, 1))) return r;
                    CU(ctx, launch_locality_labels(src_rp[best], src_col[best], n, kLocalityRounds, label, tmp, changed,
                                                   s));
                    CU(ctx, launch_order_by_label(label, n, ctx->orig_local + base, tmp, s));
                }
                CU(ctx, launch_invert(ctx->orig_local + base, n, ctx->row_local + base, s));
                for (uint32_t k = 0; k < g.n_nets; ++k)
                    CU(ctx, launch_csr_renumber(src_rp[k], src_col[k], ctx->orig_local + base, ctx->row_local + base, n,
                                                (uint32_t *)K.row_ptr[k], (uint32_t *)K.col[k], d_scan, s));
                pd.row_of = ctx->row_local + base;
            }
            std::vector<uint32_t> occ_gid;
            if (occ_q) {  // occupation of each row, each occupation's first row and daily count
                occ_gid.resize(n);
                for (uint32_t q2 = 0; q2 < n; ++q2) occ_gid[q2] = g.occ_group[occ_order[q2]];
                uint32_t *d_gid, *d_start;
                uint8_t *d_k;
                if ((r = dalloc(ctx, &d_gid, n))) return r;
                if ((r = dalloc(ctx, &d_start, (size_t)g.n_occ + 1))) return r;
                if ((r = dalloc(ctx, &d_k, g.n_occ))) return r;
                CU(ctx, cudaMemcpyAsync(d_gid, occ_gid.data(), 4ull * n, cudaMemcpyHostToDevice, s));
                CU(ctx, cudaMemcpyAsync(d_start, occ_start.data(), 4ull * ((size_t)g.n_occ + 1), cudaMemcpyHostToDevice, s));
                CU(ctx, cudaMemcpyAsync(d_k, g.occ_k, g.n_occ, cudaMemcpyHostToDevice, s));
                K.n_occ = g.n_occ;
                K.occ_gid = d_gid;
                K.occ_start = d_start;
                K.occ_k = d_k;
                K.occ_lattice = g.occ_lattice;
                K.thr_rewire = threshold((double)g.occ_rewire);
                ctx->ragged_occ = true;
            }
            K.net_seed = p.net_seed;
            round_keys(p.net_seed, K.nrk);
            if (g.rand_ws) {  // its Watts-Strogatz random network, rebuilt before each day (by caller id)
                WsgBuffers W{};
                K.wsg_on = 1;
                K.wsg_h = g.rand_ws_k / 2u;
                K.thr_wsg = threshold((double)g.rand_ws_beta);
                const size_t edges = (size_t)n * K.wsg_h;
                // with exposure notification the look-back window's graphs are kept
                const uint32_t ring = p.den_on ? p.den_window : 1u;
                if ((r = dalloc(ctx, &W.rew, n))) return r;
                if ((r = dalloc(ctx, &W.far, edges))) return r;
                if ((r = dalloc(ctx, &W.ends, ((size_t)n + 3) * ring))) return r;
                if ((r = dalloc(ctx, &W.land, edges * ring))) return r;
                if ((r = dalloc(ctx, &W.scratch, wsg_scratch_words(n)))) return r;
                K.wsg_rew = W.rew;
                K.wsg_start = W.ends + 2;
                K.wsg_land = W.land;
                K.wsg_ends_ring = W.ends;
                K.wsg_land_ring = W.land;
                K.wsg_ring_days = ring;
                ctx->ragged_wsg_bufs.push_back({q, W});
                ctx->ragged_wsg = true;
            }
            K.test_on = p.test_on;
            K.test_lo = p.test_lo;
            K.test_hi = p.test_hi;
            K.quar_on = p.quar_on;
            K.quar_days = p.quar_days;
            K.thr_sens = threshold(p.test_sens);
            K.thr_qdrop = threshold(p.q_dropout);
            K.vax_on = p.vax_on;
            K.vax_onset = p.vax_onset;
            K.thr_eff1 = threshold(p.vax_eff1);
            K.thr_eff2 = threshold(p.vax_eff2);
            K.vax_nonsterile = p.vax_nonsterile ? 1u : 0u;
            K.vax_strategy = p.vax_strategy;
            if (p.den_on) {  // exposure notification: the positives of its rows and days
                K.den_on = 1u;
                K.den_window = p.den_window;
                K.thr_comp = threshold(p.den_compliance);
                K.thr_adopt = threshold(p.den_adoption);
                K.den_bits = ctx->den_bits + base;
                K.den_pos = ctx->den_pos + (size_t)q * days;
                ctx->ragged_den.push_back(q);
            }
            if (p.vax_strategy && p.vax_on) {  // its doses are selected before each day from vax_start
                K.dose_today = ctx->vax_dose + base;
                ctx->ragged_vax.push_back({q, (uint32_t)std::floor(p.vax_rate * (double)n), p.vax_start,
                                           p.dose2_delay, p.elderly_bin});
            }
            K.tab = ctx->tab + q;
            K.rep = ctx->rep + q;
            K.age = ctx->age + base;
            K.dose1_day = ctx->dose1 + base;
            K.orig_id = relabel_q ? ctx->orig_local + base : nullptr;
            std::vector<Rep> reps;
            build_reps(&p, 1, nullptr, nullptr, reps);
            pd.rep = reps[0];
            CU(ctx, cudaMemcpyAsync(ctx->rep + q, &pd.rep, sizeof(Rep), cudaMemcpyHostToDevice, s));
            // tables of this population
            Tables T;
            std::memset(&T, 0, sizeof T);
            poisson_tables(&g, T);
            for (int a2 = 0; a2 < DEABM_N_AGE; ++a2) {
                T.thr_asym[a2] = threshold(p.p_asym[a2]);
                T.thr_sev[a2] = threshold(p.p_sev[a2]);
                T.thr_branch[DEABM_SEV][a2] = threshold(p.p_hosp[a2]);
                T.thr_branch[DEABM_HOSP][a2] = threshold(p.p_icu[a2]);
                T.thr_branch[DEABM_ICU][a2] = threshold(p.p_death[a2]);
            }
            std::memcpy(T.dur_lo, p.dur_lo, sizeof T.dur_lo);
            std::memcpy(T.dur_hi, p.dur_hi, sizeof T.dur_hi);
            CU(ctx, cudaMemcpyAsync(ctx->tab + q, &T, sizeof T, cudaMemcpyHostToDevice, s));
            set_pois32(K, T.pois);
            K.rep0 = pd.rep;
            const double gs[6] = {p.inf_shape[0], p.inf_shape[1], p.inf_shape[2], p.inf_scale[0], p.inf_scale[1],
                                  p.inf_scale[2]};
            CU(ctx, cudaMemcpyAsync(d_gamma + 6 * q, gs, sizeof gs, cudaMemcpyHostToDevice, s));
            CU(ctx, cudaMemcpyAsync(d_A + 3 * q, p.A_class, sizeof(float) * 3, cudaMemcpyHostToDevice, s));
            CU(ctx, launch_inf_table(ctx->tab + q, d_gamma + 6 * q, d_A + 3 * q, p.inf_len, s));
            // per-agent arrays go up in caller order and are put in place on the device
            uint16_t *d_in;
            if ((r = scratch_alloc(ctx, sc, &d_in, n))) return r;
            const uint32_t *perm = relabel_q ? ctx->orig_local + base : nullptr;
            auto put = [&](void *dst, const void *src, uint32_t elem) -> int {
                if (!src) {
                    CU(ctx, cudaMemsetAsync(dst, 0, (size_t)n * elem, s));
                } else if (!perm) {
                    CU(ctx, cudaMemcpyAsync(dst, src, (size_t)n * elem, cudaMemcpyHostToDevice, s));
                } else {
                    CU(ctx, cudaMemcpyAsync(d_in, src, (size_t)n * elem, cudaMemcpyHostToDevice, s));
                    CU(ctx, launch_from_caller(dst, d_in, perm, n, 1u, elem, false, s));
                }
                return DEABM_OK;
            };
            const uint32_t per_day = p.vax_on ? (uint32_t)std::floor(p.vax_rate * (double)n) : 0u;
            if (perm) {  // first-dose days from the caller-order ages (ties by caller id), then put in place
                uint8_t *d_age;
                int16_t *d_dose;
                if ((r = scratch_alloc(ctx, sc, &d_age, n))) return r;
                if ((r = scratch_alloc(ctx, sc, &d_dose, n))) return r;
                CU(ctx, cudaMemcpyAsync(d_age, a.age_bin, n, cudaMemcpyHostToDevice, s));
                CU(ctx, launch_dose1_days(d_age, n, p.vax_start, per_day, d_dose, d_scratch, s));
                CU(ctx, launch_gather_i16(ctx->dose1 + base, d_dose, perm, n, s));
                if ((r = put(ctx->age + base, a.age_bin, 1))) return r;
            } else {
                CU(ctx, cudaMemcpyAsync(ctx->age + base, a.age_bin, n, cudaMemcpyHostToDevice, s));
                CU(ctx, launch_dose1_days(ctx->age + base, n, p.vax_start, per_day, ctx->dose1 + base, d_scratch, s));
            }
            if ((r = put(ctx->S0.stage + base, a.stage, 1))) return r;
            if ((r = put(ctx->S0.timer + base, a.timer, 2))) return r;
            if ((r = put(ctx->S0.tinf + base, a.tinf, 2))) return r;
            if ((r = put(ctx->S0.flags + base, a.flags, 1))) return r;
            if ((r = put(ctx->S0.qt + base, a.qt, 1))) return r;
            if (p.vax_strategy && ctx->S0.vd1) {  // the caller's dose days so far (none where not given)
                if (a.dose1_day && (r = put(ctx->S0.vd1 + base, a.dose1_day, 2))) return r;
                if (a.dose2_day && (r = put(ctx->S0.vd2 + base, a.dose2_day, 2))) return r;
            }
            if (K.den_on) {  // app holders, part of the initial state
                StateRef S0p{ctx->S0.stage + base, ctx->S0.timer + base, ctx->S0.tinf + base, ctx->S0.flags + base,
                             ctx->S0.qt + base};
                CU(ctx, launch_den_apps(K, S0p, s));
            }
            CU(ctx, cudaStreamSynchronize(s));  // scratch of this population ends here
            ctx->pop_seeds[q].assign(a.seed_ids, a.seed_ids + a.n_seed);  // caller ids
            if (a.n_seed) {  // on the device: local rows
                if ((r = dalloc(ctx, &ctx->d_pop_seeds[q], a.n_seed))) return r;
                CU(ctx, cudaMemcpyAsync(ctx->d_pop_seeds[q], ctx->pop_seeds[q].data(), 4ull * a.n_seed,
                                        cudaMemcpyHostToDevice, s));
                if (relabel_q) CU(ctx, launch_map_ids(ctx->d_pop_seeds[q], a.n_seed, ctx->row_local + base, s));
                CU(ctx, cudaStreamSynchronize(s));
            }
            base += n;
        }
        bool any_relabel = false;
        for (uint32_t q = 0; q < n_pops; ++q) any_relabel |= ctx->pops[q].row_of != nullptr;
        if (any_relabel) {  // readbacks put every agent back at its caller position
            ctx->relabel = true;
            if ((r = dalloc(ctx, &ctx->orig_id, N))) return r;
            for (uint32_t q = 0; q < n_pops; ++q) {
                const PopDesc &pd = ctx->pops[q];
                CU(ctx, launch_offset_ids(ctx->orig_id + pd.base, pd.row_of ? ctx->orig_local + pd.base : nullptr,
                                          pd.kp.n, pd.base, s));
            }
        }
        if ((r = dalloc(ctx, &ctx->d_pops, n_pops))) return r;
        CU(ctx, cudaMemcpyAsync(ctx->d_pops, ctx->pops.data(), sizeof(PopDesc) * n_pops, cudaMemcpyHostToDevice, s));
        ctx->max_tiles = (uint32_t)make_tiles(ctx->pops, 256).size();
        if ((r = dalloc(ctx, &ctx->d_tiles, ctx->max_tiles))) return r;
        if ((r = set_tiling(ctx, 1024, 4))) return r;
        ctx->kp = ctx->pops[0].kp;
        if ((r = deabm_reset(ctx, nullptr, nullptr))) return r;
        CU(ctx, cudaStreamSynchronize(s));
        return DEABM_OK;
    }();
    if (rc != DEABM_OK) {
        std::string msg = ctx->err;
        deabm_destroy(ctx);
        g_err = msg;
        return rc;
    }
    *out = ctx;
    return DEABM_OK;
}

// Time `days_per_trial` days for every (rows per tile, blocks per SM) candidate on
// the live state, keep the fastest, then restart at day 0.
extern "C" int deabm_autotune(deabm_ctx *ctx, uint32_t days_per_trial, uint32_t *rows_per_tile, uint32_t *blocks_per_sm)
{
    if (!ctx) return fail(nullptr, DEABM_EINVAL, "ctx is NULL");
    if (!ctx->ragged) return fail(ctx, DEABM_ESTATE, "autotuning applies to ragged batches");
    if (days_per_trial == 0 || days_per_trial > ctx->max_steps) return fail(ctx, DEABM_EINVAL, "bad days_per_trial");
    const uint32_t rows[] = {256, 512, 1024, 2048, 4096};
    const uint32_t bps[] = {2, 4, 6, 8};
    float best = 1e30f;
    uint32_t best_r = 1024, best_b = 4;
    cudaEvent_t e0, e1;
    CU(ctx, cudaEventCreate(&e0));
    CU(ctx, cudaEventCreate(&e1));
    int r = DEABM_OK;
    for (uint32_t rt : rows) {
        for (uint32_t b : bps) {
            if ((r = set_tiling(ctx, rt, b))) break;
            if ((r = deabm_reset(ctx, nullptr, nullptr))) break;
            if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) { r = DEABM_ECUDA; break; }
            if ((r = deabm_step(ctx, days_per_trial))) break;
            if (cudaEventRecord(e1, ctx->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                r = DEABM_ECUDA;
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; best_r = rt; best_b = b; }
        }
        if (r) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r) return r;
    if ((r = set_tiling(ctx, best_r, best_b))) return r;
    if ((r = deabm_reset(ctx, nullptr, nullptr))) return r;
    if (rows_per_tile) *rows_per_tile = best_r;
    if (blocks_per_sm) *blocks_per_sm = best_b;
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return DEABM_OK;
}

extern "C" int deabm_reset(deabm_ctx *ctx, const float *rep_params, const uint64_t *rep_seeds)
{
    if (!ctx) return fail(nullptr, DEABM_EINVAL, "ctx is NULL");
    if ((rep_params == nullptr) != (rep_seeds == nullptr))
        return fail(ctx, DEABM_EINVAL, "rep_params and rep_seeds go together");
    cudaStream_t s = ctx->stream;
    const size_t nb = ctx->ragged ? (size_t)ctx->n : (size_t)ctx->n * ctx->n_rep;
    if (rep_params) {
        for (uint32_t b = 0; b < ctx->n_rep; ++b) {
            const float d = rep_params[b * DEABM_N_REP_PARAMS + 13];
            if (!(d >= 1.0f && d <= 30000.0f) || d != std::floor(d))
                return fail(ctx, DEABM_EINVAL, "replicate %u: dose2_delay must be a whole number of days >= 1", b);
        }
        std::vector<Rep> reps;
        build_reps(&ctx->base, ctx->n_rep, rep_params, rep_seeds, reps);
        CU(ctx, cudaMemcpyAsync(ctx->rep, reps.data(), sizeof(Rep) * ctx->n_rep, cudaMemcpyHostToDevice, s));
        if (!ctx->ragged) ctx->kp.rep0 = reps[0];
        CU(ctx, cudaStreamSynchronize(s));  // the staging vector goes out of scope
    }
    if (ctx->ragged && rep_params)
        return fail(ctx, DEABM_ESTATE, "a ragged batch keeps the parameters it was created with");
    CU(ctx, cudaMemcpyAsync(ctx->S.stage, ctx->S0.stage, nb, cudaMemcpyDeviceToDevice, s));
    CU(ctx, cudaMemcpyAsync(ctx->S.timer, ctx->S0.timer, nb * 2, cudaMemcpyDeviceToDevice, s));
    CU(ctx, cudaMemcpyAsync(ctx->S.tinf, ctx->S0.tinf, nb * 2, cudaMemcpyDeviceToDevice, s));
    CU(ctx, cudaMemcpyAsync(ctx->S.flags, ctx->S0.flags, nb, cudaMemcpyDeviceToDevice, s));
    CU(ctx, cudaMemcpyAsync(ctx->S.qt, ctx->S0.qt, nb, cudaMemcpyDeviceToDevice, s));
    if (ctx->ragged) {
        if (ctx->S.vd1) {  // priority strategies: no doses given yet, none selected
            CU(ctx, cudaMemcpyAsync(ctx->S.vd1, ctx->S0.vd1, nb * 2, cudaMemcpyDeviceToDevice, s));
            CU(ctx, cudaMemcpyAsync(ctx->S.vd2, ctx->S0.vd2, nb * 2, cudaMemcpyDeviceToDevice, s));
            CU(ctx, cudaMemsetAsync(ctx->vax_dose, 0, nb, s));
        }
        CU(ctx, clear_next_buffers(ctx, nb));
        for (size_t q = 0; q < ctx->pops.size(); ++q) {
            const PopDesc &pd = ctx->pops[q];
            StateRef Sp{ctx->S.stage + pd.base, ctx->S.timer + pd.base, ctx->S.tinf + pd.base, ctx->S.flags + pd.base,
                        ctx->S.qt + pd.base};
            if (!ctx->pop_seeds[q].empty())
                CU(ctx, launch_seed(pd.kp, ctx->d_pop_seeds[q], (uint32_t)ctx->pop_seeds[q].size(), Sp, s));
            CU(ctx, launch_emit(pd.kp, Sp, ctx->inf[0] + pd.base, nullptr, s));
        }
        ctx->cur = 0;
        CU(ctx, cudaMemsetAsync(ctx->queue, 0, sizeof(uint32_t) * ctx->max_steps, s));
        const size_t days = ctx->max_steps;
        CU(ctx, cudaMemsetAsync(ctx->C.new_inf, 0, sizeof(int32_t) * days * ctx->n_rep, s));
        CU(ctx, cudaMemsetAsync(ctx->C.hist, 0, sizeof(int32_t) * days * ctx->n_rep * DEABM_N_STAGE, s));
        CU(ctx, cudaMemsetAsync(ctx->C.msgs, 0, sizeof(unsigned long long) * days, s));
        CU(ctx, cudaMemsetAsync(ctx->C.gath, 0, sizeof(unsigned long long) * days, s));
        CU(ctx, cudaMemsetAsync(ctx->C.den, 0, sizeof(int32_t) * days * ctx->n_rep, s));
        if (ctx->den_pos) CU(ctx, cudaMemsetAsync(ctx->den_pos, 0, sizeof(int32_t) * days * ctx->n_rep, s));
        ctx->day = 0;
        return DEABM_OK;
    }
    if (ctx->S.vd1) {
        CU(ctx, cudaMemcpyAsync(ctx->S.vd1, ctx->S0.vd1, nb * 2, cudaMemcpyDeviceToDevice, s));
        CU(ctx, cudaMemcpyAsync(ctx->S.vd2, ctx->S0.vd2, nb * 2, cudaMemcpyDeviceToDevice, s));
    }
    if (ctx->kp.den_on) {  // the app draw follows the (possibly new) seed
        CU(ctx, launch_den_apps(ctx->kp, ctx->S, s));
        CU(ctx, cudaMemsetAsync(ctx->den_pos, 0, sizeof(int32_t) * ctx->max_steps, s));
        if (ctx->n_rep == 1) {
            int r = den_list_apps(ctx, ctx->kp);
            if (r) return r;
        }
    }
    if (ctx->n_seed) CU(ctx, launch_seed(ctx->kp, ctx->seed_ids, ctx->n_seed, ctx->S, s));
    ctx->cur = 0;
    CU(ctx, clear_next_buffers(ctx, nb));
    CU(ctx, launch_emit(ctx->kp, ctx->S, ctx->inf[0], ctx->inf_rand[0], s));
    const size_t days = ctx->max_steps;
    CU(ctx, cudaMemsetAsync(ctx->C.new_inf, 0, sizeof(int32_t) * days * ctx->n_rep, s));
    CU(ctx, cudaMemsetAsync(ctx->C.hist, 0, sizeof(int32_t) * days * ctx->n_rep * DEABM_N_STAGE, s));
    CU(ctx, cudaMemsetAsync(ctx->C.msgs, 0, sizeof(unsigned long long) * days, s));
    CU(ctx, cudaMemsetAsync(ctx->C.gath, 0, sizeof(unsigned long long) * days, s));
    CU(ctx, cudaMemsetAsync(ctx->C.den, 0, sizeof(int32_t) * days * ctx->n_rep, s));
    ctx->day = 0;
    return DEABM_OK;
}

extern "C" int deabm_get_notified(deabm_ctx *ctx, uint32_t day_count, int32_t *notified)
{
    if (!ctx) return fail(nullptr, DEABM_EINVAL, "ctx is NULL");
    if (day_count > ctx->day) return fail(ctx, DEABM_EINVAL, "only %u days have run", ctx->day);
    if (!notified || !day_count) return DEABM_OK;
    CU(ctx, cudaMemcpyAsync(notified, ctx->C.den, sizeof(int32_t) * day_count * ctx->n_rep, cudaMemcpyDeviceToHost,
                            ctx->stream));
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return DEABM_OK;
}

extern "C" int deabm_save(deabm_ctx *ctx, int8_t *stage, int16_t *timer, int16_t *tinf, uint8_t *flags, uint8_t *qt,
                          int16_t *dose1_day, int16_t *dose2_day, uint32_t *day)
{
    if (!ctx) return fail(nullptr, DEABM_EINVAL, "ctx is NULL");
    if (ctx->ragged) return fail(ctx, DEABM_ESTATE, "checkpoints are not available for ragged batches");
    int r = deabm_get_state(ctx, stage, timer, tinf, flags, qt, nullptr, nullptr);
    if (r) return r;
    if ((dose1_day || dose2_day) && ctx->S.vd1 && (r = deabm_get_dose_days(ctx, dose1_day, dose2_day))) return r;
    if (day) *day = ctx->day;
    return DEABM_OK;
}

extern "C" int deabm_restore(deabm_ctx *ctx, const int8_t *stage, const int16_t *timer, const int16_t *tinf,
                             const uint8_t *flags, const uint8_t *qt, const int16_t *dose1_day,
                             const int16_t *dose2_day, uint32_t day)
{
    if (!ctx) return fail(nullptr, DEABM_EINVAL, "ctx is NULL");
    if (ctx->ragged) return fail(ctx, DEABM_ESTATE, "checkpoints are not available for ragged batches");
    if (!stage || !timer || !tinf || !flags || !qt) return fail(ctx, DEABM_EINVAL, "stage, timer, tinf, flags and qt are required");
    if (day > ctx->max_steps) return fail(ctx, DEABM_EINVAL, "day %u > max_steps %u", day, ctx->max_steps);
    if (ctx->S.vd1 && (!dose1_day || !dose2_day))
        return fail(ctx, DEABM_EINVAL, "dose days are required under a vaccination priority strategy");
    const uint32_t n = ctx->n, B = ctx->n_rep;
    const size_t nb = (size_t)n * B;
    uint32_t jb = first_bad_row(n, [&](uint32_t q) {
        for (uint32_t b = 0; b < B; ++b) {
            const size_t i = (size_t)q * B + b;
            if (stage[i] < 0 || stage[i] >= DEABM_N_STAGE || (qt[i] & 0x80u)) return true;
        }
        return false;
    });
    if (jb < n) return fail(ctx, DEABM_EINVAL, "agent %u: not a stage code or qt bit 7 set", jb);
    cudaStream_t s = ctx->stream;
    DevScratch sc;
    uint16_t *d_in = nullptr;
    int r;
    if (ctx->relabel && (r = scratch_alloc(ctx, sc, &d_in, nb))) return r;
    const uint32_t *perm = ctx->relabel ? ctx->orig_id : nullptr;
    auto put = [&](void *dst, const void *src, uint32_t elem, uint32_t reps) -> int {
        if (!perm) {
            CU(ctx, cudaMemcpyAsync(dst, src, (size_t)n * reps * elem, cudaMemcpyHostToDevice, s));
        } else {
            CU(ctx, cudaMemcpyAsync(d_in, src, (size_t)n * reps * elem, cudaMemcpyHostToDevice, s));
            CU(ctx, launch_from_caller(dst, d_in, perm, n, reps, elem, true, s));
        }
        return DEABM_OK;
    };
    if ((r = put(ctx->S.stage, stage, 1, B))) return r;
    if ((r = put(ctx->S.timer, timer, 2, B))) return r;
    if ((r = put(ctx->S.tinf, tinf, 2, B))) return r;
    if ((r = put(ctx->S.flags, flags, 1, B))) return r;
    if ((r = put(ctx->S.qt, qt, 1, B))) return r;
    if (ctx->S.vd1) {
        if ((r = put(ctx->S.vd1, dose1_day, 2, B))) return r;
        if ((r = put(ctx->S.vd2, dose2_day, 2, B))) return r;
    }
    ctx->day = day;
    ctx->cur = 0;
    CU(ctx, clear_next_buffers(ctx, nb));
    CU(ctx, launch_emit(ctx->kp, ctx->S, ctx->inf[0], ctx->inf_rand[0], s));
    // counters of the days to come start from zero again
    const size_t rest = ctx->max_steps - day;
    CU(ctx, cudaMemsetAsync(ctx->C.new_inf + (size_t)day * B, 0, sizeof(int32_t) * rest * B, s));
    CU(ctx, cudaMemsetAsync(ctx->C.hist + (size_t)day * B * DEABM_N_STAGE, 0,
                            sizeof(int32_t) * rest * B * DEABM_N_STAGE, s));
    CU(ctx, cudaMemsetAsync(ctx->C.msgs + day, 0, sizeof(unsigned long long) * rest, s));
    CU(ctx, cudaMemsetAsync(ctx->C.gath + day, 0, sizeof(unsigned long long) * rest, s));
    CU(ctx, cudaMemsetAsync(ctx->C.den + (size_t)day * B, 0, sizeof(int32_t) * rest * B, s));
    if (ctx->kp.den_on) {
        CU(ctx, cudaMemsetAsync(ctx->den_pos + day, 0, sizeof(int32_t) * rest, s));
        const uint32_t W = ctx->kp.den_window;
        // (batched contexts keep no records: their pass redraws the contacts)
        if (ctx->n_rep == 1) CU(ctx, launch_den_records(ctx->kp, day + 1u > W ? day + 1u - W : 0u, day, s));
        if (ctx->kp.wsg_on)  // the Watts-Strogatz graphs of the look-back window's earlier days
            for (uint32_t d = day + 1u > W ? day + 1u - W : 0u; d < day; ++d) {
                KParams kd = ctx->kp;
                CU(ctx, wsg_day(ctx, kd, d));
            }
    }
    CU(ctx, cudaStreamSynchronize(s));  // host arrays and device scratch end here
    return DEABM_OK;
}

extern "C" int deabm_info(const deabm_ctx *ctx, uint32_t *day, uint32_t *n_agents, uint32_t *n_rep)
{
    if (!ctx) return fail(nullptr, DEABM_EINVAL, "ctx is NULL");
    if (day) *day = ctx->day;
    if (n_agents) *n_agents = ctx->n;
    if (n_rep) *n_rep = ctx->n_rep;
    return DEABM_OK;
}

extern "C" int deabm_sync(deabm_ctx *ctx)
{
    if (!ctx) return fail(nullptr, DEABM_EINVAL, "ctx is NULL");
    CU(ctx, cudaStreamSynchronize(ctx->stream));
    return DEABM_OK;
}

extern "C" const char *deabm_last_error(const deabm_ctx *ctx) { return ctx ? ctx->err.c_str() : g_err.c_str(); }

extern "C" void deabm_destroy(deabm_ctx *ctx)
{
    if (!ctx) return;
    if (!ctx->allocs.empty()) (void)cudaStreamSynchronize(ctx->stream);
    if (ctx->graph) (void)cudaGraphExecDestroy(ctx->graph);
    for (void *ptr : ctx->allocs) (void)cudaFree(ptr);
    if (ctx->own_stream) (void)cudaStreamDestroy(ctx->own_stream);
    delete ctx;
}
