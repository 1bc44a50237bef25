/*
 * deabm.h -- C ABI of the GB300 (sm_103a) DeepABM-COVID step library, libdeabm.so.
 *
 * The library runs the per-day simulation step of DeepABM-COVID (Chopra et al.,
 * "DeepABM: Scalable, efficient and differentiable agent-based simulations via
 * graph neural networks", arXiv 2110.04421) on one GPU:
 *   - Sec. 2.1 / Sec. 3 "Infection Transmission", Eq. 1-2: each interaction i->j
 *     carries R S_{a_j} A_{s_i} B_n / I * (integral over the day of the gamma
 *     infectiousness density); messages are summed per destination into lambda_j
 *     and p_j = 1 - exp(-lambda_j dt) (message passing over the interaction graph);
 *   - Sec. 3 "Interaction Networks": static household / occupation networks given
 *     as destination-sorted CSR, plus a random network regenerated every day on
 *     the device from a counter-based generator (Philox4x32-10);
 *   - Sec. 3 "Agent State Definition" / "Disease Progression": eleven disease
 *     stages, integer day timers, Bernoulli infection draw;
 *   - Sec. 4.1 self-quarantine, Sec. 4.3 testing, Sec. 4.4 / Sec. 5 two-dose
 *     vaccination.
 * Points the paper leaves open (stage durations, branch probabilities, random
 * stream layout, reduction order) follow one written reading; every random
 * decision is a function of (seed, agent, step, stream), so runs are exactly
 * reproducible and comparable with an independent implementation.
 *
 * Conventions for every entry point
 *   - Return DEABM_OK (0) or a negative DEABM_E* code; deabm_last_error() gives
 *     the message.  No entry point aborts the process.
 *   - Host pointers passed to create are read during the call only (the library
 *     copies everything it needs to device memory it owns).  Output pointers are
 *     caller-owned host buffers of the stated size.
 *   - The CUDA stream is borrowed (cudaStream_t passed as void*; NULL = the
 *     legacy default stream).  Work is queued on it; deabm_step returns without
 *     waiting; calls that return host data synchronise the stream.
 *   - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef DEABM_H
#define DEABM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DEABM_OK 0
#define DEABM_EINVAL (-1)   /* invalid argument, graph, state or parameter */
#define DEABM_ENOMEM (-2)   /* device or host allocation failed */
#define DEABM_ECUDA (-3)    /* a CUDA call failed (message has the CUDA error) */
#define DEABM_ETIMEOUT (-4) /* a bounded device wait gave up */
#define DEABM_ESTATE (-5)   /* call not valid in the context's current state */

#define DEABM_MAX_NETS 4
#define DEABM_N_AGE 9       /* age bins 0-10, 11-20, ..., 80+ (Sec. 3) */
#define DEABM_N_STAGE 11    /* disease stages (Sec. 3 "Agent State Definition") */
#define DEABM_N_CLASS 3     /* infector class: asymptomatic, mild, severe (Eq. 1, s_i) */
#define DEABM_MAX_INF_LEN 64
#define DEABM_POIS_CAP 15   /* random in-contacts per agent per day are capped here */
#define DEABM_N_REP_PARAMS 14

/* stage codes (int8) */
enum {
    DEABM_S = 0, DEABM_ASYM = 1, DEABM_PRE_MILD = 2, DEABM_PRE_SEV = 3, DEABM_MILD = 4,
    DEABM_SEV = 5, DEABM_HOSP = 6, DEABM_ICU = 7, DEABM_REC = 8, DEABM_VAX = 9, DEABM_DEAD = 10
};
/* flags byte: dose 1 given, dose 2 given, pending test is positive */
#define DEABM_FL_DOSE1 0x01u
#define DEABM_FL_DOSE2 0x02u
#define DEABM_FL_POS 0x04u
#define DEABM_FL_IMMUNE 0x08u  /* non-sterilising vaccine immunity (vax_nonsterile) */
#define DEABM_FL_DEN 0x10u     /* exposure notification received: tested on the next day (den_on) */
#define DEABM_FL_APP 0x20u     /* holds the exposure-notification app (den_on; drawn by the library) */
/* qt byte: bits 0..3 quarantine days left (0 = not quarantined),
 *          bits 4..6 days until a pending test result (0 = none) */

typedef struct deabm_ctx deabm_ctx;

/* Interaction graph (Sec. 3 "Interaction Networks").
 * n_nets static networks, each a destination-sorted CSR over n_agents rows:
 * row_ptr[k] has n_agents+1 entries with row_ptr[k][0] = 0 and non-decreasing
 * values; col[k] has row_ptr[k][n_agents] entries, each a source agent id
 * < n_agents and != its row (no self-loops).  Edge j <- col[e] for
 * e in [row_ptr[j], row_ptr[j+1]).  The in-edges of a row are summed in the
 * order listed.  rand_mean > 0 adds the daily random network: each agent j
 * receives K_j ~ Poisson(rand_mean) (capped at DEABM_POIS_CAP) in-contacts
 * drawn uniformly from the other agents, regenerated every day.  rand_by_age = 1
 * makes the mean age-stratified (Sec. 3 "Interaction Networks": each agent's
 * age-stratified number of random interactions parameterises the random
 * network): K_j ~ Poisson(rand_mean_age[age_bin_j]) (each 0..1000; the network
 * is on when one of them is > 0; rand_mean is then ignored).  Not with rand_ws
 * (which ignores both) and not in deabm_lambda_noalloc.
 *
 * n_occ > 0 adds the daily occupation networks (Sec. 3 "Interaction Networks":
 * an agent's occupation is fixed, whom it meets there changes every day).
 * occ_group[j] < n_occ is agent j's occupation (host array of n_agents); every
 * day a member of occupation g receives occ_k[g] <= DEABM_POIS_CAP in-contacts
 * (host array of n_occ), each uniform over the other members of g (none for a
 * lone member), contact e from word e of Philox stream 4 keyed by (net_seed,
 * day, agent) -- block e/4, lane e%4 -- mapped to the member in place
 * floor(word * (size-1) / 2^32), skipping the agent itself, members ranked by
 * ascending id.  occ_lattice = 1 makes each occupation a Watts-Strogatz small
 * world rewired every day instead: the members sit on a ring in ascending id;
 * in-edge e of the member at place q comes from the lattice place
 * q + (e/2 + 1) (e even) or q - (e/2 + 1) (e odd), mod the occupation's size,
 * unless word 2(e%2) of block e/2 of Philox stream 9 (same key and counter
 * words) is below floor(occ_rewire 2^32), or the lattice offset is a multiple
 * of the size: then it comes from the member in place floor(word' (size-1) /
 * 2^32), skipping the agent itself, word' = word 2(e%2)+1 of that block.
 * Their sum enters Eq. 1 with weight B_net[n_nets], after the
 * stored networks and before the random network, so n_nets must be <= 3.
 * Plain, batched and ragged contexts take them (deabm_create,
 * deabm_create_batch, deabm_create_ragged: a population with n_occ > 0 is
 * numbered in occupation order), and so does the relaxed model
 * (deabm_relaxed_create: the same daily contacts in its forward and reverse
 * sweep).  n_occ = 0: occ_group and occ_k are ignored. *
 * rand_ws = 1 replaces the Poisson contacts by the paper's form of the global
 * random network (Sec. 3 "Interaction Networks": one small-world Watts-Strogatz
 * graph, re-initialised every step; rand_mean is then ignored).  The ring
 * lattice runs over all agents in caller-id order; agent i owns the undirected
 * edges to (i + m) mod n_agents, m = 1..rand_ws_k/2.  Every day each owned edge
 * is rewired when word 2((m-1)%2) of block (m-1)/2 of Philox stream 10, keyed by
 * (net_seed, day, i), is below floor(rand_ws_beta 2^32), or when i + m wraps
 * onto i: its far end becomes agent floor(w (n-1) / 2^32), skipping i, w = word
 * 2((m-1)%2)+1 of that block.  A rewired edge leaves its lattice end and reaches
 * the new one, and both ends receive each other's messages.  Agent j's messages
 * are summed in this order: its own edges m = 1..k/2, the unrewired lattice
 * edges of agents j - m, m = 1..k/2, then the rewired edges that landed on j by
 * owner ascending and m ascending.  Plain and batched contexts (the graph,
 * keyed by net_seed, is shared by every replicate column; a batched context
 * then runs the general panel kernel) and ragged batches (each population its
 * own graph); the day's graph is built on the device before each day kernel
 * (three small kernels and a prefix sum).  With exposure notification an agent's in-contacts in this network are
 * its neighbours (the edges are undirected), and the graphs of the last
 * den_window days are kept for the look-back.
 */
typedef struct {
    uint32_t n_agents;
    uint32_t n_nets;
    const uint32_t *row_ptr[DEABM_MAX_NETS];
    const uint32_t *col[DEABM_MAX_NETS];
    float rand_mean;
    uint32_t n_occ;
    const uint32_t *occ_group;
    const uint8_t *occ_k;
    uint32_t occ_lattice; /* 0: as above; 1: Watts-Strogatz (see below) */
    float occ_rewire;     /* occ_lattice = 1: rewiring probability, 0..1 */
    uint32_t rand_ws;     /* 1: the random network is a daily Watts-Strogatz graph (see below) */
    uint32_t rand_ws_k;   /* rand_ws = 1: lattice neighbours, even, 2..16 */
    float rand_ws_beta;   /* rand_ws = 1: daily rewiring probability, 0..1 */
    uint32_t rand_by_age; /* 1: per-age-bin Poisson means rand_mean_age (see above) */
    float rand_mean_age[DEABM_N_AGE];
} deabm_graph;

/* Agents (Sec. 3 "Agent State Definition"); all host arrays of n_agents entries.
 * age_bin is required (0..8).  The dynamic state arrays may be NULL, meaning all
 * susceptible with zero timers.  seed_ids lists agents infected before day 0
 * (ignored for agents that are not susceptible). */
typedef struct {
    const uint8_t *age_bin;
    const int8_t *stage;
    const int16_t *timer;
    const int16_t *tinf;
    const uint8_t *flags;
    const uint8_t *qt;
    const uint32_t *seed_ids;
    uint32_t n_seed;
    const int16_t *dose1_day;  /* [N] or NULL: day of a first dose given before the run (priority strategies) */
    const int16_t *dose2_day;  /* [N] or NULL: day of a second dose given before the run; 0x7FFF = none */
} deabm_agents;

/* Model parameters.  Eq. 1 names: R, S_age (S_a), A_class (A_s), B_net (B_n),
 * inv_Ibar (1/I).  The infectiousness curve of class c is a gamma density of
 * shape inf_shape[c] and scale inf_scale[c], integrated over each day since
 * infection t = 1..inf_len-1 (day 0 and days >= inf_len contribute 0).
 * Probabilities are doubles in [0,1]; an event of probability p happens when
 * its 32-bit random word is < floor(p * 2^32).  dur_lo/dur_hi[stage][age]
 * bound the integer stage duration in days (stages 1..7; uniform on the range).
 * Test result delays are uniform on test_lo..test_hi days (1 <= lo <= hi <= 7);
 * quar_days <= 15.  Vaccination: from day vax_start, floor(vax_rate * N) first
 * doses a day in priority order (age bin descending, then id ascending) to
 * agents not in hospital, ICU or dead; the second dose dose2_delay days later;
 * a susceptible agent becomes immune (stage VAX) vax_onset days after a dose
 * when its per-agent vaccine word is below floor(eff * 2^32) of that dose.
 * seed keys the per-agent draws, net_seed the daily random network. */
typedef struct {
    float R, inv_Ibar, dt;
    float B_net[DEABM_MAX_NETS];
    float B_rand;
    float S_age[DEABM_N_AGE];
    float A_class[DEABM_N_CLASS];
    double inf_shape[DEABM_N_CLASS], inf_scale[DEABM_N_CLASS];
    uint32_t inf_len;
    double p_asym[DEABM_N_AGE], p_sev[DEABM_N_AGE], p_hosp[DEABM_N_AGE];
    double p_icu[DEABM_N_AGE], p_death[DEABM_N_AGE];
    uint8_t dur_lo[8][DEABM_N_AGE], dur_hi[8][DEABM_N_AGE];
    uint32_t test_on;
    double test_sens;
    uint32_t test_lo, test_hi;
    uint32_t quar_on, quar_days;
    double q_dropout;
    uint32_t vax_on, vax_start, vax_onset, dose2_delay;
    double vax_rate, vax_eff1, vax_eff2;
    uint64_t seed, net_seed;
    uint32_t max_steps;   /* capacity of the per-day counters (0 = 1024) */
    uint32_t keep_lambda; /* 1: keep lambda_j and p_j of the last day for deabm_get_state */
    uint32_t vax_strategy;   /* 0: static schedule above.  1, 2, 3: a shared supply of floor(vax_rate * N)
                                doses a day from vax_start, given by priority (Sec. 5, Table 1) to agents
                                due a first dose or due a second dose (first dose >= dose2_delay days ago),
                                none in hospital, ICU or dead; age bin descending inside each group:
                                1 standard (second doses first), 2 delayed second dose (first doses first),
                                3 delayed except the elderly (bins >= elderly_bin interleaved by age with a
                                first dose before a second, then the others' first doses, then their second
                                doses); ties by agent id.  Plain and batched contexts (in a batched
                                context every replicate column selects from its own state with its own
                                dose2_delay and the same supply; the general panel kernel then runs
                                the day instead of the four-replicate one) and ragged batches (each
                                population from its own state with its own supply; no initial dose
                                days there). */
    uint32_t elderly_bin;    /* first age bin counted as "65+" by strategy 3 */
    uint32_t vax_nonsterile; /* 0: immunity is sterilising (stage VAX); 1: non-sterilising (Sec. 5, second
                                version): the agent stays susceptible with flag DEABM_FL_IMMUNE and any
                                later infection is asymptomatic */
    uint32_t locality_order; /* 1: number the agents internally so that the members of a group sit
                                next to each other in device memory: agents grouped by the smallest
                                id reaching them along the in-edges of the stored network with the
                                most edges (up to 8 rounds of min-label propagation on the device,
                                fewer once no label moves), groups
                                in label order, ids ascending inside a group; results and every
                                array the ABI returns are unchanged (random draws and outputs use
                                the caller's agent ids) */
    /* Digital exposure notification (Sec. 4.2); plain and batched contexts and
     * ragged batches, with test_on.
     * At create (and reset) agent j gets DEABM_FL_APP when word x of Philox
     * stream 6 keyed (seed, j, day word 0xFFFFFFFD) is below floor(den_adoption
     * 2^32); in a batched context each replicate column draws its own app holders
     * (and compliance words) with its own seed, so column b reproduces the plain
     * run with that seed.  An app holder whose positive test result lands on day t notifies,
     * after every agent's update of day t, each app holder that is out of
     * quarantine, not in hospital, ICU or dead, and had it as an in-contact on one
     * of the days max(0, t-den_window+1) .. t (stored networks, daily occupation
     * and random networks); a notified agent sets DEABM_FL_DEN when word x of
     * stream 6 keyed (seed, j, t) is below floor(den_compliance 2^32) and takes a
     * test on day t+1 unless a result is pending or it is quarantined.  Any test
     * is positive only for an agent in stages 1..5 (with probability test_sens).
     * den_window: 1..64 days (7 in Sec. 4.2). */
    uint32_t den_on;
    double den_adoption, den_compliance;
    uint32_t den_window;
} deabm_params;

/* Create a plain (one replicate) simulation: the population of Sec. 3 "Agent
 * State Definition" on the interaction networks of Sec. 3 "Interaction Networks",
 * with the infectiousness curve of Eq. 1 (its daily integrals, built on the
 * device) and the vaccination schedule of Sec. 4.4 / Sec. 5.  Validates the graph
 * (monotone row_ptr, col < n_agents, no self-loops, < 2^32 edges), the agents
 * (age bins, stage codes) and the parameters, copies everything to the device on
 * `stream` and infects seed_ids.  The network weights B_n travel in params, not
 * in the graph: they are per-replicate parameters of Eq. 1 (varied across the
 * columns of a batch), while the graph is shared.  On success *out owns all
 * device memory it allocated.  Errors: DEABM_EINVAL, DEABM_ENOMEM, DEABM_ECUDA. */
int deabm_create(const deabm_graph *graph, const deabm_agents *agents, const deabm_params *params,
                 void *cuda_stream, deabm_ctx **out);

/* Create a batch of n_rep replicates sharing one graph (state laid out [N][n_rep],
 * replicate fastest).  rep_params is a host [n_rep][14] float array:
 * R, B_net[0], B_net[1], B_rand, S_age[0..8], dose2_delay (whole days); the
 * other parameters come from `base`.  rep_seeds [n_rep] keys each replicate's
 * per-agent draws; all replicates share the day's random network (base->net_seed).
 * Replicate r reproduces deabm_create with those parameters and seed exactly.
 * 1 <= n_rep <= 1024. */
int deabm_create_batch(const deabm_graph *graph, const deabm_agents *agents, const deabm_params *base,
                       uint32_t n_rep, const float *rep_params, const uint64_t *rep_seeds,
                       void *cuda_stream, deabm_ctx **out);

/* Create a ragged batch: n_pops independent populations of different sizes
 * (graphs[q], agents[q], params[q] each as for deabm_create; no keep_lambda:
 * DEABM_EINVAL otherwise) simulated together, one
 * kernel launch per day for all of them (after the day's dose selection of each
 * population under a vaccination priority strategy, Sec. 5 Table 1, and the day's
 * graph of each population with a Watts-Strogatz random network: a few small
 * launches per such population; followed by the notification pass of each
 * population with exposure notification, Sec. 4.2, one launch each):
 * resident thread blocks take tiles of
 * rows (never spanning two populations) from a per-day work queue.  A population
 * whose params ask for locality_order is numbered internally like a plain
 * context (its random contacts reach rows through a caller id -> row map).
 * Population q's results equal those of deabm_create on its own inputs.  State arrays are
 * concatenated in population order (sum of n_agents entries); per-day counters
 * are [day][population] (deabm_info's n_rep = n_pops).  deabm_run captures its T
 * days as one CUDA graph and replays it; a NULL stream here means a stream the
 * context creates (capture needs a stream other than the legacy default one).
 * deabm_reset restarts at day 0 with the same parameters (rep_params must be NULL). */
int deabm_create_ragged(uint32_t n_pops, const deabm_graph *graphs, const deabm_agents *agents,
                        const deabm_params *params, void *cuda_stream, deabm_ctx **out);

/* Ragged batches only: time days_per_trial days for each candidate tiling (rows
 * per tile 256..4096, resident blocks per SM 2..8) on this context's own data,
 * keep the fastest and restart at day 0.  Either output may be NULL.  Synchronises. */
int deabm_autotune(deabm_ctx *ctx, uint32_t days_per_trial, uint32_t *rows_per_tile, uint32_t *blocks_per_sm);

/* Queue n_steps days on the context's stream and return without waiting.  One
 * day is one step of the simulation (Sec. 2.1 message passing; Sec. 3
 * "Infection Transmission", Eq. 1-2, the draw; Sec. 3 "Disease Progression" and
 * Sec. 4 interventions, the state update), all agents updated from the state at
 * the start of the day.  DEABM_ESTATE if the day counter would pass max_steps. */
int deabm_step(deabm_ctx *ctx, uint32_t n_steps);

/* Run T days, then copy the per-day counters of those days to the host and
 * synchronise.  new_inf: host int32 [T][n_rep] new infections per day;
 * hist: host int32 [T][n_rep][11] stage counts after each day, or NULL (the
 * daily incidence and stage curves the paper reports, Sec. 4.5 and Sec. 5). */
int deabm_run(deabm_ctx *ctx, uint32_t T, int32_t *new_inf, int32_t *hist);

/* Copy the current state (host arrays of n_agents * n_rep entries; any may be
 * NULL): the stage of Sec. 3 "Agent State Definition" and the timers of "Disease
 * Progression"; and, if params.keep_lambda was set, lambda (Eq. 1 summed over the
 * agent's interactions) and p = 1 - exp(-lambda dt) (Eq. 2) of the last day.
 * Caller's agent order.  Synchronises the stream. */
int deabm_get_state(deabm_ctx *ctx, int8_t *stage, int16_t *timer, int16_t *tinf, uint8_t *flags,
                    uint8_t *qt, float *lambda, float *p);

/* Days of each agent's first and second dose under a priority strategy
 * (host int16 [n_agents][n_rep] in caller order, 0x7FFF = none; either may be
 * NULL; ragged batches: the populations' agents concatenated, 0x7FFF throughout
 * a population without a strategy).  Synchronises. */
int deabm_get_dose_days(deabm_ctx *ctx, int16_t *dose1_day, int16_t *dose2_day);

/* Per-day counters already run: days [0, day_count) of new infections
 * [day][n_rep], stage histogram [day][n_rep][11] (Sec. 4.5 outcomes) and
 * messages processed [day] (static in-edges + that day's random in-contacts, per
 * replicate: the paper's interactions, Abstract and Sec. 1).
 * Any output may be NULL.  Synchronises. */
int deabm_get_counters(deabm_ctx *ctx, uint32_t day_count, int32_t *new_inf, int32_t *hist,
                       uint64_t *messages);

/* Messages gathered per day, days [0, day_count) (host uint64 [day]): the
 * in-contacts (stored, occupation, random) of the destinations that evaluated
 * Eq. 1 -- the agents susceptible at the start of the day (Eq. 2 applies to them
 * alone), or every agent when lambda is kept or exposure notification is on --
 * summed over populations in ragged batches.  The batched kernels gather every
 * agent's in-contacts for every replicate, so there this equals the messages of
 * deabm_get_counters.  Returns DEABM_OK, DEABM_EINVAL (NULL, more days than
 * run), DEABM_ECUDA.  Synchronises. */
int deabm_get_gathered(deabm_ctx *ctx, uint32_t day_count, uint64_t *gathered);

/* Tables the device built: infectiousness [3][inf_len] (FP32), Poisson CDF
 * thresholds [15], first-dose day per agent [n_agents] (0x7FFF = never).
 * Any output may be NULL.  Synchronises. */
int deabm_get_tables(deabm_ctx *ctx, float *inf_table, uint64_t *poisson_thr, int16_t *dose1_day);

/* Restart a context at day 0 with new per-replicate parameters and seeds (same
 * layout as deabm_create_batch; both NULL keeps the current ones): the initial
 * state given at create is restored, the initial cases are infected again with
 * the new seeds, the per-day counters are cleared.  Lets one context generate
 * many ensembles without re-uploading the graph.  Asynchronous. */
int deabm_reset(deabm_ctx *ctx, const float *rep_params, const uint64_t *rep_seeds);

/* Checkpoint and resume.  Draws are keyed by (seed, agent, day, stream), so the
 * state at the start of a day plus the day index determine every later day
 * exactly.  deabm_save writes the state at the start of the next day to run
 * (stage, timer, tinf, flags, qt: host arrays [n_agents][n_rep] in caller order,
 * as deabm_get_state) and, under a priority strategy, the dose days (host
 * [n_agents][n_rep], 0x7FFF = none; NULL otherwise); *day receives the day index.
 * deabm_restore puts such a state back into a context created with the same
 * graph and parameters (this one or another) and sets its day: the next
 * deabm_step runs that day.  The day's emitted infectiousness is rebuilt from
 * the state, exposure-notification records of the previous den_window - 1 days
 * are redrawn from their Philox words, and the per-day counters of days >= day
 * are cleared (earlier ones are kept as they are).  Plain and batched contexts;
 * DEABM_ESTATE for ragged batches.  Any array may be NULL on save; on restore
 * stage..qt are required and checked like deabm_create's.  Returns DEABM_OK,
 * DEABM_EINVAL (day > max_steps, bad codes), DEABM_ESTATE, DEABM_ECUDA.
 * Synchronises. */
int deabm_save(deabm_ctx *ctx, int8_t *stage, int16_t *timer, int16_t *tinf, uint8_t *flags, uint8_t *qt,
               int16_t *dose1_day, int16_t *dose2_day, uint32_t *day);
int deabm_restore(deabm_ctx *ctx, const int8_t *stage, const int16_t *timer, const int16_t *tinf,
                  const uint8_t *flags, const uint8_t *qt, const int16_t *dose1_day, const int16_t *dose2_day,
                  uint32_t day);

/* Failure injection for tests (the paper has no counterpart; off by default): the
 * `after`-th device allocation made from now on by a simulation context (create,
 * batch, ragged; arrays and set-up scratch) fails as if cudaMalloc had run out of
 * memory -- the call reports DEABM_ENOMEM and releases everything it had
 * allocated -- and the injection switches itself off.  after = 0 switches it
 * off.  Process-wide; meant for single-threaded tests. */
void deabm_inject_alloc_failure(uint32_t after);

/* ---- Infection rates of one day without allocating memory ------------------------------
 * The paper has no counterpart: this is a library convenience.  It exists for
 * callers that may not allocate device memory where they call us (code living
 * inside a memory pool another runtime sized up front, hosts whose allocator
 * hooks forbid cudaMalloc after start-up, real-time loops that cannot afford an
 * allocation).  Everything the caller owns is passed in: graph_dev has the same
 * layout as deabm_graph but its row_ptr / col arrays are DEVICE pointers, and so
 * are age_bin, stage, tinf, qt (n_agents entries each, caller numbering, the
 * state at the start of `day`) and the output lambda (float[n_agents]).  The
 * device arrays cannot be checked on the host: the CSR rules of deabm_create
 * apply and invalid indices are the caller's error; a stage code outside 0..10
 * emits nothing; an age_bin outside 0..8 gives lambda = NaN for that agent (no
 * read outside the parameter block).  graph_dev->n_occ must be 0 (daily
 * occupation networks need a context, DEABM_EINVAL otherwise).  lambda_j equals what deabm_step computes for that day
 * and state (Eq. 1 summed over the static networks and the day's random network,
 * with params' R, inv_Ibar, B_net, B_rand, S_age, A_class, infectiousness curve
 * and net_seed).
 * Working memory: a fixed array compiled into the library (4 MiB + 4 KiB on every
 * GPU that loads it, held until the process exits).  At most
 * DEABM_NOALLOC_MAX_AGENTS agents; larger populations get DEABM_EINVAL before
 * any GPU work.  No cudaMalloc, cudaFree or other allocating call is made.  Every
 * call looks up the array's device address on the current device (where the
 * caller's buffers must live); the first lookup on a device may load the
 * library's device code there, so make the first call on each device before any
 * stream capture.
 * All calls share the array and it keeps the last call's contents; calls whose
 * GPU work overlaps (other streams or threads) race, so serialise them.  Work is
 * queued on cuda_stream and the call returns without waiting.  Errors:
 * DEABM_EINVAL, DEABM_ECUDA; message from deabm_lambda_noalloc_last_error(). */
#define DEABM_NOALLOC_MAX_AGENTS 1048576u
int deabm_lambda_noalloc(const deabm_graph *graph_dev, const uint8_t *age_bin, const int8_t *stage,
                         const int16_t *tinf, const uint8_t *qt, const deabm_params *params, uint32_t day,
                         float *lambda, void *cuda_stream);
const char *deabm_lambda_noalloc_last_error(void);

/* Exposure notification (Sec. 4.2, den_on): notified[d][b] = agents of replicate
 * column b notified at the end of day d, for d < day_count (day_count <= days
 * run; host array of day_count x n_rep int32, n_rep = 1 in plain contexts).
 * Zeros when den_on = 0 (ragged batches: [d][population], zeros in the columns
 * of populations without exposure notification).  Returns
 * DEABM_OK, DEABM_EINVAL, DEABM_ECUDA. */
int deabm_get_notified(deabm_ctx *ctx, uint32_t day_count, int32_t *notified);

/* Days run so far, agents, replicates. */
int deabm_info(const deabm_ctx *ctx, uint32_t *day, uint32_t *n_agents, uint32_t *n_rep);

/* Wait for all queued work on the context's stream. */
int deabm_sync(deabm_ctx *ctx);

/* Message of the last error on ctx (or of the calling thread when ctx is NULL).
 * The string stays valid until the next call on the same ctx / thread. */
const char *deabm_last_error(const deabm_ctx *ctx);

/* Free all device memory of ctx (the library-side lifetime of the simulated
 * population; the paper has no counterpart).  NULL-safe. */
void deabm_destroy(deabm_ctx *ctx);

/* ------------------------------------------------------------------------------------------
 * Relaxed (differentiable) simulation for gradient-based calibration.
 * The paper proposes learning the simulator's parameters by gradient descent
 * against aggregate data ("inverse" simulation: Abstract, Sec. 1, Sec. 6) but
 * defines no relaxation.  The model here (one reading, stated in full):
 *   each agent's symptom class is drawn once before day 0 (asymptomatic with
 *   p_asym[age], else severe with p_sev[age], else mild);  x_j(t), s_j(t) are the
 *   infected / susceptible mass of agent j (initial cases: x(-1) = 1, s(0) = 0);
 *   inf_i(t) = sum_{d=1}^{inf_len-1} A_c infT_c[d] x_i(t-d);  lambda_j(t) as in Eq. 1
 *   over the static networks, the day's occupation contacts (graph->n_occ > 0, weight
 *   B_net[n_nets]) and the day's random network;
 *   g_j(t) = sigmoid((log(expm1(lambda_j)) + l_j(t)) / tau) with logistic noise
 *   l = log(u) - log(1-u), u = ((w >> 8) + 0.5) 2^-24, w = Philox(seed; j, t, 8, 0).x
 *   (a binary Gumbel-softmax relaxation of the Eq. 2 draw);
 *   x_j(t) = s_j(t) g_j(t);  s_j(t+1) = s_j(t) - x_j(t);  I(t) = sum_j x_j(t);
 *   loss = (1/T) sum_t (log(I(t) + 1) - target_t)^2.
 * theta (host float[13]) = R, B_net[0], B_net[1], B_rand, S_age[0..8]; B_net[2..3],
 * inv_Ibar, A_class, the infectiousness curve, seed and net_seed come from params.
 * Error messages of these calls: deabm_relaxed_last_error() (per thread).
 * ------------------------------------------------------------------------------------------ */
#define DEABM_N_THETA 13
typedef struct deabm_relaxed deabm_relaxed;

/* Validate and copy the graph (and build its transpose), age bins and initial
 * cases (agents->seed_ids; the dynamic state arrays are ignored).  max_days
 * bounds T of later calls; the reverse sweep keeps a checkpoint every
 * ckpt_every days and recomputes the days in between.  tau > 0.
 * Errors: DEABM_EINVAL, DEABM_ENOMEM, DEABM_ECUDA. */
int deabm_relaxed_create(const deabm_graph *graph, const deabm_agents *agents, const deabm_params *params,
                         float tau, uint32_t max_days, uint32_t ckpt_every, void *cuda_stream,
                         deabm_relaxed **out);

/* Forward T days at theta; incidence (host float[T], may be NULL) = I(t).  Synchronises. */
int deabm_relaxed_forward(deabm_relaxed *ctx, uint32_t T, const float *theta, float *incidence);

/* Loss and its gradient d loss / d theta (host float[13]) at theta against
 * target (host float[T], log(I*(t) + 1)); incidence (float[T]) may be NULL.
 * Forward with checkpoints, then the reverse sweep along the transpose of every
 * network (the day's random contacts regenerated).  Synchronises. */
int deabm_grad(deabm_relaxed *ctx, uint32_t T, const float *theta, const float *target, float *loss, float *grad,
               float *incidence);

/* The loss and gradient of B parameter columns at once (the Abstract's and
 * Sec. 1's gradient-based calibration over many candidate parameter sets): theta
 * host float[B][13] (each >= 0, finite), target host float[T][B] (column b =
 * log(I*_b(t) + 1)); loss float[B], grad float[B][13] (d loss_b / d theta_b) and
 * incidence float[T][B] are host outputs, any may be NULL (target is required for
 * loss and grad).  The columns share the graph, the initial cases and the
 * relaxed draw's noise; each column's per-agent sums run as in deabm_grad, with
 * agent state laid out [agent][column], so every day reads each edge list once
 * for all columns.  Device arrays for B columns are allocated on the first call
 * that needs them (about (L + 1) (T / ckpt_every + 2) + 7 ckpt_every floats per
 * agent and column; DEABM_ENOMEM if they do not fit) and kept for later calls.
 * 1 <= B <= 4096.  Synchronises.  Errors: DEABM_EINVAL, DEABM_ENOMEM, DEABM_ECUDA. */
int deabm_grad_batch(deabm_relaxed *ctx, uint32_t T, uint32_t B, const float *theta, const float *target,
                     float *loss, float *grad, float *incidence);

/* `steps` Adam steps (lr; beta 0.9 / 0.999; eps 1e-8; parameters kept >= 0)
 * from theta0 against target, entirely on the device.  theta_out (float[13])
 * and loss_trace (float[steps], the loss before each step) may be NULL. */
int deabm_calibrate(deabm_relaxed *ctx, uint32_t T, const float *theta0, const float *target, uint32_t steps,
                    float lr, float *theta_out, float *loss_trace);

const char *deabm_relaxed_last_error(void);

/* Free all device memory of ctx.  NULL-safe. */
void deabm_relaxed_destroy(deabm_relaxed *ctx);

/* ------------------------------------------------------------------------------------------
 * Learned surrogate: an MLP from the 14 simulation parameters to the daily
 * log incidence (not in the paper, which only hopes to bring agent-based models
 * and learning closer, Sec. 6).  n_in -> hidden x depth (GELU, tanh form:
 * z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))) -> n_out,
 * BF16 operands with FP32 accumulation on the tensor cores, FP32 master weights.
 * Parameter layout (FP32, host): for each layer l, W_l [fan_in x fan_out]
 * row-major, then b_l [fan_out].  Data pointers x / y are DEVICE FP32 arrays
 * [batch x n_in] / [batch x n_out] (the caller's allocation).  Errors:
 * deabm_mlp_last_error() (per thread).
 * ------------------------------------------------------------------------------------------ */
typedef struct deabm_mlp deabm_mlp;

/* hidden % 8 == 0, n_out even, 1 <= depth <= 16, batch <= max_batch <= 2^22. */
int deabm_mlp_create(uint32_t n_in, uint32_t hidden, uint32_t depth, uint32_t n_out, uint32_t max_batch,
                     void *cuda_stream, deabm_mlp **out);
int deabm_mlp_param_count(const deabm_mlp *mlp, uint64_t *count);
/* Load FP32 parameters (host, layout above) and reset the Adam state.  Synchronises. */
int deabm_mlp_set_params(deabm_mlp *mlp, const float *params);
/* Copy the FP32 parameters and / or the last computed gradients (host; either may be NULL). */
int deabm_mlp_get_params(deabm_mlp *mlp, float *params, float *grads);
/* y = MLP(x) for `batch` rows (device pointers).  Asynchronous.  When the shape
 * allows (n_in <= 64, hidden a multiple of 64 up to 256, n_out <= 256) this is one
 * fused kernel on the tcgen05 tensor cores with the accumulator in TMEM;
 * otherwise, or after deabm_mlp_use_tcgen05(mlp, 0, ...), the per-layer
 * mma.sync GEMMs run.  A bounded wait that gave up inside the fused kernel is
 * reported by the next deabm_mlp_sync as DEABM_ETIMEOUT. */
int deabm_mlp_forward(deabm_mlp *mlp, const float *x, uint32_t batch, float *y);
/* Choose the forward path (1: fused tcgen05 when eligible, 0: per-layer GEMMs);
 * *available (may be NULL) tells whether the fused path applies to this shape. */
int deabm_mlp_use_tcgen05(deabm_mlp *mlp, int enable, int *available);
/* Loss (1/(batch n_out)) sum (MLP(x) - y)^2 and its gradients (kept in the
 * context, read with deabm_mlp_get_params); loss -> host float, may be NULL.
 * On the fused-forward shapes (see deabm_mlp_forward) and with tcgen05 enabled,
 * the forward pass that keeps its activations, the input gradients and the
 * weight gradients are GEMMs on the tcgen05 tensor cores (TMA operand tiles,
 * TMEM accumulators; weight gradients split over the batch and summed in a fixed
 * order); otherwise the per-layer mma.sync GEMMs.  A bounded wait that gave up
 * is reported by the next deabm_mlp_sync as DEABM_ETIMEOUT. */
int deabm_mlp_grad(deabm_mlp *mlp, const float *x, const float *y, uint32_t batch, float *loss);
/* deabm_mlp_grad, then one Adam step (beta 0.9 / 0.999, eps 1e-8) with rate lr.
 * loss (host, may be NULL: no synchronisation) is the loss before the step. */
int deabm_mlp_train_step(deabm_mlp *mlp, const float *x, const float *y, uint32_t batch, float lr, float *loss);
/* One Adam step (Kingma and Ba, Algorithm 1: beta 0.9 / 0.999, eps 1e-8, the
 * context's own moments and step count) with rate lr on gradients the caller
 * supplies, e.g. gradients summed over data-parallel ranks.  grads: FP32 in the
 * deabm_mlp_get_params layout (per layer W [fan_in x fan_out] row-major, then b);
 * a device pointer when on_device != 0 (queued, asynchronous), else a host
 * pointer (copied, then the call waits for the step).  deabm_mlp_train_step is
 * deabm_mlp_grad followed by this step.  Returns DEABM_OK, DEABM_EINVAL (NULL,
 * lr not finite and > 0), DEABM_ECUDA. */
int deabm_mlp_apply_grads(deabm_mlp *mlp, const float *grads, uint32_t on_device, float lr);
/* Bound of every wait inside the tcgen05 kernels (on a copy or an MMA landing):
 * `polls` potentially blocking tries, 2^26 by default (0 restores it); 1 = one
 * non-blocking test, so a wait that is not already satisfied gives up at once.  A
 * kernel whose wait gave up records it, waits (with the default bound) for the
 * copies and MMAs it had started, frees its Tensor Memory and returns; the next
 * deabm_mlp_sync reports DEABM_ETIMEOUT and the context stays usable.  Returns
 * DEABM_OK, DEABM_EINVAL (NULL). */
int deabm_mlp_set_wait_limit(deabm_mlp *mlp, uint32_t polls);
/* Wait for the MLP's queued work; DEABM_ETIMEOUT if a bounded device wait gave up. */
int deabm_mlp_sync(deabm_mlp *mlp);
const char *deabm_mlp_last_error(void);
/* NULL-safe. */
void deabm_mlp_destroy(deabm_mlp *mlp);

#ifdef __cplusplus
}
#endif
#endif /* DEABM_H */
