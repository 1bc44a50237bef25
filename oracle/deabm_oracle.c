/*
 * deabm_oracle.c -- plain, slow CPU oracle of the DeepABM-COVID simulation step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this file's library.  It shares no code, header,
 * table or constant generator with the CUDA path; both sides are written from
 * the paper (DeepABM, Chopra et al., arXiv 2110.04421) and from the written
 * readings of the points the paper leaves open.
 *
 * What one step computes (Sec. 3 "Infection Transmission", Eq. 1-2; Sec. 3
 * "Disease Progression"; Sec. 4 interventions):
 *   inf_i      = A_{c(i)} * infT[c(i)][tinf_i]   if i is infectious and not quarantined, else 0
 *   infT[c][t] = integral_{t-1}^{t} gamma_pdf(u; shape_c, scale_c) du           (Eq. 1)
 *   H_{n,j}    = sum over the in-edges of j in static network n of inf_src, in CSR order
 *   O_j        = sum over the day's occupation in-contacts of j of inf_src, in draw order
 *                (optional: occupation membership fixed, contacts drawn anew each step)
 *   Rn_j       = sum over the k_j daily random in-contacts of j of inf_src, in draw order
 *   lambda_j   = (R*inv_Ibar) * S_{age_j} * (sum_n B_n H_{n,j} + B_o O_j + B_r Rn_j)  (Eq. 1 summed)
 *   p_j        = 1 - exp(-lambda_j dt)                                             (Eq. 2, aggregated)
 *   infected   = stage_j == S  and  u_j < p_j
 * followed by the integer stage/timer machine, testing, quarantine and vaccination.
 *
 * Every loop below is a literal per-agent / per-edge loop.  Floating point sums
 * run left to right from +0.0f in the order the CSR lists the edges; products
 * are rounded one at a time (build with -ffp-contract=off).  A parallel FP64
 * path (same order, unrounded infectiousness) gives the accuracy reference.
 *
 * Threads: the per-agent loops may run on several host threads (OpenMP over
 * agents, or_set_threads; one thread by default).  Each agent's sums, draw and
 * update touch only that agent's outputs and read the state of the start of the
 * step, and the counters are integer sums, so every thread count gives the same
 * results bit for bit.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

/* ---- disease stages (Sec. 3 "Agent State Definition": eleven values) ---- */
enum {
    ST_S = 0, ST_ASYM = 1, ST_PRE_MILD = 2, ST_PRE_SEV = 3, ST_MILD = 4, ST_SEV = 5,
    ST_HOSP = 6, ST_ICU = 7, ST_REC = 8, ST_VAX = 9, ST_DEAD = 10
};
#define OR_N_STAGE 11
#define OR_N_AGE 9
#define OR_N_CLASS 3
#define OR_MAX_NETS 4
#define OR_MAX_INF_LEN 64
#define OR_POIS_CAP 15

/* flags byte */
#define FL_DOSE1 0x01u
#define FL_DOSE2 0x02u
#define FL_POS 0x04u
#define FL_IMMUNE 0x08u  /* non-sterilising vaccine immunity: infections are asymptomatic (Sec. 5) */
#define FL_DEN 0x10u     /* exposure notification received: test on the next step (Sec. 4.2) */
#define FL_APP 0x20u     /* holds the exposure-notification app (Sec. 4.2) */
/* qt byte: low nibble = quarantine days left, bits 4..6 = days until the test result */
#define QT_QDAYS(q) ((q) & 0x0Fu)
#define QT_TCD(q) (((q) >> 4) & 0x07u)
#define QT_MAKE(qd, cd) ((uint8_t)(((qd) & 0x0Fu) | (((cd) & 0x07u) << 4)))

/* Philox counter word 2 ("stream") values */
#define SM_INF 0u     /* x: infection uniform, y: quarantine dropout */
#define SM_PROG 1u    /* x: asymptomatic?, y: duration, z: severe?, w: secondary branch */
#define SM_RNET 3u    /* random network: word 0 = contact count, words 1.. = contacts */
#define SM_OCC 4u     /* daily occupation network: word e = contact e */
#define SM_TEST 5u    /* x: test positive?, y: result delay */
#define SM_DEN 6u     /* x: complies with a notification; step word 0xFFFFFFFD: x = holds the app */
#define SM_VAX 7u     /* x: vaccine response (step word fixed at 0) */
#define SM_GUMBEL 8u  /* relaxed draw noise */
#define SM_WS 9u      /* Watts-Strogatz occupation contacts: block e/2, lanes 2(e%2), 2(e%2)+1 = rewire coin, place */
#define SM_WSG 10u    /* Watts-Strogatz global random network: edge m of agent i in block (m-1)/2, lanes
                         2((m-1)%2), 2((m-1)%2)+1 = rewire coin, new far end */

typedef struct {
    uint32_t n, n_nets;
    const uint32_t *row_ptr[OR_MAX_NETS];
    const uint32_t *col[OR_MAX_NETS];
    float B_net[OR_MAX_NETS];
    float rand_mean, B_rand;
    float R, inv_Ibar, dt;
    float S_age[OR_N_AGE];
    float A_class[OR_N_CLASS];
    double inf_shape[OR_N_CLASS], inf_scale[OR_N_CLASS];
    uint32_t inf_len;
    double p_asym[OR_N_AGE], p_sev[OR_N_AGE], p_hosp[OR_N_AGE], p_icu[OR_N_AGE], p_death[OR_N_AGE];
    uint8_t dur_lo[8][OR_N_AGE], dur_hi[8][OR_N_AGE];
    uint32_t test_on;  double test_sens; uint32_t test_lo, test_hi;
    uint32_t quar_on, quar_days; double q_dropout;
    uint32_t vax_on, vax_start, vax_onset, dose2_delay;
    double vax_rate, vax_eff1, vax_eff2;
    uint64_t seed, net_seed;
    uint32_t vax_strategy;  /* 0 static schedule; 1 standard, 2 delayed second dose, 3 delayed except elderly */
    uint32_t elderly_bin;   /* first age bin counted as "65+" by strategy 3 */
    uint32_t vax_nonsterile; /* 1: immunity is non-sterilising (Sec. 5, second version) */
    /* daily occupation networks (Sec. 3, Interaction Networks: fixed membership,
     * contacts drawn anew every step); n_occ = 0: none.  Its weight is
     * B_net[n_nets], after the stored networks. */
    uint32_t n_occ;
    const uint32_t *occ_group; /* [n] occupation of each agent, < n_occ */
    const uint8_t *occ_k;      /* [n_occ] in-contacts per agent per step, <= 15 */
    uint32_t occ_lattice;      /* 0: contacts uniform over the occupation; 1: Watts-Strogatz ring lattice */
    float occ_rewire;          /* lattice in-edges rewired each step with this probability */
    /* digital exposure notification (Sec. 4.2) */
    uint32_t den_on;
    double den_adoption, den_compliance;
    uint32_t den_window;       /* steps of contacts looked back over, >= 1 */
    /* the global random network as a Watts-Strogatz graph re-initialised every
     * step (Sec. 3, Interaction Networks) instead of the Poisson contacts:
     * rand_ws_k lattice neighbours (even, 2..16), rewiring probability rand_ws_beta */
    uint32_t rand_ws, rand_ws_k;
    double rand_ws_beta;
    /* age-stratified random interactions (Sec. 3, Interaction Networks: each
     * agent's age-stratified number of random interactions parameterises the
     * random network): with rand_by_age set, agent j's daily in-contact count is
     * Poisson(rand_mean_age[age_j]) instead of Poisson(rand_mean) */
    uint32_t rand_by_age;
    float rand_mean_age[OR_N_AGE];
} or_model;

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
 * multiply-xor round on a 128-bit counter with a Weyl-sequence key schedule. */
void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t m0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t m1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(m0 >> 32), lo0 = (uint32_t)m0;
        uint32_t hi1 = (uint32_t)(m1 >> 32), lo1 = (uint32_t)m1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* draw (agent, step, stream, word-block) under a 64-bit seed */
static void draw4(uint64_t seed, uint32_t agent, uint32_t step, uint32_t stream, uint32_t blk, uint32_t out[4])
{
    uint32_t ctr[4] = {agent, step, stream, blk};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox(ctr, key, out);
}

/* event with probability p decided by a 32-bit word: word < floor(p * 2^32) */
uint64_t or_threshold(double p)
{
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return (uint64_t)1 << 32;
    return (uint64_t)floor(p * 4294967296.0);
}

static int happens(uint32_t word, double p) { return (uint64_t)word < or_threshold(p); }

/* integer uniform on {lo..hi} from a 32-bit word (multiply-shift) */
static uint32_t uniform_int(uint32_t word, uint32_t lo, uint32_t hi)
{
    uint64_t span = (uint64_t)(hi - lo + 1u);
    return lo + (uint32_t)(((uint64_t)word * span) >> 32);
}

/* ------------------------------------------------------------------------- */
/* Eq. 1's integral: gamma density integrated over one day, by direct quadrature
 * of the density: 16 equal panels on [t-1, t], 20-point Gauss-Legendre on each.
 * The nodes are the roots of the Legendre polynomial P_20 found by Newton
 * iteration on the three-term recurrence; w_i = 2 / ((1 - x_i^2) P_20'(x_i)^2). */
static double gl_x[20], gl_w[20];
static int gl_ready = 0;

static void gl_init(void)
{
    const int n = 20;
    for (int i = 0; i < n; ++i) {
        double x = cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            double dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1; p1 = p2;
        }
        double dp = n * (x * p1 - p0) / (x * x - 1.0);
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    gl_ready = 1;
}

double or_gamma_pdf(double u, double shape, double scale)
{
    if (u <= 0.0) return 0.0;
    return exp((shape - 1.0) * log(u) - u / scale - lgamma(shape) - shape * log(scale));
}

/* regularized lower incomplete gamma P(s, x) by its power series
 * P(s, x) = x^s e^{-x} sum_{m>=0} x^m / Gamma(s + m + 1)  (the gamma CDF at x*scale) */
static double lower_gamma_series(double s, double x)
{
    if (x <= 0.0) return 0.0;
    double term = exp(s * log(x) - x - lgamma(s + 1.0)), sum = term;
    for (int m = 1; m < 100000; ++m) {
        term *= x / (s + m);
        sum += term;
        if (term < sum * 1e-17) break;
    }
    return sum;
}

/* integral of the gamma density over [a, b] (0 <= a < b).  An interval that
 * starts at 0 (where the density of a shape below 2 is not smooth) is the gamma
 * CDF itself, taken from its series; any other interval is integrated by
 * quadrature of the density, which avoids the cancellation of F(b) - F(a). */
double or_gamma_integral(double a, double b, double shape, double scale)
{
    if (!gl_ready) gl_init();
    if (b <= 0.0) return 0.0;
    if (a <= 0.0) return lower_gamma_series(shape, b / scale);
    const int panels = 16;
    double h = (b - a) / panels, total = 0.0;
    for (int p = 0; p < panels; ++p) {
        double lo = a + p * h, mid = lo + 0.5 * h, s = 0.0;
        for (int i = 0; i < 20; ++i) s += gl_w[i] * or_gamma_pdf(mid + 0.5 * h * gl_x[i], shape, scale);
        total += 0.5 * h * s;
    }
    return total;
}

/* infT[c][t] for t < len, FP64 and its FP32 rounding; infT[c][0] = 0 */
void or_inf_table(const or_model *m, double *t64, float *t32)
{
    for (int c = 0; c < OR_N_CLASS; ++c)
        for (uint32_t t = 0; t < m->inf_len; ++t) {
            double v = (t == 0) ? 0.0
                                : or_gamma_integral((double)t - 1.0, (double)t, m->inf_shape[c], m->inf_scale[c]);
            t64[c * m->inf_len + t] = v;
            t32[c * m->inf_len + t] = (float)v;
        }
}

/* Poisson(mean) CDF thresholds: thr[k] = floor(P(K <= k) * 2^32), k = 0..cap-1.
 * P accumulated as t_0 = exp(-mean), t_k = (t_{k-1} * mean) / k, c_k = c_{k-1} + t_k. */
void or_poisson_thresholds(double mean, uint64_t *thr)
{
    double t = exp(-mean), c = t;
    thr[0] = or_threshold(c);
    for (int k = 1; k < OR_POIS_CAP; ++k) {
        t = (t * mean) / (double)k;
        c = c + t;
        thr[k] = or_threshold(c);
    }
}

static uint32_t poisson_count(uint32_t word, const uint64_t *thr)
{
    uint32_t k = 0;
    while (k < OR_POIS_CAP && (uint64_t)word >= thr[k]) ++k;
    return k;
}

/* the daily random network: in-contacts of agent j on day `step`.
 * Returns the count; contacts[] receives the source ids in draw order. */
static uint32_t random_contacts(uint64_t net_seed, uint32_t n, uint32_t j, uint32_t step,
                                const uint64_t *thr, uint32_t *contacts)
{
    uint32_t w[4];
    draw4(net_seed, j, step, SM_RNET, 0, w);
    uint32_t k = poisson_count(w[0], thr);
    for (uint32_t e = 0; e < k; ++e) {
        uint32_t idx = e + 1u; /* word 0 of block 0 is the count */
        uint32_t blk[4];
        draw4(net_seed, j, step, SM_RNET, idx / 4u, blk);
        uint32_t x = blk[idx % 4u];
        uint32_t v = (uint32_t)(((uint64_t)x * (uint64_t)(n - 1u)) >> 32);
        if (v >= j) v += 1u;
        contacts[e] = v;
    }
    return k;
}

uint32_t or_random_contacts(uint64_t net_seed, uint32_t n, uint32_t j, uint32_t step, double mean,
                            uint32_t *contacts)
{
    uint64_t thr[OR_POIS_CAP];
    or_poisson_thresholds(mean, thr);
    return random_contacts(net_seed, n, j, step, thr, contacts);
}

/* ------------------------------------------------------------------------- */
/* The global random network as a Watts-Strogatz graph (Watts and Strogatz 1998),
 * re-initialised every step (Sec. 3, Interaction Networks).  The ring lattice
 * runs over all agents in id order; agent i owns the edges to the next h = k/2
 * agents, edge m joining i and (i + m) mod n (m = 1..h).  Every step each owned
 * edge is rewired with probability beta (always when i + m wraps onto i): its far
 * end moves to an agent drawn uniformly from the other n - 1.  Edges are
 * undirected, so a rewired edge leaves the old far end and reaches the new one,
 * and both ends of every edge receive each other's messages.  Agent j's
 * neighbours, in the order their messages are summed: its own edges m = 1..h
 * (the far end, new or lattice); the lattice edges m = 1..h of agent j - m that
 * were not rewired; the rewired edges that landed on j, by owner ascending, then m. */
typedef struct {
    uint32_t h;
    uint8_t *rew;      /* [n*h] edge (i, m) rewired this step */
    uint32_t *far;     /* [n*h] far end of edge (i, m) */
    uint32_t *start;   /* [n+1] first landing edge of each agent */
    uint32_t *land;    /* owners of the landing edges, grouped by the agent they landed on */
} or_wsg;

static void wsg_build(const or_model *m, uint32_t t, or_wsg *g)
{
    const uint32_t n = m->n, h = m->rand_ws_k / 2u;
    g->h = h;
    g->rew = (uint8_t *)calloc((size_t)n * h + 1u, 1);
    g->far = (uint32_t *)calloc((size_t)n * h + 1u, sizeof(uint32_t));
    g->start = (uint32_t *)calloc((size_t)n + 1u, sizeof(uint32_t));
    for (uint32_t i = 0; i < n; ++i) {
        for (uint32_t e = 1; e <= h; ++e) {
            uint32_t w[4];
            draw4(m->net_seed, i, t, SM_WSG, (e - 1u) / 2u, w);
            const uint32_t coin = w[2u * ((e - 1u) % 2u)], word = w[2u * ((e - 1u) % 2u) + 1u];
            const size_t q = (size_t)i * h + (e - 1u);
            if (e % n == 0u || happens(coin, m->rand_ws_beta)) {
                uint32_t v = (uint32_t)(((uint64_t)word * (uint64_t)(n - 1u)) >> 32);
                if (v >= i) v += 1u;
                g->rew[q] = 1;
                g->far[q] = v;
                g->start[v + 1u]++;
            } else {
                g->far[q] = (uint32_t)(((uint64_t)i + e) % n);
            }
        }
    }
    for (uint32_t j = 0; j < n; ++j) g->start[j + 1u] += g->start[j];
    g->land = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)g->start[n] + 1u));
    uint32_t *fill = (uint32_t *)calloc((size_t)n + 1u, sizeof(uint32_t));
    for (uint32_t i = 0; i < n; ++i) /* owners ascending, then m: each group comes out sorted */
        for (uint32_t e = 1; e <= h; ++e) {
            const size_t q = (size_t)i * h + (e - 1u);
            if (g->rew[q]) {
                const uint32_t v = g->far[q];
                g->land[g->start[v] + fill[v]++] = i;
            }
        }
    free(fill);
}

static void wsg_free(or_wsg *g) { free(g->rew); free(g->far); free(g->start); free(g->land); }

/* agent j's neighbours this step, in summation order; returns their number */
static uint32_t wsg_neighbours(const or_model *m, const or_wsg *g, uint32_t j, uint32_t *out)
{
    const uint32_t n = m->n, h = g->h;
    uint32_t k = 0;
    for (uint32_t e = 1; e <= h; ++e) out[k++] = g->far[(size_t)j * h + (e - 1u)];
    for (uint32_t e = 1; e <= h; ++e) {
        const uint32_t i = (uint32_t)(((uint64_t)j + (uint64_t)n - (e % n)) % n);
        if (!g->rew[(size_t)i * h + (e - 1u)]) out[k++] = i;
    }
    for (uint32_t q = g->start[j]; q < g->start[j + 1u]; ++q) out[k++] = g->land[q];
    return k;
}

/* is one of agent j's neighbours marked in src? */
static int wsg_any(const or_model *m, const or_wsg *g, uint32_t j, const uint8_t *src)
{
    const uint32_t n = m->n, h = g->h;
    for (uint32_t e = 1; e <= h; ++e)
        if (src[g->far[(size_t)j * h + (e - 1u)]]) return 1;
    for (uint32_t e = 1; e <= h; ++e) {
        const uint32_t i = (uint32_t)(((uint64_t)j + (uint64_t)n - (e % n)) % n);
        if (!g->rew[(size_t)i * h + (e - 1u)] && src[i]) return 1;
    }
    for (uint32_t q = g->start[j]; q < g->start[j + 1u]; ++q)
        if (src[g->land[q]]) return 1;
    return 0;
}

/* the sums of inf over agent j's neighbours in summation order (FP32 left to
 * right from +0, FP64 alongside); returns their number */
static uint32_t wsg_sum(const or_model *m, const or_wsg *g, uint32_t j, const float *inf32, const double *inf64,
                        float *r32, double *r64)
{
    const uint32_t n = m->n, h = g->h;
    uint32_t k = 0;
    float s32 = 0.0f;
    double s64 = 0.0;
    for (uint32_t e = 1; e <= h; ++e) {
        const uint32_t v = g->far[(size_t)j * h + (e - 1u)];
        s32 = s32 + inf32[v];
        s64 = s64 + inf64[v];
        ++k;
    }
    for (uint32_t e = 1; e <= h; ++e) {
        const uint32_t i = (uint32_t)(((uint64_t)j + (uint64_t)n - (e % n)) % n);
        if (!g->rew[(size_t)i * h + (e - 1u)]) {
            s32 = s32 + inf32[i];
            s64 = s64 + inf64[i];
            ++k;
        }
    }
    for (uint32_t q = g->start[j]; q < g->start[j + 1u]; ++q) {
        s32 = s32 + inf32[g->land[q]];
        s64 = s64 + inf64[g->land[q]];
        ++k;
    }
    *r32 = s32;
    *r64 = s64;
    return k;
}

/* the neighbour lists of one step for the tests: start[n+1], nb[start[n]] */
int or_wsg_neighbours(const or_model *m, uint32_t t, uint32_t *start, uint32_t *nb, uint32_t cap)
{
    if (!m->rand_ws || m->rand_ws_k < 2u || m->rand_ws_k > 16u || m->rand_ws_k % 2u || m->n < 2u) return -1;
    or_wsg g;
    wsg_build(m, t, &g);
    uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)m->rand_ws_k + g.start[m->n] + 1u));
    uint32_t off = 0;
    int rc = 0;
    start[0] = 0;
    for (uint32_t j = 0; j < m->n; ++j) {
        const uint32_t k = wsg_neighbours(m, &g, j, tmp);
        if (off + k > cap) { rc = -1; break; }
        memcpy(nb + off, tmp, sizeof(uint32_t) * k);
        off += k;
        start[j + 1] = off;
    }
    free(tmp);
    wsg_free(&g);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* static vaccination schedule: priority = age bin descending, then id ascending;
 * Q = floor(rate * N) first doses a day from vax_start; day1 = start + rank / Q.
 * Agents that the campaign never reaches get 0x7FFF. */
static const uint8_t *cmp_age;
static int cmp_priority(const void *a, const void *b)
{
    uint32_t i = *(const uint32_t *)a, j = *(const uint32_t *)b;
    if (cmp_age[i] != cmp_age[j]) return cmp_age[i] > cmp_age[j] ? -1 : 1;
    return i < j ? -1 : (i > j ? 1 : 0);
}

void or_vax_days(uint32_t n, const uint8_t *age, uint32_t start, double rate, int16_t *day1)
{
    uint32_t q = (uint32_t)floor(rate * (double)n);
    uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    for (uint32_t i = 0; i < n; ++i) order[i] = i;
    cmp_age = age;
    qsort(order, n, sizeof(uint32_t), cmp_priority);
    for (uint32_t r = 0; r < n; ++r) {
        uint32_t i = order[r];
        if (q == 0) { day1[i] = 0x7FFF; continue; }
        uint64_t d = (uint64_t)start + r / q;
        day1[i] = d > 0x7FFF ? 0x7FFF : (int16_t)d;
    }
    free(order);
}

/* ------------------------------------------------------------------------- */
static int infectious_class(int st)
{
    switch (st) {
    case ST_ASYM: return 0;
    case ST_PRE_MILD: case ST_MILD: return 1;
    case ST_PRE_SEV: case ST_SEV: return 2;
    default: return -1; /* hospitalised and ICU agents are out of the community networks */
    }
}

static uint32_t duration(const or_model *m, int st, int age, uint32_t word)
{
    return uniform_int(word, m->dur_lo[st][age], m->dur_hi[st][age]);
}

/* Per-step diagnostics for the tests (any pointer may be NULL). */
typedef struct {
    float *lambda32;   /* [N] */
    double *lambda64;  /* [N] */
    float *p32;        /* [N] */
    float *u32;        /* [N] */
    float *inf32;      /* [N] infectiousness used in this step */
    uint8_t *near;     /* [N] 1 where a susceptible's |u - p| < 1e-6 */
    uint32_t *rand_k;  /* [N] random in-contact count */
    int32_t new_inf;
    int64_t messages;  /* household+occupation+random in-edges processed */
    int32_t hist[OR_N_STAGE];
    int32_t den_notified;  /* app holders notified at the end of this step */
    int64_t messages_sus;  /* the in-edges counted in `messages` whose destination was
                              susceptible at the start of the step (Eq. 2 applies to them) */
} or_diag;

/*
 * One synchronous step t: every read sees the state at the start of the step.
 * State arrays are updated in place after all reads are done.
 */
typedef struct {
    double t64[OR_N_CLASS * OR_MAX_INF_LEN];
    float t32[OR_N_CLASS * OR_MAX_INF_LEN];
    uint64_t pois[OR_POIS_CAP];
    uint64_t pois_age[OR_N_AGE][OR_POIS_CAP];  /* rand_by_age: thresholds of each age bin's mean */
} or_tables;

/* is the Poisson random network on (some agent has a positive mean, and the
 * network is not the Watts-Strogatz graph, which replaces it)? */
static int rand_poisson_on(const or_model *m)
{
    if (m->rand_ws) return 0;
    if (!m->rand_by_age) return m->rand_mean > 0.0f;
    for (int a = 0; a < OR_N_AGE; ++a)
        if (m->rand_mean_age[a] > 0.0f) return 1;
    return 0;
}

/* the Poisson thresholds of an agent of age bin a */
static const uint64_t *pois_of(const or_model *m, const or_tables *tb, int a)
{
    return m->rand_by_age ? tb->pois_age[a] : tb->pois;
}

static int check_model(const or_model *m)
{
    if (m->inf_len == 0 || m->inf_len > OR_MAX_INF_LEN || m->n_nets > OR_MAX_NETS) return -1;
    if (m->quar_days > 15 || m->test_hi > 7 || m->test_lo < 1 || m->test_lo > m->test_hi) return -1;
    if (rand_poisson_on(m) && m->n < 2) return -1;
    if (m->rand_by_age)
        for (int a = 0; a < OR_N_AGE; ++a)
            if (!(m->rand_mean_age[a] >= 0.0f)) return -1;
    if (m->rand_ws && (m->rand_ws_k < 2u || m->rand_ws_k > 16u || m->rand_ws_k % 2u || m->n < 2u ||
                       !(m->rand_ws_beta >= 0.0 && m->rand_ws_beta <= 1.0)))
        return -1;
    if (m->vax_strategy > 3 || m->elderly_bin > 9) return -1;
    if (m->den_on && (!m->test_on || m->den_window < 1 || m->den_window > 64)) return -1;
    if (m->n_occ) {
        if (m->n_nets >= OR_MAX_NETS || !m->occ_group || !m->occ_k) return -1;
        for (uint32_t g = 0; g < m->n_occ; ++g)
            if (m->occ_k[g] > OR_POIS_CAP) return -1;
        for (uint32_t j = 0; j < m->n; ++j)
            if (m->occ_group[j] >= m->n_occ) return -1;
        if (m->occ_lattice > 1 || !(m->occ_rewire >= 0.0f && m->occ_rewire <= 1.0f)) return -1;
    }
    return 0;
}

static void make_tables(const or_model *m, or_tables *tb)
{
    or_inf_table(m, tb->t64, tb->t32);
    or_poisson_thresholds((double)m->rand_mean, tb->pois);
    for (int a = 0; a < OR_N_AGE; ++a) or_poisson_thresholds((double)m->rand_mean_age[a], tb->pois_age[a]);
}

/* Daily dose selection of the priority strategies (Sec. 5, Table 1): a shared
 * supply of floor(rate * N) doses a day goes to the eligible agents with the
 * smallest (key, id); first-dose eligible = no dose yet, second-dose eligible =
 * first dose at least dose2_delay days ago; agents in hospital, ICU or dead are
 * not eligible.  Keys (age bin descending inside each group):
 *   standard:            second doses, then first doses;
 *   delayed second dose: first doses, then second doses;
 *   delayed except 65+:  agents of the elderly bins by age with a first dose
 *                        before a second dose of the same bin, then the others'
 *                        first doses, then their second doses. */
typedef struct { uint32_t key, id, type; } vcand;

static int cmp_vcand(const void *a, const void *b)
{
    const vcand *x = (const vcand *)a, *y = (const vcand *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->id < y->id ? -1 : (x->id > y->id ? 1 : 0);
}

static uint32_t vax_key(uint32_t strategy, uint32_t elderly_bin, int age, uint32_t type)
{
    const uint32_t older = (uint32_t)(8 - age);
    if (strategy == 1) return (type == 2 ? 0u : 1u) * 16u + older;
    if (strategy == 2) return (type == 1 ? 0u : 1u) * 16u + older;
    if ((uint32_t)age >= elderly_bin) return older * 2u + (type - 1u);
    return (type == 1 ? 1u : 2u) * 64u + older * 2u;
}

static void select_doses(const or_model *m, const uint8_t *age, uint32_t t, const int8_t *stage, const uint8_t *flags,
                         const int16_t *vd1, uint8_t *dose_today)
{
    const uint32_t n = m->n;
    const uint32_t q = (uint32_t)floor(m->vax_rate * (double)n);
    vcand *c = (vcand *)malloc(sizeof(vcand) * (n ? n : 1));
    uint32_t k = 0;
    for (uint32_t j = 0; j < n; ++j) {
        dose_today[j] = 0;
        const int st = stage[j];
        if (st == ST_HOSP || st == ST_ICU || st == ST_DEAD) continue;
        uint32_t type = 0;
        if (!(flags[j] & FL_DOSE1)) type = 1;
        else if (!(flags[j] & FL_DOSE2) && (int64_t)t - (int64_t)vd1[j] >= (int64_t)m->dose2_delay) type = 2;
        if (!type) continue;
        c[k].key = vax_key(m->vax_strategy, m->elderly_bin, age[j], type);
        c[k].id = j;
        c[k].type = type;
        ++k;
    }
    qsort(c, k, sizeof(vcand), cmp_vcand);
    for (uint32_t r = 0; r < k && r < q; ++r) dose_today[c[r].id] = (uint8_t)c[r].type;
    free(c);
}

/* Members of every occupation in ascending agent id: members[start[g] ..
 * start[g+1]) are the agents of occupation g, pos[j] is j's place among them. */
typedef struct {
    uint32_t *start, *members, *pos;
} or_occ;

static void occ_build(const or_model *m, or_occ *o)
{
    const uint32_t n = m->n, G = m->n_occ;
    o->start = (uint32_t *)calloc(G + 1u, sizeof(uint32_t));
    o->members = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    o->pos = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t *fill = (uint32_t *)calloc(G + 1u, sizeof(uint32_t));
    for (uint32_t j = 0; j < n; ++j) o->start[m->occ_group[j] + 1u]++;
    for (uint32_t g = 0; g < G; ++g) o->start[g + 1u] += o->start[g];
    for (uint32_t j = 0; j < n; ++j) { /* j ascending: members stay sorted */
        const uint32_t g = m->occ_group[j];
        o->pos[j] = fill[g];
        o->members[o->start[g] + fill[g]++] = j;
    }
    free(fill);
}

static void occ_free(or_occ *o) { free(o->start); free(o->members); free(o->pos); }

/* Watts-Strogatz contacts (Sec. 3, Interaction Networks; Watts and Strogatz
 * 1998), drawn anew every step: the members of an occupation sit on a ring in
 * ascending id; in-edge e of the member at place q comes from the lattice place
 * q + (e/2 + 1) for even e, q - (e/2 + 1) for odd e (mod size), unless its coin
 * falls under occ_rewire (or the lattice offset is a multiple of the size), in
 * which case it comes from a uniform other member. */
static uint32_t occ_ws_contacts(const or_model *m, const or_occ *o, uint32_t j, uint32_t step, uint32_t *contacts)
{
    const uint32_t g = m->occ_group[j];
    const uint32_t beg = o->start[g], size = o->start[g + 1u] - beg;
    if (size < 2u) return 0;
    const uint32_t k = m->occ_k[g], q = o->pos[j];
    for (uint32_t e = 0; e < k; ++e) {
        uint32_t blk[4];
        draw4(m->net_seed, j, step, SM_WS, e / 2u, blk);
        const uint32_t coin = blk[2u * (e % 2u)], word = blk[2u * (e % 2u) + 1u];
        const uint32_t hop = (e / 2u + 1u) % size;
        const uint32_t off = (e % 2u == 0u) ? hop : (size - hop) % size;
        uint32_t r;
        if (off == 0u || happens(coin, (double)m->occ_rewire)) {
            r = (uint32_t)(((uint64_t)word * (uint64_t)(size - 1u)) >> 32);
            if (r >= q) r += 1u;
        } else {
            r = (q + off) % size;
        }
        contacts[e] = o->members[beg + r];
    }
    return k;
}

/* the day's occupation in-contacts of agent j: occ_k[g] of them (none for a
 * lone member), each uniform over the other members of j's occupation, from
 * word e of the SM_OCC stream (block e/4, lane e%4); Watts-Strogatz contacts
 * when occ_lattice is set. */
static uint32_t occ_contacts(const or_model *m, const or_occ *o, uint32_t j, uint32_t step, uint32_t *contacts)
{
    if (m->occ_lattice) return occ_ws_contacts(m, o, j, step, contacts);
    const uint32_t g = m->occ_group[j];
    const uint32_t beg = o->start[g], size = o->start[g + 1u] - beg;
    if (size < 2u) return 0;
    const uint32_t k = m->occ_k[g];
    for (uint32_t e = 0; e < k; ++e) {
        uint32_t blk[4];
        draw4(m->net_seed, j, step, SM_OCC, e / 4u, blk);
        uint32_t r = (uint32_t)(((uint64_t)blk[e % 4u] * (uint64_t)(size - 1u)) >> 32);
        if (r >= o->pos[j]) r += 1u;
        contacts[e] = o->members[beg + r];
    }
    return k;
}

uint32_t or_occ_contacts(const or_model *m, uint32_t j, uint32_t step, uint32_t *contacts)
{
    if (check_model(m) || !m->n_occ || j >= m->n) return 0;
    or_occ o;
    occ_build(m, &o);
    uint32_t k = occ_contacts(m, &o, j, step, contacts);
    occ_free(&o);
    return k;
}

static int g_threads = 1;

/* Host threads for the per-agent loops (>= 1); returns the number in effect. */
int or_set_threads(int threads)
{
#ifdef _OPENMP
    g_threads = threads > 0 ? threads : 1;
#else
    (void)threads;
    g_threads = 1;
#endif
    return g_threads;
}

static int step_impl(const or_model *m, const or_tables *tb, const uint8_t *age, const int16_t *vday1,
                     uint32_t t, int8_t *stage, int16_t *timer, int16_t *tinf, uint8_t *flags, uint8_t *qt,
                     int16_t *vd1, int16_t *vd2, or_diag *dg)
{
    const uint32_t n = m->n, L = m->inf_len;
    const double *t64 = tb->t64;
    const float *t32 = tb->t32;

    float *inf32 = (float *)malloc(sizeof(float) * (n ? n : 1));
    double *inf64 = (double *)malloc(sizeof(double) * (n ? n : 1));
    uint8_t *newinf = (uint8_t *)calloc(n ? n : 1, 1);

    /* a1: per-source infectiousness from the state at the start of step t */
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (uint32_t i = 0; i < n; ++i) {
        int c = infectious_class(stage[i]);
        int ti = tinf[i];
        int quarantined = QT_QDAYS(qt[i]) > 0;
        if (c < 0 || quarantined || ti < 0 || (uint32_t)ti >= L) { inf32[i] = 0.0f; inf64[i] = 0.0; continue; }
        inf32[i] = m->A_class[c] * t32[c * L + ti];
        inf64[i] = (double)m->A_class[c] * t64[c * L + ti];
    }

    /* a2-a5: per destination sums, lambda, p, Bernoulli draw */
    const float c_R = m->R * m->inv_Ibar;
    int64_t messages = 0, messages_sus = 0;
    int32_t n_new = 0;
    or_occ occ = {NULL, NULL, NULL};
    if (m->n_occ) occ_build(m, &occ);
    or_wsg wsg = {0, NULL, NULL, NULL, NULL};
    if (m->rand_ws) wsg_build(m, t, &wsg);
#pragma omp parallel for schedule(static) num_threads(g_threads) reduction(+ : messages, messages_sus, n_new)
    for (uint32_t j = 0; j < n; ++j) {
        const int64_t messages_before = messages;
        uint32_t contacts[OR_POIS_CAP];
        float s32 = 0.0f;
        double s64 = 0.0;
        for (uint32_t net = 0; net < m->n_nets; ++net) {
            float h32 = 0.0f;
            double h64 = 0.0;
            for (uint32_t e = m->row_ptr[net][j]; e < m->row_ptr[net][j + 1]; ++e) {
                uint32_t src = m->col[net][e];
                h32 = h32 + inf32[src];
                h64 = h64 + inf64[src];
            }
            messages += m->row_ptr[net][j + 1] - m->row_ptr[net][j];
            float term = m->B_net[net] * h32;
            s32 = (net == 0) ? term : s32 + term;
            s64 += (double)m->B_net[net] * h64;
        }
        if (m->n_occ) {
            const uint32_t ko = occ_contacts(m, &occ, j, t, contacts);
            float h32 = 0.0f;
            double h64 = 0.0;
            for (uint32_t e = 0; e < ko; ++e) { h32 = h32 + inf32[contacts[e]]; h64 = h64 + inf64[contacts[e]]; }
            float term = m->B_net[m->n_nets] * h32;
            s32 = (m->n_nets == 0) ? term : s32 + term;
            s64 += (double)m->B_net[m->n_nets] * h64;
            messages += ko;
        }
        uint32_t k = 0;
        if (m->rand_ws) {
            float r32;
            double r64;
            k = wsg_sum(m, &wsg, j, inf32, inf64, &r32, &r64);
            float term = m->B_rand * r32;
            s32 = (m->n_nets == 0 && m->n_occ == 0) ? term : s32 + term;
            s64 += (double)m->B_rand * r64;
            messages += k;
        } else if (rand_poisson_on(m)) {
            k = random_contacts(m->net_seed, n, j, t, pois_of(m, tb, age[j]), contacts);
            float r32 = 0.0f;
            double r64 = 0.0;
            for (uint32_t e = 0; e < k; ++e) { r32 = r32 + inf32[contacts[e]]; r64 = r64 + inf64[contacts[e]]; }
            float term = m->B_rand * r32;
            s32 = (m->n_nets == 0 && m->n_occ == 0) ? term : s32 + term;
            s64 += (double)m->B_rand * r64;
            messages += k;
        }
        if (stage[j] == ST_S) messages_sus += messages - messages_before;
        float sus = m->S_age[age[j]];
        float lam = (c_R * sus) * s32;
        double lam64 = (double)m->R * (double)m->inv_Ibar * (double)sus * s64;
        float p = (float)(-expm1(-(double)(lam * m->dt)));
        uint32_t w[4];
        draw4(m->seed, j, t, SM_INF, 0, w);
        float u = (float)(w[0] >> 8) * (1.0f / 16777216.0f);
        if (stage[j] == ST_S && u < p) { newinf[j] = 1; ++n_new; }
        if (dg) {
            if (dg->lambda32) dg->lambda32[j] = lam;
            if (dg->lambda64) dg->lambda64[j] = lam64;
            if (dg->p32) dg->p32[j] = p;
            if (dg->u32) dg->u32[j] = u;
            if (dg->inf32) dg->inf32[j] = inf32[j];
            if (dg->rand_k) dg->rand_k[j] = k;
            if (dg->near) dg->near[j] = (stage[j] == ST_S && fabs((double)u - (double)p) < 1e-6) ? 1 : 0;
        }
    }

    /* dose selection of the priority strategies, from the state at the start of the day */
    uint8_t *dose_today = NULL;
    uint8_t *den_src = m->den_on ? (uint8_t *)calloc(n ? n : 1, 1) : NULL; /* positive app holders of the step */
    if (m->vax_on && m->vax_strategy != 0 && t >= m->vax_start) {
        dose_today = (uint8_t *)malloc(n ? n : 1);
        select_doses(m, age, t, stage, flags, vd1, dose_today);
    }

    /* a6-a7: state machine and interventions, agent by agent */
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (uint32_t j = 0; j < n; ++j) {
        int st = stage[j], a = age[j];
        int tm = timer[j], ti = tinf[j];
        uint32_t fl = flags[j];
        uint32_t qd = QT_QDAYS(qt[j]), cd = QT_TCD(qt[j]);
        int onset = 0;

        /* disease progression (Sec. 3 "Disease Progression") */
        if (newinf[j]) {
            uint32_t w[4];
            draw4(m->seed, j, t, SM_PROG, 0, w);
            if (fl & FL_IMMUNE) st = ST_ASYM;  /* vaccinated, non-sterilising: asymptomatic infection */
            else if (happens(w[0], m->p_asym[a])) st = ST_ASYM;
            else if (happens(w[2], m->p_sev[a])) st = ST_PRE_SEV;
            else st = ST_PRE_MILD;
            tm = (int)duration(m, st, a, w[1]);
            ti = 1;
        } else if (st >= ST_ASYM && st <= ST_ICU) {
            ti = ti < 32767 ? ti + 1 : 32767;
            tm = tm - 1;
            if (tm <= 0) {
                uint32_t w[4];
                draw4(m->seed, j, t, SM_PROG, 0, w);
                switch (st) {
                case ST_ASYM: st = ST_REC; break;
                case ST_PRE_MILD: st = ST_MILD; onset = 1; break;
                case ST_PRE_SEV: st = ST_SEV; onset = 1; break;
                case ST_MILD: st = ST_REC; break;
                case ST_SEV: st = happens(w[3], m->p_hosp[a]) ? ST_HOSP : ST_REC; break;
                case ST_HOSP: st = happens(w[3], m->p_icu[a]) ? ST_ICU : ST_REC; break;
                case ST_ICU: st = happens(w[3], m->p_death[a]) ? ST_DEAD : ST_REC; break;
                }
                tm = (st >= ST_ASYM && st <= ST_ICU) ? (int)duration(m, st, a, w[1]) : 0;
            }
        }

        /* quarantine already running: daily dropout, then one day served (Sec. 4.1) */
        if (qd > 0) {
            uint32_t w[4];
            draw4(m->seed, j, t, SM_INF, 0, w);
            if (happens(w[1], m->q_dropout)) qd = 0; else qd -= 1;
        }
        /* pending test result (Sec. 4.3) */
        if (cd > 0) {
            cd -= 1;
            if (cd == 0) {
                if (fl & FL_POS) {
                    if (m->quar_on) qd = m->quar_days;
                    if (den_src && (fl & FL_APP)) den_src[j] = 1; /* notifies its contacts (Sec. 4.2) */
                }
                fl &= ~FL_POS;
            }
        } else if ((onset || (fl & FL_DEN)) && m->test_on && qd == 0) {
            /* symptom onset, or yesterday's exposure notification: take a test.
             * Only an infected agent in the community can test positive. */
            uint32_t w[4];
            draw4(m->seed, j, t, SM_TEST, 0, w);
            if (st >= ST_ASYM && st <= ST_SEV && happens(w[0], m->test_sens)) fl |= FL_POS; else fl &= ~FL_POS;
            cd = uniform_int(w[1], m->test_lo, m->test_hi);
        }
        fl &= ~FL_DEN; /* a notification is acted on the next step or not at all */

        /* vaccination (Sec. 4.4 and Sec. 5) */
        if (m->vax_on && m->vax_strategy != 0) {
            if (dose_today && dose_today[j] == 1) { fl |= FL_DOSE1; vd1[j] = (int16_t)t; }
            if (dose_today && dose_today[j] == 2) { fl |= FL_DOSE2; vd2[j] = (int16_t)t; }
            if (st == ST_S && !newinf[j]) {
                uint32_t w[4];
                draw4(m->seed, j, 0, SM_VAX, 0, w);
                if (((fl & FL_DOSE1) && (int64_t)t == (int64_t)vd1[j] + m->vax_onset && happens(w[0], m->vax_eff1)) ||
                    ((fl & FL_DOSE2) && (int64_t)t == (int64_t)vd2[j] + m->vax_onset && happens(w[0], m->vax_eff2))) {
                    if (m->vax_nonsterile) fl |= FL_IMMUNE; else st = ST_VAX;
                }
            }
        } else if (m->vax_on && vday1[j] != 0x7FFF) {
            int64_t d1 = vday1[j];
            int elig = !(st == ST_HOSP || st == ST_ICU || st == ST_DEAD);
            if ((int64_t)t == d1 && elig) fl |= FL_DOSE1;
            if ((fl & FL_DOSE1) && (int64_t)t == d1 + m->dose2_delay && elig) fl |= FL_DOSE2;
            if (st == ST_S && !newinf[j]) {
                uint32_t w[4];
                draw4(m->seed, j, 0, SM_VAX, 0, w);
                if (((fl & FL_DOSE1) && (int64_t)t == d1 + m->vax_onset && happens(w[0], m->vax_eff1)) ||
                    ((fl & FL_DOSE2) && (int64_t)t == d1 + m->dose2_delay + m->vax_onset &&
                     happens(w[0], m->vax_eff2))) {
                    if (m->vax_nonsterile) fl |= FL_IMMUNE; else st = ST_VAX;
                }
            }
        }

        stage[j] = (int8_t)st;
        timer[j] = (int16_t)tm;
        tinf[j] = (int16_t)ti;
        flags[j] = (uint8_t)fl;
        qt[j] = QT_MAKE(qd, cd);
    }

    /* digital exposure notification (Sec. 4.2), after every agent's update: an app
     * holder in the community and out of quarantine is notified when one of its
     * in-contacts of the last den_window steps (this one included) had a positive
     * result this step and holds the app; it complies with probability
     * den_compliance and is then tested on the next step. */
    int32_t n_notified = 0;
    /* with the Watts-Strogatz random network, the graphs of the window's steps
     * (an agent's in-contacts there are its neighbours, the edges being undirected) */
    const uint32_t dw0 = t + 1u > m->den_window ? t + 1u - m->den_window : 0u;
    or_wsg *dwsg = NULL;
    if (den_src && m->rand_ws) {
        dwsg = (or_wsg *)calloc(t - dw0 + 1u, sizeof(or_wsg));
        for (uint32_t d = dw0; d <= t; ++d) wsg_build(m, d, &dwsg[d - dw0]);
    }
    if (den_src) {
#pragma omp parallel for schedule(static) num_threads(g_threads) reduction(+ : n_notified)
        for (uint32_t j = 0; j < n; ++j) {
            uint32_t contacts[OR_POIS_CAP];
            const int st = stage[j];
            if (!(flags[j] & FL_APP) || QT_QDAYS(qt[j]) > 0 || st == ST_HOSP || st == ST_ICU || st == ST_DEAD)
                continue;
            int hit = 0;
            for (uint32_t net = 0; net < m->n_nets && !hit; ++net)
                for (uint32_t e = m->row_ptr[net][j]; e < m->row_ptr[net][j + 1] && !hit; ++e)
                    hit = den_src[m->col[net][e]];
            const uint32_t d0 = t + 1u > m->den_window ? t + 1u - m->den_window : 0u;
            for (uint32_t d = d0; d <= t && !hit; ++d) {
                uint32_t k;
                if (m->n_occ) {
                    k = occ_contacts(m, &occ, j, d, contacts);
                    for (uint32_t e = 0; e < k && !hit; ++e) hit = den_src[contacts[e]];
                }
                if (rand_poisson_on(m)) {
                    k = random_contacts(m->net_seed, n, j, d, pois_of(m, tb, age[j]), contacts);
                    for (uint32_t e = 0; e < k && !hit; ++e) hit = den_src[contacts[e]];
                }
                if (m->rand_ws && !hit) hit = wsg_any(m, &dwsg[d - d0], j, den_src);
            }
            if (!hit) continue;
            ++n_notified;
            uint32_t w[4];
            draw4(m->seed, j, t, SM_DEN, 0, w);
            if (happens(w[0], m->den_compliance)) flags[j] |= FL_DEN;
        }
        free(den_src);
    }
    if (dwsg) {
        for (uint32_t d = dw0; d <= t; ++d) wsg_free(&dwsg[d - dw0]);
        free(dwsg);
    }

    if (dg) {
        dg->den_notified = n_notified;
        dg->new_inf = n_new;
        dg->messages = messages;
        dg->messages_sus = messages_sus;
        for (int s = 0; s < OR_N_STAGE; ++s) dg->hist[s] = 0;
        for (uint32_t j = 0; j < n; ++j) dg->hist[(int)stage[j]]++;
    }
    if (m->n_occ) occ_free(&occ);
    if (m->rand_ws) wsg_free(&wsg);
    free(inf32); free(inf64); free(newinf); free(dose_today);
    return 0;
}

int or_step(const or_model *m, const uint8_t *age, const int16_t *vday1, uint32_t t,
            int8_t *stage, int16_t *timer, int16_t *tinf, uint8_t *flags, uint8_t *qt, int16_t *vd1, int16_t *vd2,
            or_diag *dg)
{
    if (check_model(m)) return -1;
    or_tables tb;
    make_tables(m, &tb);
    return step_impl(m, &tb, age, vday1, t, stage, timer, tinf, flags, qt, vd1, vd2, dg);
}

/* infection of the initial cases before step 0: the same branch and duration
 * draws as a new infection, keyed with step word 0xFFFFFFFF */
int or_seed_infections(const or_model *m, const uint8_t *age, const uint32_t *ids, uint32_t k,
                       int8_t *stage, int16_t *timer, int16_t *tinf)
{
    for (uint32_t q = 0; q < k; ++q) {
        uint32_t j = ids[q];
        if (j >= m->n || stage[j] != ST_S) continue;
        int a = age[j], st;
        uint32_t w[4];
        draw4(m->seed, j, 0xFFFFFFFFu, SM_PROG, 0, w);
        if (happens(w[0], m->p_asym[a])) st = ST_ASYM;
        else if (happens(w[2], m->p_sev[a])) st = ST_PRE_SEV;
        else st = ST_PRE_MILD;
        stage[j] = (int8_t)st;
        timer[j] = (int16_t)duration(m, st, a, w[1]);
        tinf[j] = 1;
    }
    return 0;
}

/* T steps from t0; new_inf[T], hist[T][11], messages[T] (NULL to skip) */
int or_run(const or_model *m, const uint8_t *age, const int16_t *vday1, uint32_t t0, uint32_t T,
           int8_t *stage, int16_t *timer, int16_t *tinf, uint8_t *flags, uint8_t *qt, int16_t *vd1, int16_t *vd2,
           int32_t *new_inf, int32_t *hist, int64_t *messages, int32_t *den_notified)
{
    if (check_model(m)) return -1;
    or_tables tb;
    make_tables(m, &tb);
    or_diag dg;
    memset(&dg, 0, sizeof dg);
    for (uint32_t s = 0; s < T; ++s) {
        int rc = step_impl(m, &tb, age, vday1, t0 + s, stage, timer, tinf, flags, qt, vd1, vd2, &dg);
        if (rc) return rc;
        if (new_inf) new_inf[s] = dg.new_inf;
        if (hist) memcpy(hist + (size_t)s * OR_N_STAGE, dg.hist, sizeof dg.hist);
        if (messages) messages[s] = dg.messages;
        if (den_notified) den_notified[s] = dg.den_notified;
    }
    return 0;
}

/* exposure-notification app holders (Sec. 4.2), drawn once at initialisation:
 * agent j holds the app when word x of (seed, j, step word 0xFFFFFFFD, SM_DEN)
 * falls under den_adoption; sets or clears FL_APP in flags */
void or_den_apps(const or_model *m, uint8_t *flags)
{
    for (uint32_t j = 0; j < m->n; ++j) {
        uint32_t w[4];
        draw4(m->seed, j, 0xFFFFFFFDu, SM_DEN, 0, w);
        if (happens(w[0], m->den_adoption)) flags[j] |= FL_APP;
        else flags[j] &= (uint8_t)~FL_APP;
    }
}
