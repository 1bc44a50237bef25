/*
 * deabm_relaxed.c -- plain FP64 CPU oracle of the relaxed (differentiable) day
 * step and of its gradient.  TEST INFRASTRUCTURE ONLY (see deabm_oracle.c).
 *
 * The paper names gradient-based calibration of the simulator ("inverse ABM",
 * Abstract, Sec. 1, Sec. 6) but defines no relaxation.  The reading used here:
 *   - every agent's symptom class c_i is drawn once, before day 0, with the same
 *     thresholds as a new infection (asymptomatic, else severe, else mild);
 *   - x_j(t) in [0,1] is the infected mass of agent j on day t and s_j(t) its
 *     susceptible mass; the initial cases have x(-1) = 1, s(0) = 0;
 *   - inf_i(t) = A_{c_i} * sum_{d=1}^{L-1} infT_{c_i}[d] * x_i(t-d)     (Eq. 1 by age of infection)
 *   - lambda_j(t) = R/I * S_{a_j} * (sum_n B_n sum_{i->j} inf_i(t) + B_o sum_{occ} inf_i(t)
 *                                    + B_r sum_{rand} inf_i(t)),
 *     the occupation term present with daily occupation networks (Sec. 3,
 *     Interaction Networks: fixed membership, in-contacts drawn anew every day,
 *     as in the plain model), B_o the weight of network n_nets;
 *   - the Bernoulli(p) draw with p = 1 - exp(-lambda) (Eq. 2) is relaxed with a
 *     logistic (binary Gumbel-softmax) sample:
 *       g_j(t) = sigmoid((logit p_j(t) + l_j(t)) / tau),  logit p = log(expm1(lambda)),
 *       l = log(u) - log(1-u), u = ((w >> 8) + 0.5) 2^-24 from Philox stream 8;
 *   - x_j(t) = s_j(t) g_j(t),  s_j(t+1) = s_j(t) - x_j(t),  I(t) = sum_j x_j(t);
 *   - loss = (1/T) sum_t (log(I(t)+1) - y_t)^2.
 * Parameters theta = (R, B_0, B_1, B_r, S_0..S_8).  The random network is the
 * day's Philox network of the plain model (with age-stratified means when
 * rand_by_age is set).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define RX_MAX_NETS 4
#define RX_N_AGE 9
#define RX_MAX_L 64
#define RX_POIS_CAP 15

void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint64_t or_threshold(double p);
double or_gamma_integral(double a, double b, double shape, double scale);
void or_poisson_thresholds(double mean, uint64_t *thr);

typedef struct {
    uint32_t n, n_nets;
    const uint32_t *row_ptr[RX_MAX_NETS];
    const uint32_t *col[RX_MAX_NETS];
    double B_extra[RX_MAX_NETS];  /* weights of networks 2 and 3 (not differentiated) */
    double rand_mean, inv_Ibar, tau;
    double A_class[3];
    double inf_shape[3], inf_scale[3];
    uint32_t inf_len;
    double p_asym[RX_N_AGE], p_sev[RX_N_AGE];
    uint64_t seed, net_seed;
    /* daily occupation networks (n_occ = 0: none): occupation of each agent, daily
     * in-contacts per member, Watts-Strogatz ring lattice and its rewiring */
    uint32_t n_occ;
    const uint32_t *occ_group;
    const uint8_t *occ_k;
    uint32_t occ_lattice;
    double occ_rewire;
    /* age-stratified random interactions: agent j's daily count is
     * Poisson(rand_mean_age[age_j]) when rand_by_age is set */
    uint32_t rand_by_age;
    double rand_mean_age[RX_N_AGE];
} rx_model;

static void draw4(uint64_t seed, uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t out[4])
{
    uint32_t ctr[4] = {a, b, c, d};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox(ctr, key, out);
}

/* symptom class of each agent, fixed before day 0 (day word 0xFFFFFFFE, stream 1) */
void rx_classes(const rx_model *m, const uint8_t *age, uint8_t *cls)
{
    for (uint32_t i = 0; i < m->n; ++i) {
        uint32_t w[4];
        draw4(m->seed, i, 0xFFFFFFFEu, 1u, 0u, w);
        if ((uint64_t)w[0] < or_threshold(m->p_asym[age[i]])) cls[i] = 0;
        else if ((uint64_t)w[2] < or_threshold(m->p_sev[age[i]])) cls[i] = 2;
        else cls[i] = 1;
    }
}

static uint32_t contacts_of(const rx_model *m, const uint64_t *thr, uint32_t j, uint32_t t, uint32_t *out)
{
    uint32_t w[4];
    draw4(m->net_seed, j, t, 3u, 0u, w);
    uint32_t k = 0;
    while (k < RX_POIS_CAP && (uint64_t)w[0] >= thr[k]) ++k;
    for (uint32_t e = 0; e < k; ++e) {
        uint32_t idx = e + 1u, blk[4];
        draw4(m->net_seed, j, t, 3u, idx / 4u, blk);
        uint32_t v = (uint32_t)(((uint64_t)blk[idx % 4u] * (uint64_t)(m->n - 1u)) >> 32);
        if (v >= j) v += 1u;
        out[e] = v;
    }
    return k;
}

/* Members of every occupation in ascending agent id (start[g] .. start[g+1]) and
 * each agent's place among them. */
typedef struct {
    uint32_t *start, *members, *pos;
} rx_occ;

static void rx_occ_build(const rx_model *m, rx_occ *o)
{
    const uint32_t n = m->n, G = m->n_occ;
    o->start = (uint32_t *)calloc(G + 1u, sizeof(uint32_t));
    o->members = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    o->pos = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t *fill = (uint32_t *)calloc(G + 1u, sizeof(uint32_t));
    for (uint32_t j = 0; j < n; ++j) o->start[m->occ_group[j] + 1u]++;
    for (uint32_t g = 0; g < G; ++g) o->start[g + 1u] += o->start[g];
    for (uint32_t j = 0; j < n; ++j) {
        const uint32_t g = m->occ_group[j];
        o->pos[j] = fill[g];
        o->members[o->start[g] + fill[g]++] = j;
    }
    free(fill);
}

/* The day's occupation in-contacts of agent j on day t (as the plain model draws
 * them): occ_k[g] of them, none for a lone member.  Uniform: contact e is the
 * member at place floor(w (size-1) / 2^32) among the others, w = word e % 4 of
 * block e / 4 of stream 4.  Ring lattice: in-edge e comes from place q + (e/2+1)
 * (e even) or q - (e/2+1) (e odd) mod size, unless its coin (word 2(e%2) of block
 * e/2 of stream 9) is below the rewiring threshold or the offset is a multiple of
 * the size, when word 2(e%2)+1 picks a uniform other member. */
static uint32_t rx_occ_contacts(const rx_model *m, const rx_occ *o, uint32_t j, uint32_t t, uint32_t *out)
{
    const uint32_t g = m->occ_group[j];
    const uint32_t beg = o->start[g], size = o->start[g + 1u] - beg;
    if (size < 2u) return 0;
    const uint32_t k = m->occ_k[g], q = o->pos[j];
    for (uint32_t e = 0; e < k; ++e) {
        uint32_t blk[4], r;
        if (m->occ_lattice) {
            draw4(m->net_seed, j, t, 9u, e / 2u, blk);
            const uint32_t coin = blk[2u * (e % 2u)], word = blk[2u * (e % 2u) + 1u];
            const uint32_t hop = (e / 2u + 1u) % size;
            const uint32_t off = (e % 2u == 0u) ? hop : (size - hop) % size;
            if (off == 0u || (uint64_t)coin < or_threshold(m->occ_rewire)) {
                r = (uint32_t)(((uint64_t)word * (uint64_t)(size - 1u)) >> 32);
                if (r >= q) r += 1u;
            } else {
                r = (q + off) % size;
            }
        } else {
            draw4(m->net_seed, j, t, 4u, e / 4u, blk);
            r = (uint32_t)(((uint64_t)blk[e % 4u] * (uint64_t)(size - 1u)) >> 32);
            if (r >= q) r += 1u;
        }
        out[e] = o->members[beg + r];
    }
    return k;
}

double rx_noise(uint64_t seed, uint32_t j, uint32_t t)
{
    uint32_t w[4];
    draw4(seed, j, t, 8u, 0u, w);
    double u = ((double)(w[0] >> 8) + 0.5) / 16777216.0;
    return log(u) - log1p(-u);
}

static double logit_p(double lam)
{
    return lam > 20.0 ? lam + log1p(-exp(-lam)) : log(expm1(lam));
}

static double sigmoid(double z) { return z >= 0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z)); }

/*
 * Forward T days with full history (FP64).  theta[13]; y[T] target log(I+1) (may be
 * NULL: loss not computed).  Outputs (any may be NULL): inc[T] = I(t); loss;
 * grad[13] = d loss / d theta by the reverse sweep below.  x_out[T*n] optional.
 */
int rx_run(const rx_model *m, const uint8_t *age, const uint32_t *seeds, uint32_t n_seeds, uint32_t T,
           const double *theta, const double *y, double *inc, double *loss, double *grad, double *x_out)
{
    const uint32_t n = m->n, L = m->inf_len;
    if (L < 2 || L > RX_MAX_L || m->n_nets > RX_MAX_NETS || m->tau <= 0.0) return -1;
    if (m->n_occ) {
        if (m->n_nets >= RX_MAX_NETS || !m->occ_group || !m->occ_k || m->occ_lattice > 1) return -1;
        for (uint32_t g = 0; g < m->n_occ; ++g)
            if (m->occ_k[g] > RX_POIS_CAP) return -1;
        for (uint32_t j = 0; j < m->n; ++j)
            if (m->occ_group[j] >= m->n_occ) return -1;
    }
    const double R = theta[0], B[RX_MAX_NETS] = {theta[1], theta[2], m->B_extra[2], m->B_extra[3]};
    const double Br = theta[3];
    const double *S = theta + 4;
    const double cR = R * m->inv_Ibar;
    double infT[3][RX_MAX_L];
    for (int c = 0; c < 3; ++c)
        for (uint32_t d = 0; d < L; ++d)
            infT[c][d] = d == 0 ? 0.0 : m->A_class[c] * or_gamma_integral(d - 1.0, (double)d, m->inf_shape[c], m->inf_scale[c]);
    /* Poisson thresholds of each age bin (all the same without rand_by_age) */
    uint64_t thr_age[RX_N_AGE][RX_POIS_CAP];
    int rand_on = m->rand_by_age ? 0 : m->rand_mean > 0.0;
    for (int a = 0; a < RX_N_AGE; ++a) {
        or_poisson_thresholds(m->rand_by_age ? m->rand_mean_age[a] : m->rand_mean, thr_age[a]);
        if (m->rand_by_age && m->rand_mean_age[a] > 0.0) rand_on = 1;
    }
    uint8_t *cls = (uint8_t *)malloc(n ? n : 1);
    rx_classes(m, age, cls);

    /* history: x[(t+1)*n + j] for t = -1..T-1 */
    const size_t H = (size_t)(T + 1) * n;
    double *x = (double *)calloc(H ? H : 1, sizeof(double));
    double *s = (double *)malloc(sizeof(double) * ((size_t)(T + 1) * n + 1));
    double *g = (double *)malloc(sizeof(double) * ((size_t)T * n + 1));
    double *lam = (double *)malloc(sizeof(double) * ((size_t)T * n + 1));
    double *Hs = (double *)malloc(sizeof(double) * ((size_t)T * n * (RX_MAX_NETS + 1) + 1));
    double *Ssum = (double *)malloc(sizeof(double) * ((size_t)T * n + 1));
    double *inf = (double *)malloc(sizeof(double) * (n ? n : 1));
    double *I = (double *)calloc(T ? T : 1, sizeof(double));
    uint32_t cts[RX_POIS_CAP], octs[RX_POIS_CAP];
    rx_occ oc = {NULL, NULL, NULL};
    if (m->n_occ) rx_occ_build(m, &oc);
    for (uint32_t j = 0; j < n; ++j) s[j] = 1.0;
    for (uint32_t q = 0; q < n_seeds; ++q) {
        x[seeds[q]] = 1.0;        /* day -1 */
        s[seeds[q]] = 0.0;
    }
    for (uint32_t t = 0; t < T; ++t) {
        for (uint32_t i = 0; i < n; ++i) {
            double v = 0.0;
            for (uint32_t d = 1; d < L && d <= t + 1; ++d) v += infT[cls[i]][d] * x[(size_t)(t + 1 - d) * n + i];
            inf[i] = v;
        }
        for (uint32_t j = 0; j < n; ++j) {
            double ssum = 0.0;
            for (uint32_t net = 0; net < m->n_nets; ++net) {
                double h = 0.0;
                for (uint32_t e = m->row_ptr[net][j]; e < m->row_ptr[net][j + 1]; ++e) h += inf[m->col[net][e]];
                Hs[((size_t)t * (RX_MAX_NETS + 1) + net) * n + j] = h;
                ssum += B[net] * h;
            }
            if (m->n_occ) {  /* the occupation term, in the slot of network n_nets */
                double h = 0.0;
                const uint32_t k = rx_occ_contacts(m, &oc, j, t, octs);
                for (uint32_t e = 0; e < k; ++e) h += inf[octs[e]];
                Hs[((size_t)t * (RX_MAX_NETS + 1) + m->n_nets) * n + j] = h;
                ssum += B[m->n_nets] * h;
            }
            double r = 0.0;
            if (rand_on) {
                uint32_t k = contacts_of(m, thr_age[age[j]], j, t, cts);
                for (uint32_t e = 0; e < k; ++e) r += inf[cts[e]];
            }
            Hs[((size_t)t * (RX_MAX_NETS + 1) + RX_MAX_NETS) * n + j] = r;
            ssum += Br * r;
            const double lj = cR * S[age[j]] * ssum;
            const double gj = lj > 0.0 ? sigmoid((logit_p(lj) + rx_noise(m->seed, j, t)) / m->tau) : 0.0;
            const double sj = s[(size_t)t * n + j];
            const double xj = sj * gj;
            x[(size_t)(t + 1) * n + j] = xj;
            s[(size_t)(t + 1) * n + j] = sj - xj;
            g[(size_t)t * n + j] = gj;
            lam[(size_t)t * n + j] = lj;
            Ssum[(size_t)t * n + j] = ssum;
            I[t] += xj;
        }
    }
    if (inc) memcpy(inc, I, sizeof(double) * T);
    double Lval = 0.0;
    if (y) {
        for (uint32_t t = 0; t < T; ++t) {
            const double d = log(I[t] + 1.0) - y[t];
            Lval += d * d;
        }
        Lval /= (double)T;
        if (loss) *loss = Lval;
    }
    if (x_out) memcpy(x_out, x + n, sizeof(double) * (size_t)T * n);

    if (grad && y) {
        /* reverse sweep; ibar[t*n + i] = d loss / d inf_i(t) */
        double *ibar = (double *)calloc((size_t)T * n + 1, sizeof(double));
        double *sbar = (double *)calloc(n ? n : 1, sizeof(double)); /* d loss / d s(t+1) */
        double gR = 0.0, gB[RX_MAX_NETS] = {0}, gBr = 0.0, gS[RX_N_AGE] = {0};
        for (int t = (int)T - 1; t >= 0; --t) {
            const double Ibar = 2.0 / T * (log(I[t] + 1.0) - y[t]) / (I[t] + 1.0);
            for (uint32_t j = 0; j < n; ++j) {
                double xbar = Ibar - sbar[j];
                for (uint32_t d = 1; d < L && (uint32_t)t + d < T; ++d) xbar += infT[cls[j]][d] * ibar[(size_t)(t + d) * n + j];
                const size_t q = (size_t)t * n + j;
                const double gj = g[q], lj = lam[q], sj = s[q];
                const double gbar = xbar * sj;
                double lbar = 0.0;
                if (lj > 0.0) lbar = gbar * gj * (1.0 - gj) / (m->tau * (-expm1(-lj)));
                sbar[j] = xbar * gj + sbar[j];
                const double coef = lbar * cR * S[age[j]];
                gR += lbar * m->inv_Ibar * S[age[j]] * Ssum[q];
                gS[age[j]] += lbar * cR * Ssum[q];
                for (uint32_t net = 0; net < m->n_nets; ++net) {
                    gB[net] += coef * Hs[((size_t)t * (RX_MAX_NETS + 1) + net) * n + j];
                    for (uint32_t e = m->row_ptr[net][j]; e < m->row_ptr[net][j + 1]; ++e)
                        ibar[(size_t)t * n + m->col[net][e]] += B[net] * coef;
                }
                if (m->n_occ) {
                    gB[m->n_nets] += coef * Hs[((size_t)t * (RX_MAX_NETS + 1) + m->n_nets) * n + j];
                    const uint32_t k = rx_occ_contacts(m, &oc, j, (uint32_t)t, octs);
                    for (uint32_t e = 0; e < k; ++e) ibar[(size_t)t * n + octs[e]] += B[m->n_nets] * coef;
                }
                if (rand_on) {
                    gBr += coef * Hs[((size_t)t * (RX_MAX_NETS + 1) + RX_MAX_NETS) * n + j];
                    uint32_t k = contacts_of(m, thr_age[age[j]], j, (uint32_t)t, cts);
                    for (uint32_t e = 0; e < k; ++e) ibar[(size_t)t * n + cts[e]] += Br * coef;
                }
            }
        }
        grad[0] = gR;
        grad[1] = gB[0];
        grad[2] = gB[1];
        grad[3] = gBr;
        for (int a = 0; a < RX_N_AGE; ++a) grad[4 + a] = gS[a];
        free(ibar);
        free(sbar);
    }
    free(cls); free(x); free(s); free(g); free(lam); free(Hs); free(Ssum); free(inf); free(I);
    free(oc.start); free(oc.members); free(oc.pos);
    return 0;
}
