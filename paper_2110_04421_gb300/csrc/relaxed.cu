// relaxed.cu -- the relaxed (differentiable) day step, its reverse sweep and
// on-device Adam calibration (include/deabm.h: deabm_relaxed_*, deabm_grad,
// deabm_calibrate).
//
// The paper names gradient-based calibration of the simulator ("inverse ABM",
// Abstract, Sec. 1, Sec. 6) without defining a relaxation.  The model run here:
//   x_j(t) = s_j(t) * g_j(t),  s_j(t+1) = s_j(t) - x_j(t),  I(t) = sum_j x_j(t)
//   g_j(t) = sigmoid((log expm1(lambda_j(t)) + l_j(t)) / tau)   (binary Gumbel-softmax
//            relaxation of the Eq. 2 draw; l = logistic noise from Philox stream 8)
//   lambda_j(t) = R/I * S_{a_j} * (sum_n B_n sum_{i->j} inf_i(t) + B_o sum_occ inf_i(t)
//                                  + B_r sum_rand inf_i(t))   (Eq. 1; the occupation term with
//                 daily occupation networks, B_o the weight of network n_nets)
//   inf_i(t) = sum_{d=1}^{L-1} A_{c_i} infT_{c_i}[d] * x_i(t-d)
//   loss = (1/T) sum_t (log(I(t)+1) - y_t)^2
// The reverse sweep carries d loss / d x back through the susceptible mass and,
// along the transpose of every network, to the infectiousness of the sources;
// the days are recomputed segment by segment from checkpoints (Philox noise,
// random and occupation contacts are regenerated, never stored).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "deabm.h"
#include "deabm_device.cuh"
#include "kernels.h"

namespace deabm {

constexpr uint32_t kRxBlock = 256;
constexpr int kTheta = DEABM_N_THETA;

struct RxParams {
    uint32_t n, n_nets, L, rand_on, T, nblk;
    uint32_t rand_by_age;  // 1: agent j's random-contact count from tab->pois_age[age_j]
    uint32_t nh;  // per-day H slots: the stored networks, the occupation term (n_occ > 0), the random network
    // daily occupation networks (n_occ = 0: none), by agent id: occupation, place
    // among its members; members of occupation g in ascending id at
    // occ_members[occ_start[g] ..]; daily in-contacts per member; lattice rewiring
    uint32_t n_occ, occ_lattice;
    uint64_t thr_rewire;
    const uint32_t *occ_gid, *occ_pos, *occ_start, *occ_members;
    const uint8_t *occ_k;
    float tau, inv_Ibar;
    float B_extra[DEABM_MAX_NETS];
    uint64_t seed, net_seed;
    const uint32_t *row_ptr[DEABM_MAX_NETS], *col[DEABM_MAX_NETS];
    const uint32_t *tr_ptr[DEABM_MAX_NETS], *tr_col[DEABM_MAX_NETS];
    const Tables *tab;
    const uint8_t *age, *cls;
    const float *theta;  // R, B_0, B_1, B_r, S_0..S_8 (device)
};

__device__ __forceinline__ float rx_weight(const RxParams &P, uint32_t net)
{
    return net < 2 ? P.theta[1 + net] : P.B_extra[net];
}

// The day's occupation in-contacts of agent j on day t, drawn as in the plain
// model (uniform over the other members from stream 4, or the Watts-Strogatz
// lattice with rewiring from stream 9); f(agent id) for each, in draw order.
template <class F>
__device__ __forceinline__ void rx_occ_for(const RxParams &P, uint32_t j, uint32_t t, F f)
{
    const uint32_t g = __ldg(P.occ_gid + j);
    const uint32_t beg = __ldg(P.occ_start + g), size = __ldg(P.occ_start + g + 1u) - beg;
    if (size < 2u) return;
    const uint32_t k = __ldg(P.occ_k + g), q = __ldg(P.occ_pos + j);
    const uint2 nk = seed_key(P.net_seed);
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    for (uint32_t e = 0; e < k; ++e) {
        uint32_t r;
        if (P.occ_lattice) {
            if ((e & 1u) == 0u) w = draw(nk, j, t, kStreamWs, e >> 1);
            const uint32_t coin = (e & 1u) ? w.z : w.x, word = (e & 1u) ? w.w : w.y;
            const uint32_t m = (e >> 1) + 1u, hop = m < size ? m : m % size;
            const uint32_t off = (e & 1u) == 0u ? hop : (hop == 0u ? 0u : size - hop);
            if (off == 0u || (uint64_t)coin < P.thr_rewire) {
                r = (uint32_t)(((uint64_t)word * (uint64_t)(size - 1u)) >> 32);
                r += (r >= q) ? 1u : 0u;
            } else {
                r = q + off;
                r = r >= size ? r - size : r;
            }
        } else {
            if ((e & 3u) == 0u) w = draw(nk, j, t, kStreamOcc, e >> 2);
            const uint32_t x = (e & 3u) == 0u ? w.x : (e & 3u) == 1u ? w.y : (e & 3u) == 2u ? w.z : w.w;
            r = (uint32_t)(((uint64_t)x * (uint64_t)(size - 1u)) >> 32);
            r += (r >= q) ? 1u : 0u;
        }
        f(__ldg(P.occ_members + beg + r));
    }
}

// the Poisson thresholds of agent j's daily random-contact count
__device__ __forceinline__ const uint64_t *rx_pois(const RxParams &P, uint32_t j)
{
    return P.rand_by_age ? P.tab->pois_age[P.age[j]] : P.tab->pois;
}

__device__ __forceinline__ float sigmoidf_(float z)
{
    if (z >= 0.0f) return 1.0f / (1.0f + expf(-z));
    const float e = expf(z);
    return e / (1.0f + e);
}

__device__ __forceinline__ float logit_p(float lam)
{
    return lam > 20.0f ? lam + log1pf(-expf(-lam)) : logf(expm1f(lam));
}

__device__ __forceinline__ float logistic_noise(uint64_t seed, uint32_t j, uint32_t t)
{
    const uint32_t w = draw(seed_key(seed), j, t, kStreamGumbel).x;
    const float u = ((float)(w >> 8) + 0.5f) * (1.0f / 16777216.0f);
    return logf(u) - log1pf(-u);
}

// slot of day `day` (>= -L) in a ring of L days; day -1 -> slot 0.  Days before -1
// map to slots not yet written this run, which hold zeros.
__device__ __forceinline__ uint32_t ring_slot(int day, uint32_t L)
{
    const int m = (day + 1) % (int)L;
    return (uint32_t)(m < 0 ? m + (int)L : m);
}

// symptom class fixed before day 0: asymptomatic (0), else severe (2), else mild (1)
__global__ void rx_class_kernel(const RxParams P, uint8_t *cls)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    const uint4 w = draw(seed_key(P.seed), i, 0xFFFFFFFEu, kStreamProg);
    const int a = P.age[i];
    cls[i] = (uint64_t)w.x < __ldg(&P.tab->thr_asym[a]) ? 0 : ((uint64_t)w.z < __ldg(&P.tab->thr_sev[a]) ? 2 : 1);
}

// inf_i(t) from the ring of the last L days of x: the sum over d = 1 .. L-1 of
// A_c infT_c[d] x_i(t-d), d ascending
__device__ __forceinline__ float rx_inf_of(const RxParams &P, int t, const float *__restrict__ xring, uint32_t i)
{
    const int c = P.cls[i];
    float v = 0.0f;
    for (uint32_t d = 1; d < P.L; ++d)
        v += __ldg(&P.tab->infT[c][d]) * xring[(size_t)ring_slot(t - (int)d, P.L) * P.n + i];
    return v;
}

// inf(t) of every agent (the first day of a run or of a recomputed segment; the
// day kernel computes each later day's for its own agent)
__global__ void rx_inf_kernel(const RxParams P, int t, const float *__restrict__ xring, float *__restrict__ inf)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;
    inf[i] = rx_inf_of(P, t, xring, i);
}

struct RxSeg {  // per-day records of one checkpoint segment (k = t - t0)
    float *x, *g, *s, *lam, *H;  // H: [K][nh][N]
};

// Day t: reads inf(t), writes x(t) into the ring and then the agent's own
// inf(t+1) into inf_next (the ring then holds every x it needs), so no separate
// launch computes the next day's infectiousness.
template <bool REC>
__global__ void __launch_bounds__(kRxBlock) rx_day_kernel(const RxParams P, int t, int k, const float *__restrict__ inf,
                                                          float *__restrict__ s, float *__restrict__ xring, RxSeg seg,
                                                          float *__restrict__ Ipart, float *__restrict__ inf_next)
{
    __shared__ float warp_sum[kRxBlock / 32];
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    float x = 0.0f;
    if (j < P.n) {
        const float R = P.theta[0];
        float ssum = 0.0f;
        for (uint32_t net = 0; net < P.n_nets; ++net) {
            float h = 0.0f;
            for (uint32_t e = __ldg(P.row_ptr[net] + j); e < __ldg(P.row_ptr[net] + j + 1); ++e)
                h = __fadd_rn(h, __ldg(inf + __ldg(P.col[net] + e)));
            ssum = __fadd_rn(ssum, __fmul_rn(rx_weight(P, net), h));
            if (REC) seg.H[((size_t)k * P.nh + net) * P.n + j] = h;
        }
        if (P.n_occ) {
            float h = 0.0f;
            rx_occ_for(P, j, (uint32_t)t, [&](uint32_t v) { h = __fadd_rn(h, __ldg(inf + v)); });
            ssum = __fadd_rn(ssum, __fmul_rn(rx_weight(P, P.n_nets), h));
            if (REC) seg.H[((size_t)k * P.nh + P.n_nets) * P.n + j] = h;
        }
        float r = 0.0f;
        if (P.rand_on) {
            const uint2 nk = seed_key(P.net_seed);
            uint4 w = draw(nk, j, (uint32_t)t, kStreamRnet, 0u);
            const uint64_t *thr = rx_pois(P, j);
            uint32_t kk = 0;
            while (kk < DEABM_POIS_CAP && (uint64_t)w.x >= __ldg(thr + kk)) ++kk;
            for (uint32_t e = 0; e < kk; ++e) {
                const uint32_t idx = e + 1u;
                if ((idx & 3u) == 0u) w = draw(nk, j, (uint32_t)t, kStreamRnet, idx >> 2);
                const uint32_t xw = (idx & 3u) == 1u ? w.y : (idx & 3u) == 2u ? w.z : (idx & 3u) == 3u ? w.w : w.x;
                uint32_t v = (uint32_t)(((uint64_t)xw * (uint64_t)(P.n - 1u)) >> 32);
                v += (v >= j) ? 1u : 0u;
                r = __fadd_rn(r, __ldg(inf + v));
            }
            ssum = __fadd_rn(ssum, __fmul_rn(P.theta[3], r));
        }
        if (REC) seg.H[((size_t)k * P.nh + P.nh - 1u) * P.n + j] = r;
        const float lam = R * P.inv_Ibar * P.theta[4 + P.age[j]] * ssum;
        const float g = lam > 0.0f ? sigmoidf_((logit_p(lam) + logistic_noise(P.seed, j, (uint32_t)t)) / P.tau) : 0.0f;
        const float sj = s[j];
        x = sj * g;
        s[j] = sj - x;
        xring[(size_t)ring_slot(t, P.L) * P.n + j] = x;
        inf_next[j] = rx_inf_of(P, t + 1, xring, j);  // this thread's own ring entries only
        if (REC) {
            seg.x[(size_t)k * P.n + j] = x;
            seg.g[(size_t)k * P.n + j] = g;
            seg.s[(size_t)k * P.n + j] = sj;
            seg.lam[(size_t)k * P.n + j] = lam;
        }
    }
    // block partial of I(t) in a fixed order (deterministic)
    float v = x;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, off);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.0f;
        for (uint32_t w = 0; w < kRxBlock / 32; ++w) b += warp_sum[w];
        Ipart[(size_t)t * P.nblk + blockIdx.x] = b;
    }
}

// I(t), the loss and d loss / d I(t); one block
__global__ void rx_loss_kernel(const RxParams P, uint32_t T, const float *Ipart, const float *y, float *I, float *Ibar,
                               float *loss, float *loss_trace)
{
    __shared__ double part[256];
    double acc = 0.0;
    for (uint32_t t = threadIdx.x; t < T; t += blockDim.x) {
        double s = 0.0;
        for (uint32_t b = 0; b < P.nblk; ++b) s += Ipart[(size_t)t * P.nblk + b];
        I[t] = (float)s;
        if (y) {
            const double d = log(s + 1.0) - (double)y[t];
            acc += d * d;
            Ibar[t] = (float)(2.0 / T * d / (s + 1.0));
        }
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0 && y) {
        double L = 0.0;
        for (uint32_t q = 0; q < blockDim.x; ++q) L += part[q];
        *loss = (float)(L / T);
        if (loss_trace) *loss_trace = (float)(L / T);
    }
}

// reverse of day t: d loss / d x, d loss / d lambda, the susceptible-mass adjoint,
// each agent's coefficient for the transpose scatter and the parameter partials
// One launch per reverse day t.  First this agent's d loss / d inf(t+1) is
// completed with the stored networks' part: a gather along the transpose CSR of
// the coefficients of day t+1 (coef_next, all written by the previous launch),
// added to what the generated networks scattered into that slot; then the
// adjoint of day t reads the agent's own slots t+1 .. t+L-1, clears slot t-1
// (slot t+L-1, just read) for the next launch's scatters, and writes coef(t).
__global__ void __launch_bounds__(kRxBlock) rx_adj_kernel(const RxParams P, int t, int k, const float *__restrict__ Ibar,
                                                          float *__restrict__ ibring, float *__restrict__ sbar,
                                                          float *__restrict__ coef, const float *__restrict__ coef_next,
                                                          RxSeg seg, double *gpart)
{
    __shared__ float red[kTheta][kRxBlock / 32];
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    float contrib[kTheta];
#pragma unroll
    for (int q = 0; q < kTheta; ++q) contrib[q] = 0.0f;
    if (j < P.n) {
        const int c = P.cls[j], a = P.age[j];
        if ((uint32_t)t + 1u < P.T) {
            float v = 0.0f;
            for (uint32_t net = 0; net < P.n_nets; ++net) {
                float h = 0.0f;
                for (uint32_t e = __ldg(P.tr_ptr[net] + j); e < __ldg(P.tr_ptr[net] + j + 1); ++e)
                    h += __ldg(coef_next + __ldg(P.tr_col[net] + e));
                v += rx_weight(P, net) * h;
            }
            ibring[(size_t)(((uint32_t)t + 1u) % P.L) * P.n + j] += v;
        }
        float xbar = Ibar[t] - sbar[j];
        for (uint32_t d = 1; d < P.L && (uint32_t)t + d < P.T; ++d)
            xbar += __ldg(&P.tab->infT[c][d]) * ibring[(size_t)(((uint32_t)t + d) % P.L) * P.n + j];
        ibring[(size_t)(((uint32_t)t + P.L - 1u) % P.L) * P.n + j] = 0.0f;
        const size_t q = (size_t)k * P.n + j;
        const float g = seg.g[q], lam = seg.lam[q], sj = seg.s[q];
        const float gbar = xbar * sj;
        // d g / d lambda = g (1 - g) / (tau (1 - e^-lambda)); it is 0 wherever g is 0
        // (also when lambda is so small that 1 - e^-lambda underflows in FP32)
        const float lbar = (lam > 0.0f && g > 0.0f) ? gbar * g * (1.0f - g) / (P.tau * (-expm1f(-lam))) : 0.0f;
        sbar[j] = xbar * g + sbar[j];
        const float R = P.theta[0], Sa = P.theta[4 + a], cR = R * P.inv_Ibar;
        const float cf = lbar * cR * Sa;
        coef[j] = cf;
        // d loss / d inf_i(t) along the day's generated networks: this destination
        // regenerates its random and occupation contacts and adds to theirs
        // (atomics; the slot was cleared by the launch of day t+1, and the stored
        // networks' gathers are added to it by the launch of day t-1)
        if (cf != 0.0f) {
            float *dst = ibring + (size_t)((uint32_t)t % P.L) * P.n;
            if (P.rand_on) {
                const float cfr = cf * P.theta[3];
                const uint2 nk = seed_key(P.net_seed);
                uint4 w = draw(nk, j, (uint32_t)t, kStreamRnet, 0u);
                const uint64_t *thr = rx_pois(P, j);
                uint32_t kk = 0;
                while (kk < DEABM_POIS_CAP && (uint64_t)w.x >= __ldg(thr + kk)) ++kk;
                for (uint32_t e = 0; e < kk; ++e) {
                    const uint32_t idx = e + 1u;
                    if ((idx & 3u) == 0u) w = draw(nk, j, (uint32_t)t, kStreamRnet, idx >> 2);
                    const uint32_t xw = (idx & 3u) == 1u ? w.y : (idx & 3u) == 2u ? w.z : (idx & 3u) == 3u ? w.w : w.x;
                    uint32_t v = (uint32_t)(((uint64_t)xw * (uint64_t)(P.n - 1u)) >> 32);
                    v += (v >= j) ? 1u : 0u;
                    atomicAdd(dst + v, cfr);
                }
            }
            if (P.n_occ) {
                const float cfo = cf * rx_weight(P, P.n_nets);
                rx_occ_for(P, j, (uint32_t)t, [&](uint32_t v) { atomicAdd(dst + v, cfo); });
            }
        }
        float ssum = 0.0f;
        const uint32_t nw = P.nh - 1u;  // weighted network slots (stored, occupation); the random one last
        for (uint32_t net = 0; net < P.nh; ++net) {
            const float h = seg.H[((size_t)k * P.nh + net) * P.n + j];
            const float w = net < nw ? rx_weight(P, net) : P.theta[3];
            ssum += w * h;
            if (net < 2 && net < nw) contrib[1 + net] = cf * h;
            if (net == nw && P.rand_on) contrib[3] = cf * h;
        }
        contrib[0] = lbar * P.inv_Ibar * Sa * ssum;
#pragma unroll
        for (int q2 = 0; q2 < DEABM_N_AGE; ++q2) contrib[4 + q2] = (q2 == a) ? lbar * cR * ssum : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < kTheta; ++q) {
        float v = contrib[q];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, off);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < kTheta) {
        double b = 0.0;
        for (uint32_t w = 0; w < kRxBlock / 32; ++w) b += red[threadIdx.x][w];
        gpart[(size_t)blockIdx.x * kTheta + threadIdx.x] += b;
    }
}

__global__ void rx_grad_reduce_kernel(const RxParams P, const double *gpart, float *grad)
{
    const int q = threadIdx.x;
    if (q >= kTheta) return;
    double s = 0.0;
    for (uint32_t b = 0; b < P.nblk; ++b) s += gpart[(size_t)b * kTheta + q];
    grad[q] = (float)s;
}

// projected Adam on theta (parameters stay >= 0)
__global__ void adam_kernel(float *theta, float *m, float *v, const float *grad, float lr, float b1, float b2, float eps,
                            int step)
{
    const int q = threadIdx.x;
    if (q >= kTheta) return;
    const float g = grad[q];
    m[q] = b1 * m[q] + (1.0f - b1) * g;
    v[q] = b2 * v[q] + (1.0f - b2) * g * g;
    const float mh = m[q] / (1.0f - powf(b1, (float)step)), vh = v[q] / (1.0f - powf(b2, (float)step));
    theta[q] = fmaxf(theta[q] - lr * mh / (sqrtf(vh) + eps), 0.0f);
}

__global__ void rx_init_kernel(const RxParams P, const uint32_t *seeds, uint32_t n_seeds, float *s, float *xring)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P.n) s[i] = 1.0f;
    for (size_t q = i; q < (size_t)P.L * P.n; q += (size_t)gridDim.x * blockDim.x) xring[q] = 0.0f;
}

__global__ void rx_seed_kernel(const RxParams P, const uint32_t *seeds, uint32_t n_seeds, float *s, float *xring)
{
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_seeds) return;
    s[seeds[q]] = 0.0f;
    xring[seeds[q]] = 1.0f;  // slot 0 = day -1
}


// ------------------------------------------------------------------ B parameter columns
// The same relaxed model for B parameter vectors theta_b at once (deabm_grad_batch):
// every per-agent array becomes [agent][column] with the column fastest.  A block
// is 8 agents x 32 columns, a warp one agent's 32 columns, so each CSR entry is
// one broadcast load for 32 columns and each gather a contiguous 128-byte run:
// the edge lists are read once a day for all columns.  The columns share the
// graph, the initial cases and the noise (common random numbers); only theta
// differs.  Every per-column sum runs in the single-column order, so a column
// equals a single run up to FMA contraction and the scatter atomics' order.
struct RxbArrays {
    uint32_t B, nbx;        // columns; blocks along the agents (8 agents each)
    const float *theta;     // [B][13]
    float *s, *xring, *inf, *Ipart, *ibring, *sbar, *coef;
    float *x, *g, *sr, *lam, *H;  // segment records [K][N][B]; H [K][nh][N][B]
    double *gpart;          // [nbx][B][13]
};

__device__ __forceinline__ float rxb_weight(const RxParams &P, const float *th, uint32_t net)
{
    return net < 2 ? th[1 + net] : P.B_extra[net];
}

__global__ void rxb_init_kernel(const RxParams P, RxbArrays A, const uint32_t *seeds, uint32_t n_seeds)
{
    const size_t nb = (size_t)P.n * A.B, stride = (size_t)gridDim.x * blockDim.x;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < (size_t)P.L * nb; q += stride) {
        if (q < nb) A.s[q] = 1.0f;
        A.xring[q] = 0.0f;
    }
}

__global__ void rxb_seed_kernel(const RxParams P, RxbArrays A, const uint32_t *seeds, uint32_t n_seeds)
{
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)n_seeds * A.B) return;
    const size_t i = (size_t)seeds[q / A.B] * A.B + q % A.B;
    A.s[i] = 0.0f;
    A.xring[i] = 1.0f;  // slot 0 = day -1
}

__global__ void rxb_inf_kernel(const RxParams P, RxbArrays A, int t)
{
    const uint32_t i = blockIdx.x * 8u + threadIdx.y, b = blockIdx.y * 32u + threadIdx.x;
    if (i >= P.n || b >= A.B) return;
    const int c = P.cls[i];
    float v = 0.0f;
    for (uint32_t d = 1; d < P.L; ++d)
        v += __ldg(&P.tab->infT[c][d]) * A.xring[((size_t)ring_slot(t - (int)d, P.L) * P.n + i) * A.B + b];
    A.inf[(size_t)i * A.B + b] = v;
}

template <bool REC>
__global__ void __launch_bounds__(256) rxb_day_kernel(const RxParams P, RxbArrays A, int t, int k)
{
    __shared__ float sI[8][32];
    const uint32_t lane = threadIdx.x, ay = threadIdx.y;
    const uint32_t j = blockIdx.x * 8u + ay, b = blockIdx.y * 32u + lane;
    const uint32_t B = A.B;
    float x = 0.0f;
    if (j < P.n && b < B) {
        const float *th = A.theta + (size_t)b * kTheta;
        const float *inf = A.inf;
        const size_t nn = P.nh;
        float ssum = 0.0f;
        for (uint32_t net = 0; net < P.n_nets; ++net) {
            float h = 0.0f;
            for (uint32_t e = __ldg(P.row_ptr[net] + j); e < __ldg(P.row_ptr[net] + j + 1); ++e)
                h = __fadd_rn(h, __ldg(inf + (size_t)__ldg(P.col[net] + e) * B + b));
            ssum = __fadd_rn(ssum, __fmul_rn(rxb_weight(P, th, net), h));
            if (REC) A.H[(((size_t)k * nn + net) * P.n + j) * B + b] = h;
        }
        if (P.n_occ) {
            float h = 0.0f;
            rx_occ_for(P, j, (uint32_t)t, [&](uint32_t v) { h = __fadd_rn(h, __ldg(inf + (size_t)v * B + b)); });
            ssum = __fadd_rn(ssum, __fmul_rn(rxb_weight(P, th, P.n_nets), h));
            if (REC) A.H[(((size_t)k * nn + P.n_nets) * P.n + j) * B + b] = h;
        }
        float r = 0.0f;
        if (P.rand_on) {
            const uint2 nk = seed_key(P.net_seed);
            uint4 w = draw(nk, j, (uint32_t)t, kStreamRnet, 0u);
            const uint64_t *thr = rx_pois(P, j);
            uint32_t kk = 0;
            while (kk < DEABM_POIS_CAP && (uint64_t)w.x >= __ldg(thr + kk)) ++kk;
            for (uint32_t e = 0; e < kk; ++e) {
                const uint32_t idx = e + 1u;
                if ((idx & 3u) == 0u) w = draw(nk, j, (uint32_t)t, kStreamRnet, idx >> 2);
                const uint32_t xw = (idx & 3u) == 1u ? w.y : (idx & 3u) == 2u ? w.z : (idx & 3u) == 3u ? w.w : w.x;
                uint32_t v = (uint32_t)(((uint64_t)xw * (uint64_t)(P.n - 1u)) >> 32);
                v += (v >= j) ? 1u : 0u;
                r = __fadd_rn(r, __ldg(inf + (size_t)v * B + b));
            }
            ssum = __fadd_rn(ssum, __fmul_rn(th[3], r));
        }
        if (REC) A.H[(((size_t)k * nn + nn - 1u) * P.n + j) * B + b] = r;
        const float lam = th[0] * P.inv_Ibar * th[4 + P.age[j]] * ssum;
        const float g = lam > 0.0f ? sigmoidf_((logit_p(lam) + logistic_noise(P.seed, j, (uint32_t)t)) / P.tau) : 0.0f;
        const size_t q = (size_t)j * B + b;
        const float sj = A.s[q];
        x = sj * g;
        A.s[q] = sj - x;
        A.xring[(size_t)ring_slot(t, P.L) * P.n * B + q] = x;
        if (REC) {
            const size_t qk = (size_t)k * P.n * B + q;
            A.x[qk] = x;
            A.g[qk] = g;
            A.sr[qk] = sj;
            A.lam[qk] = lam;
        }
    }
    // block partial of I(t) per column over the block's 8 agents, in a fixed order
    sI[ay][lane] = x;
    __syncthreads();
    if (ay == 0 && b < B) {
        float v = 0.0f;
        for (uint32_t q = 0; q < 8u; ++q) v += sI[q][lane];
        A.Ipart[((size_t)t * A.nbx + blockIdx.x) * B + b] = v;
    }
}

// I(t), the loss and d loss / d I(t) of column blockIdx.x (256 threads, fixed tree)
__global__ void rxb_loss_kernel(const RxParams P, RxbArrays A, uint32_t T, const float *y, float *I, float *Ibar,
                                float *loss)
{
    __shared__ double red[256];
    const uint32_t b = blockIdx.x, B = A.B;
    double acc = 0.0;
    for (uint32_t t = 0; t < T; ++t) {
        double s = 0.0;
        for (uint32_t q = threadIdx.x; q < A.nbx; q += blockDim.x) s += A.Ipart[((size_t)t * A.nbx + q) * B + b];
        red[threadIdx.x] = s;
        __syncthreads();
        for (uint32_t w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double tot = red[0];
            I[(size_t)t * B + b] = (float)tot;
            if (y) {
                const double d = log(tot + 1.0) - (double)y[(size_t)t * B + b];
                acc += d * d;
                Ibar[(size_t)t * B + b] = (float)(2.0 / T * d / (tot + 1.0));
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && y) loss[b] = (float)(acc / T);
}

__global__ void __launch_bounds__(256) rxb_adj_kernel(const RxParams P, RxbArrays A, int t, int k, const float *Ibar)
{
    __shared__ float red[kTheta][8][32];
    const uint32_t lane = threadIdx.x, ay = threadIdx.y;
    const uint32_t j = blockIdx.x * 8u + ay, b = blockIdx.y * 32u + lane;
    const uint32_t B = A.B;
    float contrib[kTheta];
#pragma unroll
    for (int q = 0; q < kTheta; ++q) contrib[q] = 0.0f;
    if (j < P.n && b < B) {
        const float *th = A.theta + (size_t)b * kTheta;
        const int c = P.cls[j], a = P.age[j];
        const size_t qj = (size_t)j * B + b;
        float xbar = Ibar[(size_t)t * B + b] - A.sbar[qj];
        for (uint32_t d = 1; d < P.L && (uint32_t)t + d < P.T; ++d)
            xbar += __ldg(&P.tab->infT[c][d]) * A.ibring[((size_t)(((uint32_t)t + d) % P.L) * P.n) * B + qj];
        const size_t q = (size_t)k * P.n * B + qj;
        const float g = A.g[q], lam = A.lam[q], sj = A.sr[q];
        const float gbar = xbar * sj;
        const float lbar = (lam > 0.0f && g > 0.0f) ? gbar * g * (1.0f - g) / (P.tau * (-expm1f(-lam))) : 0.0f;
        A.sbar[qj] = xbar * g + A.sbar[qj];
        const float R = th[0], Sa = th[4 + a], cR = R * P.inv_Ibar;
        const float cf = lbar * cR * Sa;
        A.coef[qj] = cf;
        float ssum = 0.0f;
        const size_t nn = P.nh;
        const uint32_t nw = P.nh - 1u;  // weighted network slots (stored, occupation); the random one last
        for (uint32_t net = 0; net < P.nh; ++net) {
            const float h = A.H[(((size_t)k * nn + net) * P.n + j) * B + b];
            const float w = net < nw ? rxb_weight(P, th, net) : th[3];
            ssum += w * h;
            if (net < 2 && net < nw) contrib[1 + net] = cf * h;
            if (net == nw && P.rand_on) contrib[3] = cf * h;
        }
        contrib[0] = lbar * P.inv_Ibar * Sa * ssum;
#pragma unroll
        for (int q2 = 0; q2 < DEABM_N_AGE; ++q2) contrib[4 + q2] = (q2 == a) ? lbar * cR * ssum : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < kTheta; ++q) red[q][ay][lane] = contrib[q];
    __syncthreads();
    if (ay == 0 && b < B) {
        double *gp = A.gpart + ((size_t)blockIdx.x * B + b) * kTheta;
        for (int q = 0; q < kTheta; ++q) {
            double v = 0.0;
            for (uint32_t a2 = 0; a2 < 8u; ++a2) v += red[q][a2][lane];
            gp[q] += v;
        }
    }
}

__global__ void rxb_scatter_static_kernel(const RxParams P, RxbArrays A, int t)
{
    const uint32_t i = blockIdx.x * 8u + threadIdx.y, b = blockIdx.y * 32u + threadIdx.x;
    if (i >= P.n || b >= A.B) return;
    const float *th = A.theta + (size_t)b * kTheta;
    float v = 0.0f;
    for (uint32_t net = 0; net < P.n_nets; ++net) {
        float h = 0.0f;
        for (uint32_t e = __ldg(P.tr_ptr[net] + i); e < __ldg(P.tr_ptr[net] + i + 1); ++e)
            h += __ldg(A.coef + (size_t)__ldg(P.tr_col[net] + e) * A.B + b);
        v += rxb_weight(P, th, net) * h;
    }
    A.ibring[((size_t)((uint32_t)t % P.L) * P.n + i) * A.B + b] = v;
}

__global__ void rxb_scatter_random_kernel(const RxParams P, RxbArrays A, int t)
{
    const uint32_t j = blockIdx.x * 8u + threadIdx.y, b = blockIdx.y * 32u + threadIdx.x;
    if (j >= P.n || b >= A.B) return;
    const float cf = A.coef[(size_t)j * A.B + b] * A.theta[(size_t)b * kTheta + 3];
    if (cf == 0.0f) return;
    const uint2 nk = seed_key(P.net_seed);
    uint4 w = draw(nk, j, (uint32_t)t, kStreamRnet, 0u);
    const uint64_t *thr = rx_pois(P, j);
    uint32_t kk = 0;
    while (kk < DEABM_POIS_CAP && (uint64_t)w.x >= __ldg(thr + kk)) ++kk;
    float *dst = A.ibring + (size_t)((uint32_t)t % P.L) * P.n * A.B;
    for (uint32_t e = 0; e < kk; ++e) {
        const uint32_t idx = e + 1u;
        if ((idx & 3u) == 0u) w = draw(nk, j, (uint32_t)t, kStreamRnet, idx >> 2);
        const uint32_t xw = (idx & 3u) == 1u ? w.y : (idx & 3u) == 2u ? w.z : (idx & 3u) == 3u ? w.w : w.x;
        uint32_t v = (uint32_t)(((uint64_t)xw * (uint64_t)(P.n - 1u)) >> 32);
        v += (v >= j) ? 1u : 0u;
        atomicAdd(dst + (size_t)v * A.B + b, cf);
    }
}

__global__ void rxb_scatter_occ_kernel(const RxParams P, RxbArrays A, int t)
{
    const uint32_t j = blockIdx.x * 8u + threadIdx.y, b = blockIdx.y * 32u + threadIdx.x;
    if (j >= P.n || b >= A.B) return;
    const float cf = A.coef[(size_t)j * A.B + b] * rxb_weight(P, A.theta + (size_t)b * kTheta, P.n_nets);
    if (cf == 0.0f) return;
    float *dst = A.ibring + (size_t)((uint32_t)t % P.L) * P.n * A.B;
    rx_occ_for(P, j, (uint32_t)t, [&](uint32_t v) { atomicAdd(dst + (size_t)v * A.B + b, cf); });
}

__global__ void rxb_grad_reduce_kernel(const RxbArrays A, float *grad)
{
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;  // (column, parameter)
    if (q >= A.B * (uint32_t)kTheta) return;
    const uint32_t b = q / kTheta, p = q % kTheta;
    double s = 0.0;
    for (uint32_t blk = 0; blk < A.nbx; ++blk) s += A.gpart[((size_t)blk * A.B + b) * kTheta + p];
    grad[q] = (float)s;
}

}  // namespace deabm

using namespace deabm;

// ------------------------------------------------------------------------------------ host side
struct deabm_relaxed {
    cudaStream_t stream = nullptr;
    uint32_t n = 0, L = 0, max_days = 0, K = 10, nseg = 0, n_nets = 0, n_seeds = 0;
    std::vector<void *> allocs;
    RxParams P{};
    float *theta = nullptr, *adam_m = nullptr, *adam_v = nullptr, *grad = nullptr;
    float *s = nullptr, *xring = nullptr, *inf = nullptr, *ckpt = nullptr;
    RxSeg seg{};
    float *Ipart = nullptr, *I = nullptr, *y = nullptr, *Ibar = nullptr, *loss = nullptr, *loss_trace = nullptr;
    float *ibring = nullptr, *sbar = nullptr, *coef = nullptr;
    // B parameter columns (deabm_grad_batch): arrays for bat_cap columns, allocated
    // on the first call that needs them
    uint32_t bat_cap = 0;
    std::vector<void *> bat_allocs;
    RxbArrays bat{};
    float *b_ckpt = nullptr, *b_I = nullptr, *b_y = nullptr, *b_Ibar = nullptr, *b_loss = nullptr, *b_grad = nullptr;
    float *b_theta = nullptr;
    double *gpart = nullptr;
    uint32_t *seeds = nullptr;
    uint32_t trace_cap = 0;
    // one gradient (forward with checkpoints, reverse sweep) as a CUDA graph,
    // captured for a horizon T and replayed while T stays the same
    cudaGraphExec_t grad_graph = nullptr;
    uint32_t graph_T = 0;
    cudaStream_t cap_stream = nullptr;  // capture happens here (the caller's stream may be the legacy one)
};

static thread_local std::string g_rx_err;

static int rx_fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_rx_err = buf;
    return code;
}

#define RCU(call)                                                                                                  \
    do {                                                                                                           \
        cudaError_t e_ = (call);                                                                                   \
        if (e_ != cudaSuccess)                                                                                     \
            return rx_fail(e_ == cudaErrorMemoryAllocation ? DEABM_ENOMEM : DEABM_ECUDA, "%s: %s (%s:%d)", #call, \
                           cudaGetErrorString(e_), __FILE__, __LINE__);                                            \
    } while (0)

template <class T>
static int rx_alloc(deabm_relaxed *c, T **out, size_t count)
{
    void *p = nullptr;
    const size_t bytes = count ? count * sizeof(T) : sizeof(T);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return rx_fail(DEABM_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
    }
    c->allocs.push_back(p);
    *out = (T *)p;
    return DEABM_OK;
}

static uint64_t rx_threshold(double p)
{
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return (uint64_t)1 << 32;
    return (uint64_t)std::floor(p * 4294967296.0);
}

extern "C" void deabm_relaxed_destroy(deabm_relaxed *c)
{
    if (!c) return;
    if (!c->allocs.empty()) (void)cudaStreamSynchronize(c->stream);
    if (c->grad_graph) (void)cudaGraphExecDestroy(c->grad_graph);
    if (c->cap_stream) (void)cudaStreamDestroy(c->cap_stream);
    for (void *p : c->allocs) (void)cudaFree(p);
    for (void *p : c->bat_allocs) (void)cudaFree(p);
    delete c;
}

extern "C" int deabm_relaxed_create(const deabm_graph *g, const deabm_agents *a, const deabm_params *p, float tau,
                                    uint32_t max_days, uint32_t ckpt_every, void *stream, deabm_relaxed **out)
{
    if (!out) return rx_fail(DEABM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!g || !a || !p || !a->age_bin) return rx_fail(DEABM_EINVAL, "graph, agents (age_bin) and params are required");
    const uint32_t n = g->n_agents;
    if (n == 0 || n >= (1u << 31) || g->n_nets > DEABM_MAX_NETS) return rx_fail(DEABM_EINVAL, "bad graph size");
    if (!(tau > 0.0f)) return rx_fail(DEABM_EINVAL, "tau must be > 0");
    if (g->n_occ) {
        if (g->n_nets >= DEABM_MAX_NETS) return rx_fail(DEABM_EINVAL, "daily occupations need n_nets < %d", DEABM_MAX_NETS);
        if (!g->occ_group || !g->occ_k) return rx_fail(DEABM_EINVAL, "occ_group and occ_k are required");
        if (g->occ_lattice > 1 || !(g->occ_rewire >= 0.0f && g->occ_rewire <= 1.0f))
            return rx_fail(DEABM_EINVAL, "occ_lattice must be 0 or 1 and occ_rewire in [0,1]");
        for (uint32_t q = 0; q < g->n_occ; ++q)
            if (g->occ_k[q] > DEABM_POIS_CAP) return rx_fail(DEABM_EINVAL, "occ_k must be <= %d", DEABM_POIS_CAP);
        for (uint32_t j = 0; j < n; ++j)
            if (g->occ_group[j] >= g->n_occ) return rx_fail(DEABM_EINVAL, "occ_group out of range");
    }
    if (p->den_on) return rx_fail(DEABM_EINVAL, "exposure notification is not available in the relaxed model");
    if (max_days == 0 || ckpt_every == 0) return rx_fail(DEABM_EINVAL, "max_days and ckpt_every must be >= 1");
    if (p->inf_len < 2 || p->inf_len > DEABM_MAX_INF_LEN) return rx_fail(DEABM_EINVAL, "inf_len must be 2..64");
    if (g->rand_ws) return rx_fail(DEABM_EINVAL, "the relaxed model uses the Poisson random network (rand_ws must be 0)");
    if (g->rand_by_age > 1) return rx_fail(DEABM_EINVAL, "rand_by_age must be 0 or 1");
    if (g->rand_by_age)
        for (int q = 0; q < DEABM_N_AGE; ++q)
            if (!(g->rand_mean_age[q] >= 0.0f) || g->rand_mean_age[q] > 1e3f)
                return rx_fail(DEABM_EINVAL, "rand_mean_age[%d] out of range", q);
    if ((g->rand_mean > 0.0f || g->rand_by_age) && n < 2) return rx_fail(DEABM_EINVAL, "the random network needs >= 2 agents");
    for (uint32_t k = 0; k < g->n_nets; ++k) {
        const uint32_t *rp = g->row_ptr[k];
        if (!rp || rp[0] != 0 || (rp[n] && !g->col[k])) return rx_fail(DEABM_EINVAL, "bad CSR %u", k);
        for (uint32_t j = 0; j < n; ++j) {
            if (rp[j + 1] < rp[j]) return rx_fail(DEABM_EINVAL, "row_ptr[%u] decreases at %u", k, j);
            for (uint32_t e = rp[j]; e < rp[j + 1]; ++e)
                if (g->col[k][e] >= n || g->col[k][e] == j) return rx_fail(DEABM_EINVAL, "bad column in network %u", k);
        }
    }
    for (uint32_t j = 0; j < n; ++j)
        if (a->age_bin[j] >= DEABM_N_AGE) return rx_fail(DEABM_EINVAL, "age_bin out of range");
    for (uint32_t q = 0; q < a->n_seed; ++q)
        if (!a->seed_ids || a->seed_ids[q] >= n) return rx_fail(DEABM_EINVAL, "bad seed id");

    deabm_relaxed *c = new (std::nothrow) deabm_relaxed();
    if (!c) return rx_fail(DEABM_ENOMEM, "host allocation failed");
    int rc = [&]() -> int {
        c->stream = (cudaStream_t)stream;
        cudaStream_t s = c->stream;
        c->n = n;
        c->L = p->inf_len;
        c->max_days = max_days;
        c->K = ckpt_every;
        c->nseg = (max_days + ckpt_every - 1) / ckpt_every;
        c->n_nets = g->n_nets;
        const uint32_t nblk = (n + kRxBlock - 1) / kRxBlock;
        RxParams &P = c->P;
        P.n = n;
        P.n_nets = g->n_nets;
        P.L = p->inf_len;
        P.rand_by_age = g->rand_by_age ? 1u : 0u;
        P.rand_on = g->rand_mean > 0.0f;
        if (g->rand_by_age) {
            P.rand_on = 0;
            for (int q = 0; q < DEABM_N_AGE; ++q) P.rand_on |= g->rand_mean_age[q] > 0.0f ? 1u : 0u;
        }
        P.nblk = nblk;
        P.tau = tau;
        P.inv_Ibar = p->inv_Ibar;
        for (int k = 0; k < DEABM_MAX_NETS; ++k) P.B_extra[k] = p->B_net[k];
        P.seed = p->seed;
        P.net_seed = p->net_seed;
        P.n_occ = g->n_occ;
        P.nh = g->n_nets + (g->n_occ ? 1u : 0u) + 1u;
        int r;
        if (g->n_occ) {  // members of each occupation in ascending id, each agent's place
            const uint32_t G = g->n_occ;
            std::vector<uint32_t> start((size_t)G + 1, 0), members(n), pos(n), fill;
            for (uint32_t j = 0; j < n; ++j) start[g->occ_group[j] + 1]++;
            for (uint32_t q = 0; q < G; ++q) start[q + 1] += start[q];
            fill.assign(start.begin(), start.end() - 1);
            for (uint32_t j = 0; j < n; ++j) {
                const uint32_t q = g->occ_group[j];
                pos[j] = fill[q] - start[q];
                members[fill[q]++] = j;
            }
            uint32_t *d_gid, *d_pos, *d_start, *d_mem;
            uint8_t *d_k;
            if ((r = rx_alloc(c, &d_gid, n))) return r;
            if ((r = rx_alloc(c, &d_pos, n))) return r;
            if ((r = rx_alloc(c, &d_start, (size_t)G + 1))) return r;
            if ((r = rx_alloc(c, &d_mem, n))) return r;
            if ((r = rx_alloc(c, &d_k, G))) return r;
            RCU(cudaMemcpyAsync(d_gid, g->occ_group, 4ull * n, cudaMemcpyHostToDevice, s));
            RCU(cudaMemcpyAsync(d_pos, pos.data(), 4ull * n, cudaMemcpyHostToDevice, s));
            RCU(cudaMemcpyAsync(d_start, start.data(), 4ull * (G + 1), cudaMemcpyHostToDevice, s));
            RCU(cudaMemcpyAsync(d_mem, members.data(), 4ull * n, cudaMemcpyHostToDevice, s));
            RCU(cudaMemcpyAsync(d_k, g->occ_k, G, cudaMemcpyHostToDevice, s));
            RCU(cudaStreamSynchronize(s));  // the staging vectors go out of scope
            P.occ_gid = d_gid;
            P.occ_pos = d_pos;
            P.occ_start = d_start;
            P.occ_members = d_mem;
            P.occ_k = d_k;
            P.occ_lattice = g->occ_lattice;
            P.thr_rewire = rx_threshold((double)g->occ_rewire);
        }
        std::vector<uint32_t> tptr, tcol, fill;
        for (uint32_t k = 0; k < g->n_nets; ++k) {
            const uint32_t E = g->row_ptr[k][n];
            uint32_t *rp, *cl, *trp, *tcl;
            if ((r = rx_alloc(c, &rp, (size_t)n + 1))) return r;
            if ((r = rx_alloc(c, &cl, E))) return r;
            if ((r = rx_alloc(c, &trp, (size_t)n + 1))) return r;
            if ((r = rx_alloc(c, &tcl, E))) return r;
            // transpose (out-edges of each source, destinations ascending) by counting sort
            tptr.assign((size_t)n + 1, 0);
            for (uint32_t e = 0; e < E; ++e) tptr[g->col[k][e] + 1]++;
            for (uint32_t i = 0; i < n; ++i) tptr[i + 1] += tptr[i];
            fill.assign(tptr.begin(), tptr.end() - 1);
            tcol.resize(E);
            for (uint32_t j = 0; j < n; ++j)
                for (uint32_t e = g->row_ptr[k][j]; e < g->row_ptr[k][j + 1]; ++e) tcol[fill[g->col[k][e]]++] = j;
            RCU(cudaMemcpyAsync(rp, g->row_ptr[k], 4ull * (n + 1), cudaMemcpyHostToDevice, s));
            if (E) RCU(cudaMemcpyAsync(cl, g->col[k], 4ull * E, cudaMemcpyHostToDevice, s));
            RCU(cudaMemcpyAsync(trp, tptr.data(), 4ull * (n + 1), cudaMemcpyHostToDevice, s));
            if (E) RCU(cudaMemcpyAsync(tcl, tcol.data(), 4ull * E, cudaMemcpyHostToDevice, s));
            RCU(cudaStreamSynchronize(s));
            P.row_ptr[k] = rp;
            P.col[k] = cl;
            P.tr_ptr[k] = trp;
            P.tr_col[k] = tcl;
        }
        uint8_t *age, *cls;
        if ((r = rx_alloc(c, &age, n))) return r;
        if ((r = rx_alloc(c, &cls, n))) return r;
        RCU(cudaMemcpyAsync(age, a->age_bin, n, cudaMemcpyHostToDevice, s));
        P.age = age;
        P.cls = cls;
        Tables T;
        std::memset(&T, 0, sizeof T);
        for (int a = -1; a < DEABM_N_AGE; ++a) {  // the single mean (a = -1), then each age bin's
            const double m = a < 0 || !g->rand_by_age ? (double)g->rand_mean : (double)g->rand_mean_age[a];
            uint64_t *thr = a < 0 ? T.pois : T.pois_age[a];
            volatile double t = std::exp(-m), cdf = t;
            thr[0] = rx_threshold(cdf);
            for (int k = 1; k < DEABM_POIS_CAP; ++k) {
                t = (t * m) / (double)k;
                cdf = cdf + t;
                thr[k] = rx_threshold(cdf);
            }
        }
        for (int q = 0; q < DEABM_N_AGE; ++q) {
            T.thr_asym[q] = rx_threshold(p->p_asym[q]);
            T.thr_sev[q] = rx_threshold(p->p_sev[q]);
        }
        Tables *tab;
        if ((r = rx_alloc(c, &tab, 1))) return r;
        RCU(cudaMemcpyAsync(tab, &T, sizeof T, cudaMemcpyHostToDevice, s));
        double *d_gamma;
        float *d_A;
        if ((r = rx_alloc(c, &d_gamma, 6))) return r;
        if ((r = rx_alloc(c, &d_A, 3))) return r;
        const double gs[6] = {p->inf_shape[0], p->inf_shape[1], p->inf_shape[2],
                              p->inf_scale[0], p->inf_scale[1], p->inf_scale[2]};
        RCU(cudaMemcpyAsync(d_gamma, gs, sizeof gs, cudaMemcpyHostToDevice, s));
        RCU(cudaMemcpyAsync(d_A, p->A_class, sizeof(float) * 3, cudaMemcpyHostToDevice, s));
        RCU(launch_inf_table(tab, d_gamma, d_A, p->inf_len, s));
        P.tab = tab;
        if ((r = rx_alloc(c, &c->theta, kTheta))) return r;
        if ((r = rx_alloc(c, &c->adam_m, kTheta))) return r;
        if ((r = rx_alloc(c, &c->adam_v, kTheta))) return r;
        if ((r = rx_alloc(c, &c->grad, kTheta))) return r;
        P.theta = c->theta;
        rx_class_kernel<<<(n + 255) / 256, 256, 0, s>>>(P, cls);
        RCU(cudaGetLastError());
        const size_t L = c->L, K = c->K, NN = P.nh;
        if ((r = rx_alloc(c, &c->s, n))) return r;
        if ((r = rx_alloc(c, &c->xring, L * n))) return r;
        if ((r = rx_alloc(c, &c->inf, 2 * (size_t)n))) return r;  // inf(t), inf(t+1)
        if ((r = rx_alloc(c, &c->ckpt, (size_t)c->nseg * (L + 1) * n))) return r;
        if ((r = rx_alloc(c, &c->seg.x, K * n))) return r;
        if ((r = rx_alloc(c, &c->seg.g, K * n))) return r;
        if ((r = rx_alloc(c, &c->seg.s, K * n))) return r;
        if ((r = rx_alloc(c, &c->seg.lam, K * n))) return r;
        if ((r = rx_alloc(c, &c->seg.H, K * NN * n))) return r;
        if ((r = rx_alloc(c, &c->Ipart, (size_t)max_days * nblk))) return r;
        if ((r = rx_alloc(c, &c->I, max_days))) return r;
        if ((r = rx_alloc(c, &c->y, max_days))) return r;
        if ((r = rx_alloc(c, &c->Ibar, max_days))) return r;
        if ((r = rx_alloc(c, &c->loss, 1))) return r;
        if ((r = rx_alloc(c, &c->ibring, L * n))) return r;
        if ((r = rx_alloc(c, &c->sbar, n))) return r;
        if ((r = rx_alloc(c, &c->coef, 2 * (size_t)n))) return r;  // coef(t) and coef(t+1)
        if ((r = rx_alloc(c, &c->gpart, (size_t)nblk * kTheta))) return r;
        c->n_seeds = a->n_seed;
        if ((r = rx_alloc(c, &c->seeds, a->n_seed))) return r;
        if (a->n_seed) RCU(cudaMemcpyAsync(c->seeds, a->seed_ids, 4ull * a->n_seed, cudaMemcpyHostToDevice, s));
        RCU(cudaStreamSynchronize(s));
        return DEABM_OK;
    }();
    if (rc != DEABM_OK) {
        deabm_relaxed_destroy(c);
        return rc;
    }
    *out = c;
    return DEABM_OK;
}

// forward days [0, T): checkpoints every K days; records nothing else
static int rx_forward_device(deabm_relaxed *c, uint32_t T, const float *y_dev, float *loss_trace_slot)
{
    cudaStream_t s = c->stream;
    RxParams P = c->P;
    P.T = T;
    const uint32_t n = c->n, L = c->L, nb = (n + kRxBlock - 1) / kRxBlock;
    rx_init_kernel<<<nb, kRxBlock, 0, s>>>(P, c->seeds, c->n_seeds, c->s, c->xring);
    if (c->n_seeds) rx_seed_kernel<<<(c->n_seeds + 255) / 256, 256, 0, s>>>(P, c->seeds, c->n_seeds, c->s, c->xring);
    RCU(cudaGetLastError());
    if (T) rx_inf_kernel<<<nb, kRxBlock, 0, s>>>(P, 0, c->xring, c->inf);
    for (uint32_t t = 0; t < T; ++t) {
        if (t % c->K == 0) {
            float *ck = c->ckpt + (size_t)(t / c->K) * (L + 1) * n;
            RCU(cudaMemcpyAsync(ck, c->s, 4ull * n, cudaMemcpyDeviceToDevice, s));
            RCU(cudaMemcpyAsync(ck + n, c->xring, 4ull * L * n, cudaMemcpyDeviceToDevice, s));
        }
        rx_day_kernel<false><<<nb, kRxBlock, 0, s>>>(P, (int)t, 0, c->inf + (size_t)(t & 1u) * n, c->s, c->xring,
                                                    c->seg, c->Ipart, c->inf + (size_t)((t + 1u) & 1u) * n);
    }
    rx_loss_kernel<<<1, 256, 0, s>>>(P, T, c->Ipart, y_dev, c->I, c->Ibar, c->loss, loss_trace_slot);
    RCU(cudaGetLastError());
    return DEABM_OK;
}

static int rx_backward_device(deabm_relaxed *c, uint32_t T)
{
    cudaStream_t s = c->stream;
    RxParams P = c->P;
    P.T = T;
    const uint32_t n = c->n, L = c->L, nb = (n + kRxBlock - 1) / kRxBlock;
    RCU(cudaMemsetAsync(c->sbar, 0, 4ull * n, s));
    RCU(cudaMemsetAsync(c->ibring, 0, 4ull * L * n, s));
    RCU(cudaMemsetAsync(c->gpart, 0, sizeof(double) * nb * kTheta, s));
    const uint32_t nseg = (T + c->K - 1) / c->K;
    for (int sg = (int)nseg - 1; sg >= 0; --sg) {
        const uint32_t t0 = (uint32_t)sg * c->K, t1 = t0 + c->K < T ? t0 + c->K : T;
        const float *ck = c->ckpt + (size_t)sg * (L + 1) * n;
        RCU(cudaMemcpyAsync(c->s, ck, 4ull * n, cudaMemcpyDeviceToDevice, s));
        RCU(cudaMemcpyAsync(c->xring, ck + n, 4ull * L * n, cudaMemcpyDeviceToDevice, s));
        rx_inf_kernel<<<nb, kRxBlock, 0, s>>>(P, (int)t0, c->xring, c->inf + (size_t)(t0 & 1u) * n);
        for (uint32_t t = t0; t < t1; ++t)  // recompute the segment, recording it
            rx_day_kernel<true><<<nb, kRxBlock, 0, s>>>(P, (int)t, (int)(t - t0), c->inf + (size_t)(t & 1u) * n, c->s,
                                                       c->xring, c->seg, c->Ipart, c->inf + (size_t)((t + 1u) & 1u) * n);
        // one launch per reverse day (the stored networks' part of day t+1, the
        // adjoint of day t with the generated networks' scatters)
        for (int t = (int)t1 - 1; t >= (int)t0; --t)
            rx_adj_kernel<<<nb, kRxBlock, 0, s>>>(P, t, t - (int)t0, c->Ibar, c->ibring, c->sbar,
                                                  c->coef + (size_t)(t & 1) * n, c->coef + (size_t)((t + 1) & 1) * n,
                                                  c->seg, c->gpart);
    }
    rx_grad_reduce_kernel<<<1, 32, 0, s>>>(P, c->gpart, c->grad);
    RCU(cudaGetLastError());
    return DEABM_OK;
}

// forward (loss into c->loss) and reverse sweep of horizon T, replayed from a
// CUDA graph on the caller's stream: the day loop launches about 6 kernels a
// day, which the graph issues without a host round trip per launch.  The graph
// is recorded on a private stream, since the legacy default stream cannot be
// captured.
static int rx_gradient(deabm_relaxed *c, uint32_t T)
{
    if (!(c->grad_graph && c->graph_T == T)) {
        if (c->grad_graph) {
            RCU(cudaGraphExecDestroy(c->grad_graph));
            c->grad_graph = nullptr;
        }
        if (!c->cap_stream) RCU(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t g;
        const cudaStream_t user = c->stream;
        RCU(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        c->stream = c->cap_stream;  // the launchers below record into the graph
        int r = rx_forward_device(c, T, c->y, nullptr);
        if (!r) r = rx_backward_device(c, T);
        c->stream = user;
        const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
        if (r) {
            if (e == cudaSuccess) (void)cudaGraphDestroy(g);
            return r;
        }
        RCU(e);
        const cudaError_t ei = cudaGraphInstantiate(&c->grad_graph, g, 0);
        (void)cudaGraphDestroy(g);
        RCU(ei);
        c->graph_T = T;
    }
    RCU(cudaGraphLaunch(c->grad_graph, c->stream));
    return DEABM_OK;
}

static int rx_check(deabm_relaxed *c, uint32_t T)
{
    if (!c) return rx_fail(DEABM_EINVAL, "ctx is NULL");
    if (T == 0 || T > c->max_days) return rx_fail(DEABM_EINVAL, "T must be in 1..max_days (%u)", c->max_days);
    return DEABM_OK;
}

extern "C" int deabm_relaxed_forward(deabm_relaxed *c, uint32_t T, const float *theta, float *incidence)
{
    int r;
    if ((r = rx_check(c, T))) return r;
    if (!theta) return rx_fail(DEABM_EINVAL, "theta is NULL");
    RCU(cudaMemcpyAsync(c->theta, theta, 4 * kTheta, cudaMemcpyHostToDevice, c->stream));
    if ((r = rx_forward_device(c, T, nullptr, nullptr))) return r;
    if (incidence) RCU(cudaMemcpyAsync(incidence, c->I, 4ull * T, cudaMemcpyDeviceToHost, c->stream));
    RCU(cudaStreamSynchronize(c->stream));
    return DEABM_OK;
}

extern "C" int deabm_grad(deabm_relaxed *c, uint32_t T, const float *theta, const float *target, float *loss,
                          float *grad, float *incidence)
{
    int r;
    if ((r = rx_check(c, T))) return r;
    if (!theta || !target) return rx_fail(DEABM_EINVAL, "theta and target are required");
    RCU(cudaMemcpyAsync(c->theta, theta, 4 * kTheta, cudaMemcpyHostToDevice, c->stream));
    RCU(cudaMemcpyAsync(c->y, target, 4ull * T, cudaMemcpyHostToDevice, c->stream));
    if ((r = rx_gradient(c, T))) return r;
    if (loss) RCU(cudaMemcpyAsync(loss, c->loss, 4, cudaMemcpyDeviceToHost, c->stream));
    if (grad) RCU(cudaMemcpyAsync(grad, c->grad, 4 * kTheta, cudaMemcpyDeviceToHost, c->stream));
    if (incidence) RCU(cudaMemcpyAsync(incidence, c->I, 4ull * T, cudaMemcpyDeviceToHost, c->stream));
    RCU(cudaStreamSynchronize(c->stream));
    return DEABM_OK;
}

extern "C" int deabm_calibrate(deabm_relaxed *c, uint32_t T, const float *theta0, const float *target, uint32_t steps,
                               float lr, float *theta_out, float *loss_trace)
{
    int r;
    if ((r = rx_check(c, T))) return r;
    if (!theta0 || !target || !(lr > 0.0f)) return rx_fail(DEABM_EINVAL, "theta0, target and lr > 0 are required");
    if (steps > c->trace_cap) {
        float *tr;
        if ((r = rx_alloc(c, &tr, steps))) return r;
        c->loss_trace = tr;
        c->trace_cap = steps;
    }
    RCU(cudaMemcpyAsync(c->theta, theta0, 4 * kTheta, cudaMemcpyHostToDevice, c->stream));
    RCU(cudaMemcpyAsync(c->y, target, 4ull * T, cudaMemcpyHostToDevice, c->stream));
    RCU(cudaMemsetAsync(c->adam_m, 0, 4 * kTheta, c->stream));
    RCU(cudaMemsetAsync(c->adam_v, 0, 4 * kTheta, c->stream));
    for (uint32_t it = 0; it < steps; ++it) {
        if ((r = rx_gradient(c, T))) return r;
        RCU(cudaMemcpyAsync(c->loss_trace + it, c->loss, 4, cudaMemcpyDeviceToDevice, c->stream));
        adam_kernel<<<1, 32, 0, c->stream>>>(c->theta, c->adam_m, c->adam_v, c->grad, lr, 0.9f, 0.999f, 1e-8f, (int)it + 1);
        RCU(cudaGetLastError());
    }
    if (theta_out) RCU(cudaMemcpyAsync(theta_out, c->theta, 4 * kTheta, cudaMemcpyDeviceToHost, c->stream));
    if (loss_trace && steps) RCU(cudaMemcpyAsync(loss_trace, c->loss_trace, 4ull * steps, cudaMemcpyDeviceToHost, c->stream));
    RCU(cudaStreamSynchronize(c->stream));
    return DEABM_OK;
}

extern "C" const char *deabm_relaxed_last_error(void) { return g_rx_err.c_str(); }

// ------------------------------------------------------------------ B parameter columns
template <class T>
static int rxb_alloc(deabm_relaxed *c, T **out, size_t count)
{
    void *p = nullptr;
    const size_t bytes = count ? count * sizeof(T) : sizeof(T);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return rx_fail(DEABM_ENOMEM, "cudaMalloc of %zu bytes for %u columns failed", bytes, c->bat_cap);
    }
    c->bat_allocs.push_back(p);
    *out = (T *)p;
    return DEABM_OK;
}

// arrays for B columns (kept, grown when a call needs more)
static int rxb_reserve(deabm_relaxed *c, uint32_t B)
{
    if (B <= c->bat_cap) return DEABM_OK;
    RCU(cudaStreamSynchronize(c->stream));
    for (void *p : c->bat_allocs) (void)cudaFree(p);
    c->bat_allocs.clear();
    c->bat_cap = B;
    const size_t n = c->n, L = c->L, K = c->K, NN = c->P.nh, nb = n * B;
    const uint32_t nbx = (uint32_t)((n + 7) / 8);
    RxbArrays &A = c->bat;
    A.nbx = nbx;
    int r;
    if ((r = rxb_alloc(c, &c->b_theta, (size_t)B * kTheta))) return r;
    if ((r = rxb_alloc(c, &A.s, nb))) return r;
    if ((r = rxb_alloc(c, &A.xring, L * nb))) return r;
    if ((r = rxb_alloc(c, &A.inf, nb))) return r;
    if ((r = rxb_alloc(c, &c->b_ckpt, (size_t)c->nseg * (L + 1) * nb))) return r;
    if ((r = rxb_alloc(c, &A.x, K * nb))) return r;
    if ((r = rxb_alloc(c, &A.g, K * nb))) return r;
    if ((r = rxb_alloc(c, &A.sr, K * nb))) return r;
    if ((r = rxb_alloc(c, &A.lam, K * nb))) return r;
    if ((r = rxb_alloc(c, &A.H, K * NN * nb))) return r;
    if ((r = rxb_alloc(c, &A.Ipart, (size_t)c->max_days * nbx * B))) return r;
    if ((r = rxb_alloc(c, &A.ibring, L * nb))) return r;
    if ((r = rxb_alloc(c, &A.sbar, nb))) return r;
    if ((r = rxb_alloc(c, &A.coef, nb))) return r;
    if ((r = rxb_alloc(c, &A.gpart, (size_t)nbx * B * kTheta))) return r;
    if ((r = rxb_alloc(c, &c->b_I, (size_t)c->max_days * B))) return r;
    if ((r = rxb_alloc(c, &c->b_y, (size_t)c->max_days * B))) return r;
    if ((r = rxb_alloc(c, &c->b_Ibar, (size_t)c->max_days * B))) return r;
    if ((r = rxb_alloc(c, &c->b_loss, B))) return r;
    if ((r = rxb_alloc(c, &c->b_grad, (size_t)B * kTheta))) return r;
    return DEABM_OK;
}

// forward with checkpoints and the reverse sweep for B columns
static int rxb_gradient(deabm_relaxed *c, uint32_t T, uint32_t B, bool want_grad)
{
    cudaStream_t s = c->stream;
    RxParams P = c->P;
    P.T = T;
    RxbArrays A = c->bat;
    A.B = B;
    A.theta = c->b_theta;
    const size_t n = c->n, L = c->L, nb = n * B;
    const dim3 blk(32, 8), grid((unsigned)((n + 7) / 8), (B + 31) / 32);
    rxb_init_kernel<<<1024, 256, 0, s>>>(P, A, c->seeds, c->n_seeds);
    if (c->n_seeds)
        rxb_seed_kernel<<<(unsigned)(((size_t)c->n_seeds * B + 255) / 256), 256, 0, s>>>(P, A, c->seeds, c->n_seeds);
    RCU(cudaGetLastError());
    for (uint32_t t = 0; t < T; ++t) {
        if (t % c->K == 0) {
            float *ck = c->b_ckpt + (size_t)(t / c->K) * (L + 1) * nb;
            RCU(cudaMemcpyAsync(ck, A.s, 4 * nb, cudaMemcpyDeviceToDevice, s));
            RCU(cudaMemcpyAsync(ck + nb, A.xring, 4 * L * nb, cudaMemcpyDeviceToDevice, s));
        }
        rxb_inf_kernel<<<grid, blk, 0, s>>>(P, A, (int)t);
        rxb_day_kernel<false><<<grid, blk, 0, s>>>(P, A, (int)t, 0);
    }
    rxb_loss_kernel<<<B, 256, 0, s>>>(P, A, T, c->b_y, c->b_I, c->b_Ibar, c->b_loss);
    RCU(cudaGetLastError());
    if (!want_grad) return DEABM_OK;
    RCU(cudaMemsetAsync(A.sbar, 0, 4 * nb, s));
    RCU(cudaMemsetAsync(A.ibring, 0, 4 * L * nb, s));
    RCU(cudaMemsetAsync(A.gpart, 0, sizeof(double) * A.nbx * B * kTheta, s));
    const uint32_t nseg = (T + c->K - 1) / c->K;
    for (int sg = (int)nseg - 1; sg >= 0; --sg) {
        const uint32_t t0 = (uint32_t)sg * c->K, t1 = t0 + c->K < T ? t0 + c->K : T;
        const float *ck = c->b_ckpt + (size_t)sg * (L + 1) * nb;
        RCU(cudaMemcpyAsync(A.s, ck, 4 * nb, cudaMemcpyDeviceToDevice, s));
        RCU(cudaMemcpyAsync(A.xring, ck + nb, 4 * L * nb, cudaMemcpyDeviceToDevice, s));
        for (uint32_t t = t0; t < t1; ++t) {
            rxb_inf_kernel<<<grid, blk, 0, s>>>(P, A, (int)t);
            rxb_day_kernel<true><<<grid, blk, 0, s>>>(P, A, (int)t, (int)(t - t0));
        }
        for (int t = (int)t1 - 1; t >= (int)t0; --t) {
            rxb_adj_kernel<<<grid, blk, 0, s>>>(P, A, t, t - (int)t0, c->b_Ibar);
            rxb_scatter_static_kernel<<<grid, blk, 0, s>>>(P, A, t);
            if (P.rand_on) rxb_scatter_random_kernel<<<grid, blk, 0, s>>>(P, A, t);
            if (P.n_occ) rxb_scatter_occ_kernel<<<grid, blk, 0, s>>>(P, A, t);
        }
    }
    rxb_grad_reduce_kernel<<<(B * kTheta + 255) / 256, 256, 0, s>>>(A, c->b_grad);
    RCU(cudaGetLastError());
    return DEABM_OK;
}

extern "C" int deabm_grad_batch(deabm_relaxed *c, uint32_t T, uint32_t B, const float *theta, const float *target,
                                float *loss, float *grad, float *incidence)
{
    int r;
    if ((r = rx_check(c, T))) return r;
    if (B == 0 || B > 4096) return rx_fail(DEABM_EINVAL, "B must be in 1..4096");
    if (!theta || (!target && (loss || grad))) return rx_fail(DEABM_EINVAL, "theta is required, and target for loss or grad");
    for (size_t q = 0; q < (size_t)B * kTheta; ++q)
        if (!(theta[q] >= 0.0f) || !std::isfinite(theta[q]))
            return rx_fail(DEABM_EINVAL, "theta[%zu][%zu] must be finite and >= 0", q / kTheta, q % kTheta);
    if ((r = rxb_reserve(c, B))) return r;
    cudaStream_t s = c->stream;
    RCU(cudaMemcpyAsync(c->b_theta, theta, 4ull * B * kTheta, cudaMemcpyHostToDevice, s));
    if (target) RCU(cudaMemcpyAsync(c->b_y, target, 4ull * T * B, cudaMemcpyHostToDevice, s));
    c->bat.B = B;
    // without a target only the forward pass runs (the loss kernel then skips the loss)
    float *ysave = c->b_y;
    if (!target) c->b_y = nullptr;
    r = rxb_gradient(c, T, B, grad != nullptr);
    c->b_y = ysave;
    if (r) return r;
    if (loss) RCU(cudaMemcpyAsync(loss, c->b_loss, 4ull * B, cudaMemcpyDeviceToHost, s));
    if (grad) RCU(cudaMemcpyAsync(grad, c->b_grad, 4ull * B * kTheta, cudaMemcpyDeviceToHost, s));
    if (incidence) RCU(cudaMemcpyAsync(incidence, c->b_I, 4ull * T * B, cudaMemcpyDeviceToHost, s));
    RCU(cudaStreamSynchronize(s));
    return DEABM_OK;
}
