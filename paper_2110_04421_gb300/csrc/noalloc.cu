// noalloc.cu -- deabm_lambda_noalloc: the infection rates of one simulated day
// computed without allocating any memory.
//
// Who needs this: callers that are not allowed to allocate device memory at the
// point where they call us -- for example code running inside a memory pool that
// another runtime owns and sizes up front, an embedding host whose allocator
// hooks forbid cudaMalloc after start-up, or a real-time loop where an
// allocation (and the device-wide synchronisation it may imply) is not
// acceptable.  They pass their own device buffers for every input and output;
// the working memory (the day's emitted-infectiousness vector and the small
// tables) lives in a fixed array inside this library instead.
//
// The fixed array below is part of the library image: every GPU on which the
// library is loaded holds its 4 MiB + 4 KiB until the process exits.  All calls
// share it and it keeps the last call's contents, so calls whose work overlaps
// on the GPU (two streams, two host threads) race with each other; serialise
// them.  Each call rewrites every part of the array it reads, so nothing has to
// start at zero.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>

#include "day_common.cuh"
#include "deabm.h"
#include "deabm_device.cuh"
#include "gamma_day.cuh"

namespace deabm {

constexpr size_t kTablesBytes = (sizeof(Tables) + 255) / 256 * 256;
constexpr size_t kScratchBytes = kTablesBytes + (size_t)DEABM_NOALLOC_MAX_AGENTS * sizeof(float);

// [ Tables | emitted infectiousness of up to DEABM_NOALLOC_MAX_AGENTS agents ]
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct NoAllocTableArgs {
    double shape[DEABM_N_CLASS], scale[DEABM_N_CLASS];
    float A[DEABM_N_CLASS];
    uint32_t len;
    uint64_t pois[DEABM_POIS_CAP];
};

// one block: rebuild the tables in the fixed array
__global__ void na_tables_kernel(Tables *tab, const NoAllocTableArgs a)
{
    const uint32_t c = threadIdx.y, t = threadIdx.x;  // 64 x 3 threads
    float v = 0.0f;
    if (t >= 1 && t < a.len) v = __fmul_rn(a.A[c], (float)gamma_day(a.shape[c], a.scale[c], t));
    tab->infT[c][t] = v;
    if (c == 0 && t < DEABM_POIS_CAP) tab->pois[t] = a.pois[t];
}

__global__ void na_emit_kernel(const KParams P, const int8_t *stage, const int16_t *tinf, const uint8_t *qt, float *inf)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x)
        inf[i] = emitted(P.tab, P.inf_len, stage[i], tinf[i], qt[i] & 0x0Fu);
}

__global__ void __launch_bounds__(256) na_lambda_kernel(const KParams P, const Rep rp, uint32_t day, const float *inf,
                                                        float *lambda)
{
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.n) return;
    InfBuffers I;
    I.cur = inf;
    I.next = nullptr;
    I.rand_cur = inf;
    I.rand_next = nullptr;
    I.row_of = nullptr;
    uint32_t k;
    // the caller's age codes are not checked on the host (device memory): an
    // age bin outside 0..8 gives NaN instead of a read past S_age
    const uint32_t age = __ldg(P.age + j);
    lambda[j] = age < DEABM_N_AGE ? lambda_of<false>(P, rp, I, j, j, day, 1u, 0u, (int)age, &k) : __int_as_float(0x7FC00000);
}

}  // namespace deabm

using namespace deabm;

static thread_local std::string g_na_err;
static int na_fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_na_err = buf;
    return code;
}

static uint64_t na_threshold(double p)
{
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return (uint64_t)1 << 32;
    return (uint64_t)std::floor(p * 4294967296.0);
}

extern "C" int deabm_lambda_noalloc(const deabm_graph *graph_dev, const uint8_t *age_bin, const int8_t *stage,
                                    const int16_t *tinf, const uint8_t *qt, const deabm_params *params, uint32_t day,
                                    float *lambda, void *cuda_stream)
{
    if (!graph_dev || !params || !age_bin || !stage || !tinf || !qt || !lambda)
        return na_fail(DEABM_EINVAL, "deabm_lambda_noalloc: a required pointer is NULL");
    const uint32_t n = graph_dev->n_agents;
    if (n == 0) return DEABM_OK;
    if (n > DEABM_NOALLOC_MAX_AGENTS)
        return na_fail(DEABM_EINVAL, "deabm_lambda_noalloc: %u agents exceed the fixed working array (%u agents max)", n,
                       (unsigned)DEABM_NOALLOC_MAX_AGENTS);
    if (graph_dev->n_nets > DEABM_MAX_NETS) return na_fail(DEABM_EINVAL, "deabm_lambda_noalloc: n_nets > 4");
    if (graph_dev->n_occ)
        return na_fail(DEABM_EINVAL, "deabm_lambda_noalloc: daily occupation networks need a context (n_occ must be 0)");
    if (graph_dev->rand_ws)
        return na_fail(DEABM_EINVAL, "deabm_lambda_noalloc: the Watts-Strogatz random network needs a context (rand_ws must be 0)");
    if (graph_dev->rand_by_age)
        return na_fail(DEABM_EINVAL, "deabm_lambda_noalloc: age-stratified random means need a context (rand_by_age must be 0)");
    for (uint32_t k = 0; k < graph_dev->n_nets; ++k)
        if (!graph_dev->row_ptr[k] || !graph_dev->col[k])
            return na_fail(DEABM_EINVAL, "deabm_lambda_noalloc: network %u has a NULL array", k);
    if (params->inf_len == 0 || params->inf_len > DEABM_MAX_INF_LEN)
        return na_fail(DEABM_EINVAL, "deabm_lambda_noalloc: inf_len must be 1..64");
    for (int c = 0; c < DEABM_N_CLASS; ++c)
        if (!(params->inf_shape[c] > 0.0) || !(params->inf_scale[c] > 0.0))
            return na_fail(DEABM_EINVAL, "deabm_lambda_noalloc: gamma shape and scale must be > 0");
    if (!(graph_dev->rand_mean >= 0.0f) || (graph_dev->rand_mean > 0.0f && n < 2))
        return na_fail(DEABM_EINVAL, "deabm_lambda_noalloc: bad rand_mean for %u agents", n);

    // the device address of the fixed array on the current device, looked up on
    // every call (no allocation; valid after a device reset too).  The first
    // lookup on a device may load the library's device code there, so the first
    // call on each device belongs before any stream capture.
    void *base = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
    if (e != cudaSuccess || !base)
        return na_fail(DEABM_ECUDA, "cudaGetSymbolAddress of the working array: %s", cudaGetErrorString(e));
    Tables *tab = (Tables *)base;
    float *inf = (float *)((unsigned char *)base + kTablesBytes);
    cudaStream_t s = (cudaStream_t)cuda_stream;

    NoAllocTableArgs ta{};
    for (int c = 0; c < DEABM_N_CLASS; ++c) {
        ta.shape[c] = params->inf_shape[c];
        ta.scale[c] = params->inf_scale[c];
        ta.A[c] = params->A_class[c];
    }
    ta.len = params->inf_len;
    {
        // Poisson CDF thresholds: t_0 = exp(-m), t_k = (t_{k-1} * m) / k, c_k = c_{k-1} + t_k
        const double m = (double)graph_dev->rand_mean;
        volatile double t = std::exp(-m), cdf = t;
        ta.pois[0] = na_threshold(cdf);
        for (int k = 1; k < DEABM_POIS_CAP; ++k) {
            t = (t * m) / (double)k;
            cdf = cdf + t;
            ta.pois[k] = na_threshold(cdf);
        }
    }
    na_tables_kernel<<<1, dim3(DEABM_MAX_INF_LEN, DEABM_N_CLASS), 0, s>>>(tab, ta);

    KParams K{};
    K.n = n;
    K.n_nets = graph_dev->n_nets;
    K.n_rep = 1;
    K.inf_len = params->inf_len;
    K.dt = params->dt;
    K.rand_on = graph_dev->rand_mean > 0.0f ? 1u : 0u;
    for (uint32_t k = 0; k < graph_dev->n_nets; ++k) {
        K.row_ptr[k] = graph_dev->row_ptr[k];
        K.col[k] = graph_dev->col[k];
    }
    K.net_seed = params->net_seed;
    {
        uint32_t k0 = (uint32_t)params->net_seed, k1 = (uint32_t)(params->net_seed >> 32);
        for (int r = 0; r < 10; ++r) {  // the round keys of net_seed (philox_rk)
            K.nrk[2 * r] = k0;
            K.nrk[2 * r + 1] = k1;
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
    K.tab = tab;
    K.pois_fin = 0;
    for (int k = 0; k < DEABM_POIS_CAP; ++k) {
        K.pois32[k] = ta.pois[k] < ((uint64_t)1 << 32) ? (uint32_t)ta.pois[k] : 0xFFFFFFFFu;
        if (ta.pois[k] < ((uint64_t)1 << 32)) K.pois_fin = (uint32_t)k + 1u;
    }
    K.age = age_bin;
    Rep rp{};
    volatile float rv = params->R, ib = params->inv_Ibar;  // one FP32 product, as in deabm_create
    rp.cR = rv * ib;
    for (int k = 0; k < DEABM_MAX_NETS; ++k) rp.B_net[k] = params->B_net[k];
    rp.B_rand = params->B_rand;
    for (int q = 0; q < DEABM_N_AGE; ++q) rp.S_age[q] = params->S_age[q];
    const uint32_t blocks = (n + 255u) / 256u;
    na_emit_kernel<<<blocks < 4096u ? blocks : 4096u, 256, 0, s>>>(K, stage, tinf, qt, inf);
    na_lambda_kernel<<<blocks, 256, 0, s>>>(K, rp, day, inf, lambda);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(DEABM_ECUDA, "launch: %s", cudaGetErrorString(e));
    return DEABM_OK;
}

extern "C" const char *deabm_lambda_noalloc_last_error(void) { return g_na_err.c_str(); }
