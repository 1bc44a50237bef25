// setup_kernels.cu -- device set-up of a simulation: infectiousness table,
// vaccination schedule, initial infections, first emitted-infectiousness vector.
#include <cuda_runtime.h>
#include <cstdint>

#include "deabm_device.cuh"
#include "gamma_day.cuh"
#include "kernels.h"

namespace deabm {

// ---------------------------------------------------------------- Eq. 1 integral
// gamma_day() from gamma_day.cuh, rounded once to FP32 and scaled by A_c.
__global__ void inf_table_kernel(Tables *tab, const double *shape_scale, const float *A_class, uint32_t len)
{
    const uint32_t c = blockIdx.x, t = threadIdx.x;
    if (c >= DEABM_N_CLASS || t >= DEABM_MAX_INF_LEN) return;
    float v = 0.0f;
    if (t >= 1 && t < len) v = __fmul_rn(A_class[c], (float)gamma_day(shape_scale[c], shape_scale[3 + c], t));
    tab->infT[c][t] = v;
}

cudaError_t launch_inf_table(Tables *tab, const double *shape_scale, const float *A_class, uint32_t len,
                             cudaStream_t stream)
{
    inf_table_kernel<<<DEABM_N_CLASS, DEABM_MAX_INF_LEN, 0, stream>>>(tab, shape_scale, A_class, len);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- vaccination order
// Priority: age bin descending, then agent id ascending.  rank_j = number of agents
// in older bins + number of same-bin agents with a smaller id; day = start + rank / per_day.
constexpr uint32_t kRankBlock = 1024;

__global__ void age_count_kernel(const uint8_t *age, uint32_t n, uint32_t *cnt /*[blocks][9]*/)
{
    __shared__ uint32_t s[DEABM_N_AGE];
    if (threadIdx.x < DEABM_N_AGE) s[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t j = blockIdx.x * kRankBlock + threadIdx.x;
    if (j < n) atomicAdd(&s[age[j]], 1u);
    __syncthreads();
    if (threadIdx.x < DEABM_N_AGE) cnt[blockIdx.x * DEABM_N_AGE + threadIdx.x] = s[threadIdx.x];
}

// one warp per age bin: turns the per-block counts into each block's first rank
// in the priority order (in place); launched as one block of 9 warps
__global__ void __launch_bounds__(32 * DEABM_N_AGE) age_offsets_kernel(uint32_t *cnt, uint32_t blocks)
{
    __shared__ uint32_t total[DEABM_N_AGE];
    const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    uint32_t sum = 0;
    for (uint32_t q = lane; q < blocks; q += 32u) sum += cnt[q * DEABM_N_AGE + w];
    sum = __reduce_add_sync(0xFFFFFFFFu, sum);
    if (lane == 0) total[w] = sum;
    __syncthreads();
    uint32_t running = 0;
    for (uint32_t a = w + 1; a < DEABM_N_AGE; ++a) running += total[a];  // older bins come first
    for (uint32_t q0 = 0; q0 < blocks; q0 += 32u) {
        const uint32_t q = q0 + lane;
        const uint32_t c = q < blocks ? cnt[q * DEABM_N_AGE + w] : 0u;
        uint32_t incl = c;
        for (uint32_t off = 1; off < 32u; off <<= 1) {
            const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, off);
            if (lane >= off) incl += v;
        }
        if (q < blocks) cnt[q * DEABM_N_AGE + w] = running + incl - c;
        running += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
}

__global__ void __launch_bounds__(kRankBlock) dose1_kernel(const uint8_t *age, uint32_t n, const uint32_t *off,
                                                           uint32_t start, uint32_t per_day, int16_t *out)
{
    __shared__ uint32_t warp_cnt[kRankBlock / 32][DEABM_N_AGE];
    const uint32_t j = blockIdx.x * kRankBlock + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const int a = j < n ? age[j] : -1;
    uint32_t before = 0;
    for (int q = 0; q < DEABM_N_AGE; ++q) {
        const unsigned m = __ballot_sync(0xFFFFFFFFu, a == q);
        if (a == q) before = __popc(m & ((1u << lane) - 1u));
        if (lane == 0) warp_cnt[w][q] = __popc(m);
    }
    __syncthreads();
    if (j >= n) return;
    uint32_t rank = off[blockIdx.x * DEABM_N_AGE + a] + before;
    for (uint32_t v = 0; v < w; ++v) rank += warp_cnt[v][a];
    int16_t d = kNever;
    if (per_day > 0) {
        const uint64_t day = (uint64_t)start + rank / per_day;
        d = day >= (uint64_t)kNever ? kNever : (int16_t)day;
    }
    out[j] = d;
}

size_t dose1_scratch_words(uint32_t n) { return (size_t)((n + kRankBlock - 1) / kRankBlock + 1) * DEABM_N_AGE; }

cudaError_t launch_dose1_days(const uint8_t *age, uint32_t n, uint32_t start, uint32_t per_day, int16_t *out,
                              uint32_t *scratch, cudaStream_t stream)
{
    const uint32_t blocks = (n + kRankBlock - 1) / kRankBlock;
    if (blocks == 0) return cudaSuccess;
    age_count_kernel<<<blocks, kRankBlock, 0, stream>>>(age, n, scratch);
    age_offsets_kernel<<<1, 32 * DEABM_N_AGE, 0, stream>>>(scratch, blocks);
    dose1_kernel<<<blocks, kRankBlock, 0, stream>>>(age, n, scratch, start, per_day, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- initial cases
__global__ void seed_kernel(const KParams P, const uint32_t *ids, uint32_t n_ids, StateRef S)
{
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t b = blockIdx.y;
    if (q >= n_ids || b >= P.n_rep) return;
    const uint32_t j = ids[q];
    if (j >= P.n) return;
    const size_t i = (size_t)j * P.n_rep + b;
    if (S.stage[i] != DEABM_S) return;
    const uint2 key = seed_key(P.rep[b].seed);
    const uint32_t jo = P.orig_id ? P.orig_id[j] : j;
    AgentState a{};
    new_infection(P.tab, P.age[j], draw(key, jo, kSeedDay, kStreamProg), a);
    S.stage[i] = (int8_t)a.st;
    S.timer[i] = (int16_t)a.tm;
    S.tinf[i] = (int16_t)a.ti;
}

cudaError_t launch_seed(const KParams &P, const uint32_t *ids, uint32_t n_ids, const StateRef &S, cudaStream_t stream)
{
    if (n_ids == 0) return cudaSuccess;
    const dim3 grid((n_ids + 255u) / 256u, P.n_rep);
    seed_kernel<<<grid, 256, 0, stream>>>(P, ids, n_ids, S);
    return cudaGetLastError();
}

__global__ void emit_kernel(const KParams P, StateRef S, float *inf, float *inf_rand)
{
    const size_t total = (size_t)P.n * P.n_rep;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const float v = emitted(P.tab, P.inf_len, S.stage[i], S.tinf[i], S.qt[i] & 0x0Fu);
        inf[i] = v;
        if (inf_rand) {
            const size_t j = i / P.n_rep, b = i % P.n_rep;
            inf_rand[(size_t)P.orig_id[j] * P.n_rep + b] = v;
        }
    }
}

cudaError_t launch_emit(const KParams &P, const StateRef &S, float *inf, float *inf_rand, cudaStream_t stream)
{
    const size_t total = (size_t)P.n * P.n_rep;
    const uint32_t blocks = (uint32_t)((total + 255) / 256 < 152 * 16 ? (total + 255) / 256 : 152 * 16);
    if (blocks == 0) return cudaSuccess;
    emit_kernel<<<blocks, 256, 0, stream>>>(P, S, inf, inf_rand);
    return cudaGetLastError();
}

__global__ void gather_i16_kernel(int16_t *out, const int16_t *in, const uint32_t *idx, uint32_t n)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = in[idx[i]];
}

cudaError_t launch_gather_i16(int16_t *out, const int16_t *in, const uint32_t *idx, uint32_t n, cudaStream_t stream)
{
    if (n == 0) return cudaSuccess;
    gather_i16_kernel<<<(n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096, 256, 0, stream>>>(out, in, idx, n);
    return cudaGetLastError();
}

}  // namespace deabm
