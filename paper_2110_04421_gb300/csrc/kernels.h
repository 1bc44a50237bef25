// kernels.h -- host-side launchers of libdeabm's kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include "deabm_device.cuh"

namespace deabm {

// one simulated day: reads inf_cur and the state, writes the state, inf_next and the day's counters
cudaError_t launch_step(const KParams &P, uint32_t day, const InfBuffers &I, const StateRef &S, const Counters &C,
                        float *lam_out, float *p_out, cudaStream_t stream);

// one simulated day of a ragged batch of populations (persistent CTAs, tile queue)
cudaError_t launch_step_ragged(const PopDesc *pops, const Tile *tiles, uint32_t n_tiles, uint32_t *queue, uint32_t day,
                               const float *inf_cur, float *inf_next, const StateRef &S, const Counters &C,
                               uint32_t n_pops, uint32_t grid, bool occ, bool wsg, bool den, cudaStream_t stream);

// daily dose selection of the vaccination priority strategies: dose_caller[o] = 1
// for the agents (caller ids) dosed today; scratch of vax_select_scratch_words(n)
cudaError_t launch_vax_select(const KParams &P, uint32_t day, uint32_t dose2_delay, uint32_t elderly_bin,
                              uint32_t supply, const StateRef &S, uint8_t *cls_caller, uint8_t *dose_caller,
                              uint32_t *scratch, cudaStream_t stream);
size_t vax_select_scratch_words(uint32_t n);
// the same in every replicate column of a batched context (state [N][B], each
// column's dose-2 delay, the same supply): dose [caller id][B]; scratch of
// vax_select_batch_scratch_words(n, B)
cudaError_t launch_vax_select_batch(const KParams &P, uint32_t day, uint32_t elderly_bin, uint32_t supply,
                                    const StateRef &S, uint8_t *cls, uint8_t *dose, uint32_t *scratch,
                                    cudaStream_t stream);
size_t vax_select_batch_scratch_words(uint32_t n, uint32_t B);

// set-up: infectiousness table (FP64 gamma integrals, rounded once, times A_class)
cudaError_t launch_inf_table(Tables *tab, const double *shape_scale /*device [6]*/, const float *A_class /*device [3]*/,
                             uint32_t len, cudaStream_t stream);
// set-up: first-dose day of every agent from the age-priority order
cudaError_t launch_dose1_days(const uint8_t *age, uint32_t n, uint32_t start, uint32_t per_day, int16_t *out,
                              uint32_t *scratch /*device, 9 * (blocks + 1) + 9 words*/, cudaStream_t stream);
size_t dose1_scratch_words(uint32_t n);
// set-up: infections before day 0 for every replicate
cudaError_t launch_seed(const KParams &P, const uint32_t *ids, uint32_t n_ids, const StateRef &S, cudaStream_t stream);
// set-up: emitted infectiousness of the current state (inf_rand: copy by caller id, or nullptr)
cudaError_t launch_emit(const KParams &P, const StateRef &S, float *inf, float *inf_rand, cudaStream_t stream);
// exposure notification: app holders drawn at set-up (per replicate column), and
// the notification pass of a plain context that follows each day's update
cudaError_t launch_den_apps(const KParams &P, const StateRef &S, cudaStream_t stream);
cudaError_t launch_den(const KParams &P, uint32_t day, const StateRef &S, const Counters &C, cudaStream_t stream);
// the notification pass of a batched context ([N][B] state; positives in P.den_bits
// as [N][ceil(B/32)] words; row_of: caller id -> row, or nullptr when not
// relabelled; notified count of column b at C.den[day * den_stride + den_col0 + b]);
// also a ragged population's pass (one column, its counter column den_col0)
cudaError_t launch_den_batch(const KParams &P, uint32_t day, const uint32_t *row_of, const StateRef &S,
                             const Counters &C, uint32_t den_stride, uint32_t den_col0, cudaStream_t stream);
// internal numbering: min-label rounds over a CSR (at most `rounds`, even,
// fewer once the labels stop moving; result in label, tmp is scratch of n words,
// changed one device word; synchronises the stream after each pair of rounds);
// a CSR rebuilt in the new numbering (rp_new n+1
// words, col_new as many as col, scratch of scan_scratch_words(n + 1) words);
// internal-order arrays ([n][n_rep] of elem = 1, 2 or 4 bytes) back to caller order
cudaError_t launch_locality_labels(const uint32_t *rp, const uint32_t *col, uint32_t n, uint32_t rounds,
                                   uint32_t *label, uint32_t *tmp, uint32_t *changed, cudaStream_t stream);
cudaError_t launch_csr_renumber(const uint32_t *rp, const uint32_t *col, const uint32_t *new2orig,
                                const uint32_t *orig2new, uint32_t n, uint32_t *rp_new, uint32_t *col_new,
                                uint32_t *scratch, cudaStream_t stream);
size_t scan_scratch_words(size_t m);
// the day's Watts-Strogatz random network (wsg.cu): device buffers over n agents
// with h owned edges each -- rew [n], far [n h], ends [n+3] (agent v's landing
// slots are land[ends[v+2] .. ends[v+3]) after the build), land [n h],
// scratch [wsg_scratch_words(n)]
struct WsgBuffers {
    uint8_t *rew;
    uint32_t *far, *ends, *land, *scratch;
};
size_t wsg_scratch_words(uint32_t n);
cudaError_t launch_wsg_build(const KParams &P, uint32_t day, const WsgBuffers &B, cudaStream_t stream);
// points the day view (wsg_start, wsg_land) of the parameters at kp_dev (device
// memory) at slot day % wsg_ring_days of their ring of graphs
cudaError_t launch_wsg_slot(KParams *kp_dev, uint32_t day, cudaStream_t stream);
// in-place inclusive prefix sum of m words (scratch of scan_scratch_words(m) words)
cudaError_t launch_scan_inclusive(uint32_t *a, size_t m, uint32_t *scratch, cudaStream_t stream);
// new2orig[q] = the agent at internal row q: agents by ascending label (labels
// < n), ids ascending among equal labels.  label is overwritten; scratch of
// order_scratch_words(n) words.
size_t order_scratch_words(uint32_t n);
cudaError_t launch_order_by_label(uint32_t *label, uint32_t n, uint32_t *new2orig, uint32_t *scratch,
                                  cudaStream_t stream);
// orig2new[new2orig[q]] = q
cudaError_t launch_invert(const uint32_t *new2orig, uint32_t n, uint32_t *orig2new, cudaStream_t stream);
// ids[i] = orig2new[ids[i]] for i < m (every ids[i] < the population size)
cudaError_t launch_map_ids(uint32_t *ids, uint32_t m, const uint32_t *orig2new, cudaStream_t stream);
// out[v] = base + (local ? local[v] : v) for v < n
cudaError_t launch_offset_ids(uint32_t *out, const uint32_t *local, uint32_t n, uint32_t base, cudaStream_t stream);
cudaError_t launch_to_caller(void *out, const void *in, const uint32_t *orig, uint32_t n, uint32_t n_rep,
                             uint32_t elem, cudaStream_t stream);
// caller-order [n] (in_reps false) or [n][n_rep] array (elem = 1 or 2 bytes) to
// internal order [n][n_rep] (orig null: same order)
cudaError_t launch_from_caller(void *out, const void *in, const uint32_t *orig, uint32_t n, uint32_t n_rep,
                               uint32_t elem, bool in_reps, cudaStream_t stream);
// exposure notification: redraw the app holders' contact records of days [d0, d1)
cudaError_t launch_den_records(const KParams &P, uint32_t d0, uint32_t d1, cudaStream_t stream);
// out[i] = in[idx[i]] for i < n
cudaError_t launch_gather_i16(int16_t *out, const int16_t *in, const uint32_t *idx, uint32_t n, cudaStream_t stream);

}  // namespace deabm
