// relabel.cu -- the library's internal agent numbering, built on the GPU.
//
// Agents are renumbered so that the members of a group (a workplace) sit next
// to each other and a warp's in-edge gathers touch few cache lines.  The order
// is: agents grouped by the smallest id that reaches them along the in-edges
// of the network with the most edges (a min-label propagation of at most a
// fixed number of rounds, stopped once no label moves), groups in order of that
// label, ids ascending inside a group.
// Any permutation gives the same results (draws and outputs use the caller's
// ids); this one only decides where data sits.  Also here: the CSR rebuilt in
// the new numbering and the copy of internal-order arrays back to caller order.
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>

#include "kernels.h"

namespace deabm {

__global__ void label_init_kernel(uint32_t *label, uint32_t n)
{
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) label[v] = v;
}

// one Jacobi round: out[v] = min(in[v], in[u] for every in-edge u -> v); *changed
// is set when some label moved
__global__ void label_round_kernel(const uint32_t *__restrict__ rp, const uint32_t *__restrict__ col,
                                   const uint32_t *__restrict__ in, uint32_t *__restrict__ out, uint32_t n,
                                   uint32_t *changed)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const uint32_t m0 = in[v];
    uint32_t m = m0;
    const uint32_t e1 = rp[v + 1];
    for (uint32_t e = rp[v]; e < e1; ++e) m = min(m, __ldg(in + col[e]));
    out[v] = m;
    if (m != m0) *changed = 1u;
}

cudaError_t launch_locality_labels(const uint32_t *rp, const uint32_t *col, uint32_t n, uint32_t rounds,
                                   uint32_t *label, uint32_t *tmp, uint32_t *changed, cudaStream_t stream)
{
    const uint32_t blocks = (n + 255u) / 256u;
    label_init_kernel<<<blocks, 256, 0, stream>>>(label, n);
    // rounds in pairs, so that the result ends in `label`; the labels have
    // converged (and the rest would change nothing) once a pair's second round
    // moved none of them
    for (uint32_t r = 0; r + 1u < rounds; r += 2u) {
        label_round_kernel<<<blocks, 256, 0, stream>>>(rp, col, label, tmp, n, changed);
        cudaError_t e = cudaMemsetAsync(changed, 0, sizeof(uint32_t), stream);
        if (e != cudaSuccess) return e;
        label_round_kernel<<<blocks, 256, 0, stream>>>(rp, col, tmp, label, n, changed);
        uint32_t moved = 1;
        if ((e = cudaMemcpyAsync(&moved, changed, sizeof moved, cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(stream)) != cudaSuccess)
            return e;
        if (!moved) break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- CSR in the new numbering
// deg[q + 1] = in-degree of the agent now at row q (deg[0] = 0)
__global__ void csr_degree_kernel(const uint32_t *__restrict__ rp, const uint32_t *__restrict__ new2orig, uint32_t n,
                                  uint32_t *__restrict__ deg)
{
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q == 0) deg[0] = 0;
    if (q >= n) return;
    const uint32_t o = new2orig[q];
    deg[q + 1] = rp[o + 1] - rp[o];
}

// inclusive scan of a[0..m) in place, in blocks of 1024 (block totals to `sums`)
constexpr uint32_t kScanBlock = 1024;

__device__ __forceinline__ uint32_t block_inclusive_scan(uint32_t x, uint32_t *warp_tot)
{
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
#pragma unroll
    for (uint32_t d = 1; d < 32u; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31u) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t t = lane < kScanBlock / 32u ? warp_tot[lane] : 0u;
#pragma unroll
        for (uint32_t d = 1; d < 32u; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, d);
            if (lane >= d) t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    return x + (wid ? warp_tot[wid - 1] : 0u);
}

__global__ void __launch_bounds__(kScanBlock) scan_blocks_kernel(uint32_t *a, size_t m, uint32_t *sums)
{
    __shared__ uint32_t warp_tot[32];
    const size_t i = (size_t)blockIdx.x * kScanBlock + threadIdx.x;
    const uint32_t x = block_inclusive_scan(i < m ? a[i] : 0u, warp_tot);
    if (i < m) a[i] = x;
    if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = x;
}

__global__ void add_block_offsets_kernel(uint32_t *a, size_t m, const uint32_t *sums)
{
    const size_t i = (size_t)blockIdx.x * kScanBlock + threadIdx.x;
    if (blockIdx.x > 0 && i < m) a[i] += sums[blockIdx.x - 1];
}

// Two-launch scan for up to kTileScanMaxTiles tiles of 4096 words: the tiles'
// totals, then each tile scanned with the sum of the totals before it as its
// offset (every block adds up that prefix itself; at most 4096 words).  Tiles
// move through shared memory so that global loads and stores stay coalesced
// while each thread scans 16 consecutive words.
constexpr uint32_t kTileThreads = 256, kTilePer = 16, kTileWords = kTileThreads * kTilePer;
constexpr size_t kTileScanMaxTiles = 4096;

__device__ __forceinline__ uint32_t block_sum_256(uint32_t x, uint32_t *red)
{
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    x = __reduce_add_sync(0xFFFFFFFFu, x);
    if (lane == 0) red[wid] = x;
    __syncthreads();
    uint32_t t = 0;
#pragma unroll
    for (uint32_t w = 0; w < kTileThreads / 32u; ++w) t += red[w];
    return t;
}

__global__ void __launch_bounds__(kTileThreads) tile_sum_kernel(const uint32_t *a, size_t m, uint32_t *sums)
{
    __shared__ uint32_t red[kTileThreads / 32u];
    const size_t base = (size_t)blockIdx.x * kTileWords;
    uint32_t x = 0;
#pragma unroll
    for (uint32_t i = 0; i < kTilePer; ++i) {
        const size_t q = base + i * kTileThreads + threadIdx.x;
        if (q < m) x += a[q];
    }
    const uint32_t t = block_sum_256(x, red);
    if (threadIdx.x == 0) sums[blockIdx.x] = t;
}

__device__ __forceinline__ uint32_t tile_slot(uint32_t p) { return p + (p >> 5); }  // one pad word per 32

__global__ void __launch_bounds__(kTileThreads) tile_scan_kernel(uint32_t *a, size_t m, const uint32_t *sums)
{
    __shared__ uint32_t red[kTileThreads / 32u];
    __shared__ uint32_t tile[kTileWords + kTileWords / 32u];
    const uint32_t tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5;
    const size_t base = (size_t)blockIdx.x * kTileWords;
    uint32_t pre = 0;  // this tile's offset: the totals of the tiles before it
    for (uint32_t b = tid; b < blockIdx.x; b += kTileThreads) pre += sums[b];
    const uint32_t off = block_sum_256(pre, red);
#pragma unroll
    for (uint32_t i = 0; i < kTilePer; ++i) {
        const uint32_t p = i * kTileThreads + tid;
        tile[tile_slot(p)] = base + p < m ? a[base + p] : 0u;
    }
    __syncthreads();
    uint32_t v[kTilePer], run = 0;
#pragma unroll
    for (uint32_t i = 0; i < kTilePer; ++i) {
        run += tile[tile_slot(tid * kTilePer + i)];
        v[i] = run;
    }
    // exclusive scan of the threads' runs
    uint32_t x = run;
#pragma unroll
    for (uint32_t d = 1; d < 32u; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= d) x += y;
    }
    __syncthreads();  // red is reused
    if (lane == 31u) red[wid] = x;
    __syncthreads();
    uint32_t wpre = 0;
    for (uint32_t w = 0; w < wid; ++w) wpre += red[w];
    const uint32_t excl = off + wpre + x - run;
#pragma unroll
    for (uint32_t i = 0; i < kTilePer; ++i) tile[tile_slot(tid * kTilePer + i)] = v[i] + excl;
    __syncthreads();
#pragma unroll
    for (uint32_t i = 0; i < kTilePer; ++i) {
        const uint32_t p = i * kTileThreads + tid;
        if (base + p < m) a[base + p] = tile[tile_slot(p)];
    }
}

// scratch: 2 * ceil(m / 1024) + 2 words (recursive block sums)
static cudaError_t scan_inplace(uint32_t *a, size_t m, uint32_t *scratch, cudaStream_t stream)
{
    if (m == 0) return cudaSuccess;
    const size_t nt = (m + kTileWords - 1) / kTileWords;
    if (nt >= 1 && nt <= kTileScanMaxTiles) {
        tile_sum_kernel<<<(unsigned)nt, kTileThreads, 0, stream>>>(a, m, scratch);
        tile_scan_kernel<<<(unsigned)nt, kTileThreads, 0, stream>>>(a, m, scratch);
        return cudaGetLastError();
    }
    const size_t nb = (m + kScanBlock - 1) / kScanBlock;
    scan_blocks_kernel<<<(unsigned)nb, kScanBlock, 0, stream>>>(a, m, scratch);
    if (nb > 1) {
        cudaError_t e = scan_inplace(scratch, nb, scratch + nb, stream);
        if (e != cudaSuccess) return e;
        add_block_offsets_kernel<<<(unsigned)nb, kScanBlock, 0, stream>>>(a, m, scratch);
    }
    return cudaGetLastError();
}

cudaError_t launch_scan_inclusive(uint32_t *a, size_t m, uint32_t *scratch, cudaStream_t stream)
{
    return scan_inplace(a, m, scratch, stream);
}

size_t scan_scratch_words(size_t m)
{
    size_t words = 0;
    while (m > 1) {
        m = (m + kScanBlock - 1) / kScanBlock;
        words += m;
    }
    return words + 2;
}

// One warp per 32 consecutive new rows: their edges form one contiguous output
// range, which the lanes fill 32 positions at a time (coalesced writes, no idle
// lanes on short rows).  Position p belongs to the last of the 32 rows whose
// output start is <= p (a binary search over the lanes' starts); each row keeps
// its edges in the caller's order, sources renumbered.
__global__ void csr_copy_kernel(const uint32_t *__restrict__ rp, const uint32_t *__restrict__ col,
                                const uint32_t *__restrict__ new2orig, const uint32_t *__restrict__ orig2new,
                                const uint32_t *__restrict__ rp_new, uint32_t n, uint32_t *__restrict__ col_new)
{
    const unsigned full = 0xFFFFFFFFu;
    const uint32_t q0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32u, lane = threadIdx.x & 31u;
    if (q0 >= n) return;  // whole warps leave together
    const uint32_t q = q0 + lane, last = min(31u, n - 1u - q0);
    uint32_t d0 = 0, len = 0, b0 = 0;
    if (q < n) {
        const uint32_t o = new2orig[q];
        b0 = rp[o];
        len = rp[o + 1] - b0;
        d0 = rp_new[q];
    }
    const uint32_t beg = __shfl_sync(full, d0, 0), end = __shfl_sync(full, d0 + len, last);
    for (uint32_t base = beg; base < end; base += 32u) {
        const uint32_t p = base + lane;
        uint32_t r = 0;
#pragma unroll
        for (uint32_t s = 16; s >= 1u; s >>= 1) {
            const uint32_t c = r + s;
            const uint32_t dc = __shfl_sync(full, d0, c);
            if (c <= last && dc <= p) r = c;
        }
        const uint32_t dr = __shfl_sync(full, d0, r), br = __shfl_sync(full, b0, r);
        if (p < end) col_new[p] = orig2new[col[br + (p - dr)]];
    }
}

cudaError_t launch_csr_renumber(const uint32_t *rp, const uint32_t *col, const uint32_t *new2orig,
                                const uint32_t *orig2new, uint32_t n, uint32_t *rp_new, uint32_t *col_new,
                                uint32_t *scratch, cudaStream_t stream)
{
    csr_degree_kernel<<<(n + 256u) / 256u, 256, 0, stream>>>(rp, new2orig, n, rp_new);
    cudaError_t e = scan_inplace(rp_new, (size_t)n + 1, scratch, stream);
    if (e != cudaSuccess) return e;
    const uint64_t threads = ((uint64_t)n + 31u) / 32u * 32u;  // one warp per 32 rows
    csr_copy_kernel<<<(unsigned)((threads + 255u) / 256u), 256, 0, stream>>>(rp, col, new2orig, orig2new, rp_new, n,
                                                                             col_new);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- order by label
// The internal order itself: (label, id) pairs sorted by label with a
// least-significant-digit radix sort, 8 bits a pass.  Every pass is stable and
// the ids start ascending, so ids stay ascending inside a group.  Pass: per
// tile a 256-bin count (hist[1 + digit * tiles + tile], digit-major), one
// inclusive scan over all counts (giving each (digit, tile) its first output
// slot), then each tile places its pairs in order: 256 at a time, a pair's
// slot = its (digit, tile) start + equal digits before it in this tile.
constexpr uint32_t kRadixThreads = 256;

__global__ void iota_kernel(uint32_t *v, uint32_t n)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = i;
}

__global__ void __launch_bounds__(kRadixThreads) radix_count_kernel(const uint32_t *__restrict__ key, uint32_t n,
                                                                    uint32_t shift, uint32_t items,
                                                                    uint32_t *__restrict__ hist, uint32_t tiles)
{
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t t0 = (uint64_t)blockIdx.x * items * kRadixThreads;
    for (uint32_t r = 0; r < items; ++r) {
        const uint64_t i = t0 + (uint64_t)r * kRadixThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(key[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[1u + (uint64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
    if (blockIdx.x == 0 && threadIdx.x == 0) hist[0] = 0;
}

__global__ void __launch_bounds__(kRadixThreads) radix_place_kernel(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, uint32_t n, uint32_t shift, uint32_t items, const uint32_t *__restrict__ start,
    uint32_t tiles)
{
    constexpr uint32_t W = kRadixThreads / 32u;
    __shared__ uint32_t next[256];     // next free slot of each digit for this tile
    __shared__ uint32_t wcnt[W][256];  // pairs of each digit in each warp of the current 256
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    next[tid] = start[(uint64_t)tid * tiles + blockIdx.x];  // exclusive: the scan ran over hist shifted by one
    const uint64_t t0 = (uint64_t)blockIdx.x * items * kRadixThreads;
    for (uint32_t r = 0; r < items; ++r) {
#pragma unroll
        for (uint32_t w = 0; w < W; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const uint64_t i = t0 + (uint64_t)r * kRadixThreads + tid;
        const bool valid = i < n;
        const uint32_t k = valid ? kin[i] : 0u;
        const uint32_t d = valid ? (k >> shift) & 255u : 256u + lane;  // past-the-end lanes match nobody
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t before = peers & ((1u << lane) - 1u);
        if (valid && before == 0u) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t slot = next[d] + __popc(before);
            for (uint32_t w = 0; w < warp; ++w) slot += wcnt[w][d];
            kout[slot] = k;
            vout[slot] = vin[i];
        }
        __syncthreads();
        uint32_t tot = 0;
#pragma unroll
        for (uint32_t w = 0; w < W; ++w) tot += wcnt[w][tid];
        next[tid] += tot;
    }
}

// pairs per thread of a tile: 8, more for very large n so that at most 16384
// tiles (and 4 M counts) are needed
static uint32_t radix_items(uint32_t n)
{
    const uint64_t per = (uint64_t)kRadixThreads * 16384u;
    return (uint32_t)std::max<uint64_t>(8u, ((uint64_t)n + per - 1) / per);
}

static uint32_t radix_tiles(uint32_t n, uint32_t items)
{
    const uint64_t tile = (uint64_t)items * kRadixThreads;
    return (uint32_t)(((uint64_t)n + tile - 1) / tile);
}

size_t order_scratch_words(uint32_t n)
{
    const size_t m = 256u * (size_t)radix_tiles(n, radix_items(n)) + 1u;
    return 2u * (size_t)n + m + scan_scratch_words(m);
}

cudaError_t launch_order_by_label(uint32_t *label, uint32_t n, uint32_t *new2orig, uint32_t *scratch,
                                  cudaStream_t stream)
{
    const uint32_t items = radix_items(n), tiles = radix_tiles(n, items);
    const size_t m = 256u * (size_t)tiles + 1u;
    uint32_t *k2 = scratch, *v2 = scratch + n, *hist = scratch + 2u * (size_t)n, *scan_tmp = hist + m;
    const uint32_t bits = n > 1u ? 32u - (uint32_t)__builtin_clz(n - 1u) : 1u;  // labels are < n
    const uint32_t passes = (bits + 7u) / 8u;
    // keys alternate label <-> k2, values v2 <-> new2orig, so that the last pass
    // writes its values to new2orig
    uint32_t *kin = label, *kout = k2, *vin = (passes & 1u) ? v2 : new2orig, *vout = (passes & 1u) ? new2orig : v2;
    iota_kernel<<<(n + 255u) / 256u, 256, 0, stream>>>(vin, n);
    for (uint32_t p = 0; p < passes; ++p) {
        radix_count_kernel<<<tiles, kRadixThreads, 0, stream>>>(kin, n, 8u * p, items, hist, tiles);
        cudaError_t e = scan_inplace(hist, m, scan_tmp, stream);
        if (e != cudaSuccess) return e;
        radix_place_kernel<<<tiles, kRadixThreads, 0, stream>>>(kin, vin, kout, vout, n, 8u * p, items, hist, tiles);
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    return cudaGetLastError();
}

// orig2new[new2orig[q]] = q
__global__ void invert_kernel(const uint32_t *__restrict__ new2orig, uint32_t n, uint32_t *__restrict__ orig2new)
{
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) orig2new[new2orig[q]] = q;
}

cudaError_t launch_invert(const uint32_t *new2orig, uint32_t n, uint32_t *orig2new, cudaStream_t stream)
{
    invert_kernel<<<(n + 255u) / 256u, 256, 0, stream>>>(new2orig, n, orig2new);
    return cudaGetLastError();
}

// ids[i] = orig2new[ids[i]]: caller ids to internal rows
__global__ void map_ids_kernel(uint32_t *ids, uint32_t m, const uint32_t *__restrict__ orig2new)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) ids[i] = orig2new[ids[i]];
}

cudaError_t launch_map_ids(uint32_t *ids, uint32_t m, const uint32_t *orig2new, cudaStream_t stream)
{
    map_ids_kernel<<<(m + 255u) / 256u, 256, 0, stream>>>(ids, m, orig2new);
    return cudaGetLastError();
}

// out[v] = base + (local ? local[v] : v): a population's rows to rows of the
// concatenated state
__global__ void offset_ids_kernel(uint32_t *__restrict__ out, const uint32_t *__restrict__ local, uint32_t n,
                                  uint32_t base)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) out[v] = base + (local ? local[v] : v);
}

cudaError_t launch_offset_ids(uint32_t *out, const uint32_t *local, uint32_t n, uint32_t base, cudaStream_t stream)
{
    offset_ids_kernel<<<(n + 255u) / 256u, 256, 0, stream>>>(out, local, n, base);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- from caller order
// out[q * n_rep + b] = in[orig[q]] (in[q] when orig is null), or
// in[orig[q] * n_rep + b] when the input has its replicates: a caller-order array
// put in internal order (and repeated over the replicates when it has none)
template <class T>
__global__ void from_caller_kernel(T *__restrict__ out, const T *__restrict__ in, const uint32_t *__restrict__ orig,
                                   uint32_t n, uint32_t n_rep, bool in_reps)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (uint64_t)n * n_rep) return;
    const uint32_t q = (uint32_t)(i / n_rep), b = (uint32_t)(i % n_rep);
    const uint64_t o = orig ? orig[q] : q;
    out[i] = in_reps ? in[o * n_rep + b] : in[o];
}

cudaError_t launch_from_caller(void *out, const void *in, const uint32_t *orig, uint32_t n, uint32_t n_rep,
                               uint32_t elem, bool in_reps, cudaStream_t stream)
{
    const uint64_t total = (uint64_t)n * n_rep;
    const unsigned blocks = (unsigned)((total + 255u) / 256u);
    if (elem == 1)
        from_caller_kernel<uint8_t><<<blocks, 256, 0, stream>>>((uint8_t *)out, (const uint8_t *)in, orig, n, n_rep,
                                                                 in_reps);
    else
        from_caller_kernel<uint16_t><<<blocks, 256, 0, stream>>>((uint16_t *)out, (const uint16_t *)in, orig, n,
                                                                  n_rep, in_reps);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- back to caller order
// out[(orig[q] * n_rep + b) * elem ...] = in[(q * n_rep + b) * elem ...]
template <class T>
__global__ void to_caller_kernel(T *__restrict__ out, const T *__restrict__ in, const uint32_t *__restrict__ orig,
                                 uint32_t n, uint32_t n_rep)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (uint64_t)n * n_rep) return;
    const uint32_t q = (uint32_t)(i / n_rep), b = (uint32_t)(i % n_rep);
    out[(uint64_t)orig[q] * n_rep + b] = in[i];
}

cudaError_t launch_to_caller(void *out, const void *in, const uint32_t *orig, uint32_t n, uint32_t n_rep,
                             uint32_t elem, cudaStream_t stream)
{
    const uint64_t total = (uint64_t)n * n_rep;
    const unsigned blocks = (unsigned)((total + 255u) / 256u);
    if (elem == 1)
        to_caller_kernel<uint8_t><<<blocks, 256, 0, stream>>>((uint8_t *)out, (const uint8_t *)in, orig, n, n_rep);
    else if (elem == 2)
        to_caller_kernel<uint16_t><<<blocks, 256, 0, stream>>>((uint16_t *)out, (const uint16_t *)in, orig, n, n_rep);
    else
        to_caller_kernel<uint32_t><<<blocks, 256, 0, stream>>>((uint32_t *)out, (const uint32_t *)in, orig, n, n_rep);
    return cudaGetLastError();
}

}  // namespace deabm
