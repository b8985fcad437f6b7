// Tile binning helpers (Sec. III-A, "Tiles"): the scan of per-Gaussian
// counts taken in depth order, and the ranges of runs in a sorted key array.
//   k_scan_*   -- exclusive scan of counts read through the depth order
//   k_ranges   -- [start, end) of every key value's run (keys masked to their
//                 low bits), by a 32-way search per value
//   k_expand_tile_ids -- the sorted tile id of every pair, from the ranges
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.cuh"

namespace splash {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *s_w, uint32_t *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    uint32_t base = 0, tot = 0;
    for (int i = 0; i < kScanThreads / 32; i++) {
        if (i < w) base += s_w[i];
        tot += s_w[i];
    }
    __syncthreads();
    *total = tot;
    return base + x - v;
}

// per chunk: sum of tile counts (in depth order)
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(int64_t n, const uint32_t *__restrict__ order,
                                                            const uint32_t *__restrict__ tt, uint32_t *__restrict__ sums)
{
    pdl_enter();
    __shared__ uint32_t s_w[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk;
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        const int64_t i = base + j * kScanThreads + threadIdx.x;
        if (i < n) acc += tt[order[i]];
    }
    uint32_t tot;
    block_exclusive_scan(acc, s_w, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// one block: exclusive scan of the chunk sums; total pair count to *total
__global__ void __launch_bounds__(kScanThreads) k_scan_top(int nchunks, uint32_t *__restrict__ sums, uint32_t *__restrict__ total)
{
    pdl_enter();
    __shared__ uint32_t s_w[kScanThreads / 32];
    uint32_t carry = 0;
    for (int b = 0; b < nchunks; b += kScanThreads) {
        const int i = b + threadIdx.x;
        const uint32_t v = i < nchunks ? sums[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(v, s_w, &tot);
        if (i < nchunks) sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

// per chunk: exclusive offsets of each depth-ranked Gaussian's pairs. With
// `own_prefix` the chunk adds up the sums of the chunks before it itself (a
// fixed-order block sum; used when there are few chunks, in place of
// k_scan_top) and the last chunk writes the total; otherwise sums[] holds the
// exclusive prefixes k_scan_top wrote.
__global__ void __launch_bounds__(kScanThreads) k_scan_down(int64_t n, const uint32_t *__restrict__ order,
                                                          const uint32_t *__restrict__ tt, const uint32_t *__restrict__ sums,
                                                          uint32_t *__restrict__ offsets, int own_prefix,
                                                          uint32_t *__restrict__ total)
{
    pdl_enter();
    __shared__ uint32_t s_w[kScanThreads / 32];
    uint32_t pre = 0;
    if (own_prefix) {  // uniform over the grid
        uint32_t a = 0;
        for (int i = threadIdx.x; i < (int)blockIdx.x; i += kScanThreads) a += sums[i];
        block_exclusive_scan(a, s_w, &pre);  // every thread gets the block total
    } else {
        pre = sums[blockIdx.x];
    }
    // blocked arrangement: thread t owns items [t*kScanItems, (t+1)*kScanItems) of the chunk
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    uint32_t c[kScanItems];
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        const int64_t i = base + j;
        c[j] = i < n ? tt[order[i]] : 0u;
        acc += c[j];
    }
    uint32_t tot;
    uint32_t run = pre + block_exclusive_scan(acc, s_w, &tot);
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        const int64_t i = base + j;
        if (i < n) offsets[i] = run;
        run += c[j];
    }
    if (own_prefix && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = pre + tot;
}

// Start of every tile's run in the sorted pairs, one warp per tile value t
// in [0, ntiles]: the first index whose tile id is >= t (a 32-way search: each
// round probes 32 evenly spaced keys, one per lane, and keeps the sub-interval
// between the last key below t and the first at or above it). Tile t's range
// is [start(t), start(t + 1)); every tile is written, empty ones as [s, s).
__global__ void __launch_bounds__(256) k_ranges(int64_t k_host, const uint32_t *__restrict__ k_dev,
                                                const uint32_t *__restrict__ tile_ids, uint2 *__restrict__ ranges,
                                                uint32_t ntiles, uint32_t mask)
{
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t > (int64_t)ntiles) return;  // uniform over the warp
    const int64_t k = k_dev ? (int64_t)*k_dev : k_host;
    const uint32_t tv = (uint32_t)t;
    // invariant: every key before lo is < t; hi == k or key[hi] >= t
    int64_t lo = 0, hi = k;
    while (hi - lo > 32) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t p = min(lo + (int64_t)(lane + 1) * step - 1, hi - 1);
        const uint32_t ge = __ballot_sync(0xffffffffu, (tile_ids[p] & mask) >= tv);
        if (ge == 0u) {
            lo = min(lo + 32 * step, hi);  // all 32 probes below t: past the last one
        } else {
            const int f = __ffs(ge) - 1;  // first probe at or above t
            hi = min(lo + (int64_t)(f + 1) * step - 1, hi - 1);
            if (f > 0) lo = lo + (int64_t)f * step;  // one past the probe before it
        }
    }
    const int64_t q = lo + lane;
    const uint32_t ge = __ballot_sync(0xffffffffu, q < hi && (tile_ids[q] & mask) >= tv);
    const int64_t start = ge ? lo + __ffs(ge) - 1 : hi;
    if (lane == 0) {
        if (t < (int64_t)ntiles) ranges[t].x = (uint32_t)start;
        if (t > 0) ranges[t - 1].y = (uint32_t)start;
    }
}

}  // namespace

void launch_count_scan(int64_t n, const uint32_t *order, const uint32_t *tt, uint32_t *offsets, uint32_t *sums,
                       uint32_t *total, cudaStream_t s)
{
    const int nchunks = (int)((n + kScanChunk - 1) / kScanChunk);
    if (n <= 0) {
        cudaMemsetAsync(total, 0, sizeof(uint32_t), s);
        return;
    }
    launch_pdl(k_scan_reduce, nchunks, kScanThreads, 0, s, n, order, tt, sums);
    count_launch();
    // up to 1024 chunks each chunk adds up its predecessors' sums itself
    const int own = nchunks <= 1024;
    if (!own) {
        launch_pdl(k_scan_top, 1, kScanThreads, 0, s, nchunks, sums, total);
        count_launch();
    }
    launch_pdl(k_scan_down, nchunks, kScanThreads, 0, s, n, order, tt, sums, offsets, own, total);
    count_launch();
}

void launch_ranges(int64_t k_host, const uint32_t *k_dev, const uint32_t *tile_ids, uint2 *ranges, int ntiles, cudaStream_t s,
                   uint32_t key_mask)
{
    if (ntiles <= 0) return;
    const int64_t warps = (int64_t)ntiles + 1;
    launch_pdl(k_ranges, (unsigned)((warps * 32 + 255) / 256), 256, 0, s, k_host, k_dev, tile_ids, ranges, (uint32_t)ntiles,
               key_mask);
    count_launch();
}

namespace {
// one warp per tile: its run of the sorted tile ids
__global__ void __launch_bounds__(256) k_expand_tile_ids(const uint2 *__restrict__ ranges, int ntiles,
                                                         uint32_t *__restrict__ tile_ids)
{
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= ntiles) return;
    const uint2 rg = ranges[t];
    for (uint32_t i = rg.x + (threadIdx.x & 31); i < rg.y; i += 32) tile_ids[i] = (uint32_t)t;
}
}  // namespace

void launch_expand_tile_ids(const uint2 *ranges, int ntiles, uint32_t *tile_ids, cudaStream_t s)
{
    if (ntiles <= 0) return;
    k_expand_tile_ids<<<(unsigned)(((int64_t)ntiles * 32 + 255) / 256), 256, 0, s>>>(ranges, ntiles, tile_ids);
    count_launch();
}

}  // namespace splash
