// Tile binning (Sec. III-A, "Tiles"): every Gaussian is listed in each tile
// its 3-sigma bounding box covers. The lists are emitted in depth order (the
// Gaussians come from the depth sort), so a stable sort by tile index yields
// per-tile lists sorted by depth with ties broken by Gaussian index.
//   k_scan_*  -- exclusive scan of the tile counts, taken in depth order
//   k_emit    -- write (tile index, Gaussian index) pairs
//   k_ranges  -- [start, end) of every tile's run in the sorted pairs
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

// One warp per 32 consecutive depth-ordered Gaussians. Their runs of pairs are
// consecutive in the output, so the warp writes the whole range together with
// coalesced stores: output slot s belongs to the last lane whose run starts at
// or before s (a 5-step shuffle search), and is the k-th tile of that lane's
// rectangle in row-major order. A Gaussian whose run does not fit the
// capacity writes nothing and is reported.
__global__ void __launch_bounds__(256) k_emit(int64_t n, const uint32_t *__restrict__ order, const uint32_t *__restrict__ offsets,
                                              const uint32_t *__restrict__ tt, const uint2 *__restrict__ rect, int tiles_x,
                                              uint32_t *__restrict__ tile_ids, uint32_t *__restrict__ gauss_ids,
                                              uint64_t capacity, uint32_t *__restrict__ status)
{
    constexpr uint32_t kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r - lane >= n) return;  // the whole warp is past the end
    uint32_t g = 0, cnt = 0, tx0 = 0, ty0 = 0, w = 1, fit = 0, off = 0;
    if (r < n) {
        g = order[r];
        cnt = tt[g];
        off = offsets[r];
        if (cnt) {
            const uint2 rc = rect[g];
            tx0 = rc.x & 0xffffu;
            ty0 = rc.y & 0xffffu;
            w = (rc.x >> 16) - tx0 + 1;
            fit = (uint64_t)off + cnt <= capacity;
            if (!fit) atomicOr(status, kStatusCapacity);
        }
    }
    // warp-local start of each lane's run: exclusive scan of the counts
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t loc = incl - cnt;
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t s = base + lane;
        int j = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t lj = __shfl_sync(kFull, loc, j + step);
            if (lj <= s) j += step;
        }
        const uint32_t og = __shfl_sync(kFull, g, j), otx0 = __shfl_sync(kFull, tx0, j), oty0 = __shfl_sync(kFull, ty0, j);
        const uint32_t ow = __shfl_sync(kFull, w, j), ofit = __shfl_sync(kFull, fit, j), oloc = __shfl_sync(kFull, loc, j);
        const uint32_t ooff = __shfl_sync(kFull, off, j);
        if (s < total && ofit) {
            // the owner's own offset: ofit guarantees ooff + its count <= capacity
            const uint32_t k = s - oloc, dy = k / ow, dx = k - dy * ow;
            tile_ids[(uint64_t)ooff + k] = (oty0 + dy) * (uint32_t)tiles_x + otx0 + dx;
            gauss_ids[(uint64_t)ooff + k] = og;
        }
    }
}

__device__ __forceinline__ void range_ends(int64_t i, uint32_t t, uint32_t prev, uint32_t next, int64_t k,
                                           uint2 *__restrict__ ranges, uint32_t ntiles)
{
    if (t >= ntiles) return;  // only after a capacity overflow (reported through the status word)
    if (i == 0 || prev != t) ranges[t].x = (uint32_t)i;
    if (i == k - 1 || next != t) ranges[t].y = (uint32_t)(i + 1);
}

// Starts and ends of the runs of equal tile ids: four ids per thread from one
// 16-byte load (when the buffer is 16-byte aligned), plus the two neighbours.
__global__ void __launch_bounds__(256) k_ranges(int64_t k_host, const uint32_t *__restrict__ k_dev,
                                                const uint32_t *__restrict__ tile_ids, uint2 *__restrict__ ranges,
                                                uint32_t ntiles)
{
    const int64_t k = k_dev ? (int64_t)*k_dev : k_host;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t k4 = (reinterpret_cast<uintptr_t>(tile_ids) & 15) ? 0 : k / 4;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < k4; q += stride) {
        const uint4 v = reinterpret_cast<const uint4 *>(tile_ids)[q];
        const int64_t i = 4 * q;
        const uint32_t prev = i > 0 ? tile_ids[i - 1] : 0u;
        const uint32_t next = i + 4 < k ? tile_ids[i + 4] : 0u;
        range_ends(i, v.x, prev, v.y, k, ranges, ntiles);
        range_ends(i + 1, v.y, v.x, v.z, k, ranges, ntiles);
        range_ends(i + 2, v.z, v.y, v.w, k, ranges, ntiles);
        range_ends(i + 3, v.w, v.z, next, k, ranges, ntiles);
    }
    for (int64_t i = 4 * k4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride)
        range_ends(i, tile_ids[i], i > 0 ? tile_ids[i - 1] : 0u, i + 1 < k ? tile_ids[i + 1] : 0u, k, ranges, ntiles);
}

// total of the tile counts (the pair count K), one atomic per CTA (all of
// them land on one address). Summed in 64 bits: a scene whose counts add up
// past 2^32 must be reported as over capacity, not wrap to a small count.
__global__ void __launch_bounds__(256) k_sum_u64(const uint32_t *__restrict__ v, int64_t n,
                                                 unsigned long long *__restrict__ total)
{
    __shared__ unsigned long long s_w[8];
    unsigned long long acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) acc += v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned long long x = threadIdx.x < 8 ? s_w[threadIdx.x] : 0ull;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (threadIdx.x == 0 && x) atomicAdd(total, x);
    }
}

}  // namespace

void launch_pair_total(int64_t n, const uint32_t *tt, uint64_t *total, cudaStream_t s)
{
    cudaMemsetAsync(total, 0, sizeof(uint64_t), s);
    if (n <= 0) return;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 4);
    k_sum_u64<<<blocks, 256, 0, s>>>(tt, n, reinterpret_cast<unsigned long long *>(total));
    count_launch();
}

void launch_count_scan(int64_t n, const uint32_t *order, const uint32_t *tt, uint32_t *offsets, uint32_t *sums,
                       uint32_t *total, cudaStream_t s)
{
    const int nchunks = (int)((n + kScanChunk - 1) / kScanChunk);
    if (n <= 0) {
        cudaMemsetAsync(total, 0, sizeof(uint32_t), s);
        return;
    }
    k_scan_reduce<<<nchunks, kScanThreads, 0, s>>>(n, order, tt, sums);
    count_launch();
    // up to 1024 chunks each chunk adds up its predecessors' sums itself
    const int own = nchunks <= 1024;
    if (!own) {
        k_scan_top<<<1, kScanThreads, 0, s>>>(nchunks, sums, total);
        count_launch();
    }
    k_scan_down<<<nchunks, kScanThreads, 0, s>>>(n, order, tt, sums, offsets, own, total);
    count_launch();
}

void launch_emit(int64_t n, const uint32_t *order, const uint32_t *offsets, const uint32_t *tt, const uint2 *rect,
                 const TileGeom &tg, uint32_t *tile_ids, uint32_t *gauss_ids, uint64_t capacity, uint32_t *status,
                 cudaStream_t s)
{
    if (n <= 0) return;
    k_emit<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, order, offsets, tt, rect, tg.tx, tile_ids, gauss_ids, capacity,
                                                       status);
    count_launch();
}

void launch_ranges(int64_t k_host, const uint32_t *k_dev, const uint32_t *tile_ids, uint2 *ranges, int ntiles, cudaStream_t s)
{
    cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)ntiles, s);
    if (k_host <= 0) return;
    const int blocks = (int)std::min<int64_t>((k_host / 4 + 255) / 256 + 1, 148 * 16);
    k_ranges<<<blocks, 256, 0, s>>>(k_host, k_dev, tile_ids, ranges, (uint32_t)ntiles);
    count_launch();
}

}  // namespace splash
