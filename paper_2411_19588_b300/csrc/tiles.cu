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

// per chunk: exclusive offsets of each depth-ranked Gaussian's pairs
__global__ void __launch_bounds__(kScanThreads) k_scan_down(int64_t n, const uint32_t *__restrict__ order,
                                                          const uint32_t *__restrict__ tt, const uint32_t *__restrict__ sums,
                                                          uint32_t *__restrict__ offsets)
{
    __shared__ uint32_t s_w[kScanThreads / 32];
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
    uint32_t run = sums[blockIdx.x] + block_exclusive_scan(acc, s_w, &tot);
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        const int64_t i = base + j;
        if (i < n) offsets[i] = run;
        run += c[j];
    }
}

__global__ void __launch_bounds__(256) k_emit(int64_t n, const uint32_t *__restrict__ order, const uint32_t *__restrict__ offsets,
                                              const uint32_t *__restrict__ tt, const uint2 *__restrict__ rect, int tiles_x,
                                              uint32_t *__restrict__ tile_ids, uint32_t *__restrict__ gauss_ids,
                                              uint64_t capacity, uint32_t *__restrict__ status)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint32_t g = order[r];
    const uint64_t cnt = tt[g];
    if (cnt == 0) return;  // culled or off-image
    const uint2 rc = rect[g];
    const uint32_t tx0 = rc.x & 0xffffu, tx1 = rc.x >> 16, ty0 = rc.y & 0xffffu, ty1 = rc.y >> 16;
    uint64_t off = offsets[r];
    if (off + cnt > capacity) {
        atomicOr(status, kStatusCapacity);
        return;
    }
    for (uint32_t ty = ty0; ty <= ty1; ty++)
        for (uint32_t tx = tx0; tx <= tx1; tx++) {
            tile_ids[off] = ty * (uint32_t)tiles_x + tx;
            gauss_ids[off] = g;
            ++off;
        }
}

__global__ void __launch_bounds__(256) k_ranges(int64_t k_host, const uint32_t *__restrict__ k_dev,
                                                const uint32_t *__restrict__ tile_ids, uint2 *__restrict__ ranges,
                                                uint32_t ntiles)
{
    const int64_t k = k_dev ? (int64_t)*k_dev : k_host;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = tile_ids[i];
        if (t >= ntiles) continue;  // only after a capacity overflow (reported through the status word)
        if (i == 0 || tile_ids[i - 1] != t) ranges[t].x = (uint32_t)i;
        if (i == k - 1 || tile_ids[i + 1] != t) ranges[t].y = (uint32_t)(i + 1);
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
    k_scan_reduce<<<nchunks, kScanThreads, 0, s>>>(n, order, tt, sums);
    count_launch();
    k_scan_top<<<1, kScanThreads, 0, s>>>(nchunks, sums, total);
    count_launch();
    k_scan_down<<<nchunks, kScanThreads, 0, s>>>(n, order, tt, sums, offsets);
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
    const int blocks = (int)std::min<int64_t>((k_host + 255) / 256, 148 * 32);
    k_ranges<<<blocks, 256, 0, s>>>(k_host, k_dev, tile_ids, ranges, (uint32_t)ntiles);
    count_launch();
}

}  // namespace splash
