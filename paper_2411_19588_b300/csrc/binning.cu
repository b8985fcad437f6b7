// Two-level tile binning (Sec. III-A, "Tiles": every Gaussian is listed in
// each tile its 3-sigma bounding box covers, each list in increasing depth).
//
// The Gaussians, already in depth order, are binned into super-tiles of
// kSuperW x kSuperH tiles first: one stable radix pass over the (Gaussian,
// super-tile) entries, about a quarter as many as the (tile, Gaussian) pairs
// on the training views, each entry carrying the Gaussian's tile rectangle
// clipped to that super-tile. Tile t's list is then the subsequence of its
// super-tile's list whose rectangle covers t. Each super-tile's list is cut
// into chunks of kChunk entries (one warp each): the per-(chunk, tile)
// counts give every chunk's offset within each tile's list and, summed and
// scanned in tile order, every list's start; a scatter pass then writes each
// entry into the lists of the tiles it covers, in order. The lists land in
// the same compact tile-major layout, with the same ranges, as a stable sort
// of the (tile, Gaussian) pairs by tile.
//   k_pair_totals    -- K (pairs), K_s (super entries), per-Gaussian super counts
//   k_gather_counts  -- super counts in depth order, sums per emit block
//   k_block_prefix   -- exclusive offsets of the emit blocks, total K_s
//   k_emit_super     -- (super-tile | clipped rectangle, Gaussian) entries in depth order
//   (the super-tile sort: sort.cu; its list ranges are its digit offsets, or
//   come from tiles.cu when the sort takes more than one pass)
//   k_chunk_map      -- super-tile list ranges; first chunk of every super-tile
//   k_super_count    -- per chunk and tile: entries covering the tile
//   k_super_prefix   -- chunk offsets within each tile's list; tile counts
//   k_tile_scan      -- tile ranges (exclusive scan of the counts)
//   k_super_scatter  -- the tile lists
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.cuh"

namespace splash {
namespace {

constexpr int kCountScanThreads = 1024;

__device__ __forceinline__ uint32_t super_count(uint2 rc)
{
    const uint32_t tx0 = rc.x & 0xffffu, tx1 = rc.x >> 16, ty0 = rc.y & 0xffffu, ty1 = rc.y >> 16;
    return (tx1 / kSuperW - tx0 / kSuperW + 1) * (ty1 / kSuperH - ty0 / kSuperH + 1);
}

__device__ __forceinline__ ulonglong2 block_sum2(ulonglong2 x, ulonglong2 *s_w)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x.x += __shfl_down_sync(0xffffffffu, x.x, o);
        x.y += __shfl_down_sync(0xffffffffu, x.y, o);
    }
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = x;
    __syncthreads();
    ulonglong2 t = make_ulonglong2(0ull, 0ull);
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            t.x += s_w[w].x;
            t.y += s_w[w].y;
        }
    return t;  // valid in thread 0
}

// K = sum of the tile counts and K_s = sum of the super-tile counts, in 64
// bits (a total past 2^32 must be reported, not wrap); sc[g] = Gaussian g's
// super-tile count. One partial per CTA; the last CTA to finish adds them up
// in CTA order, writes the totals (and, into mapped host memory, the status
// word, K and K_s) and puts the ticket back to zero.
__global__ void __launch_bounds__(256) k_pair_totals(int64_t n, const uint32_t *__restrict__ tt,
                                                     const uint2 *__restrict__ rect, uint32_t *__restrict__ sc,
                                                     ulonglong2 *__restrict__ part, uint32_t *__restrict__ ticket,
                                                     unsigned long long *__restrict__ host,
                                                     const uint32_t *__restrict__ status)
{
    pdl_enter();
    __shared__ ulonglong2 s_w[8];
    __shared__ uint32_t s_last;
    ulonglong2 acc = make_ulonglong2(0ull, 0ull);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = tt[i];
        const uint32_t s = c ? super_count(rect[i]) : 0u;
        sc[i] = s;
        acc.x += c;
        acc.y += s;
    }
    acc = block_sum2(acc, s_w);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = acc;
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;  // uniform over the CTA
    __threadfence();
    ulonglong2 x = make_ulonglong2(0ull, 0ull);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const volatile unsigned long long *p = reinterpret_cast<const volatile unsigned long long *>(part + b);
        x.x += p[0];
        x.y += p[1];
    }
    __syncthreads();  // s_w is reused
    x = block_sum2(x, s_w);
    if (threadIdx.x == 0) {
        *ticket = 0u;
        if (host) {
            host[0] = *reinterpret_cast<const volatile uint32_t *>(status);
            host[1] = x.x;
            host[2] = x.y;
            __threadfence_system();
        }
    }
}

// The emit's offsets come in two small steps, without an offset per
// Gaussian: k_gather_counts copies the super-tile counts into depth order
// (coalesced reads for the emit) and sums them per block of kEmitBlock
// ranks; k_block_prefix (one CTA) turns the block sums into exclusive block
// offsets and the total. Each emit CTA then scans its own ranks.
constexpr int kEmitBlock = 256;
constexpr int kPrefixThreads = 1024, kPrefixItems = 8;

__global__ void __launch_bounds__(kEmitBlock) k_gather_counts(int64_t n, const uint32_t *__restrict__ order,
                                                              const uint32_t *__restrict__ sc, uint32_t *__restrict__ scs,
                                                              uint32_t *__restrict__ block_sum)
{
    pdl_enter();
    __shared__ uint32_t s_w[kEmitBlock / 32];
    const int64_t r = (int64_t)blockIdx.x * kEmitBlock + threadIdx.x;
    uint32_t c = 0;
    if (r < n) {
        c = sc[order[r]];
        scs[r] = c;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
#pragma unroll
        for (int w = 0; w < kEmitBlock / 32; w++) t += s_w[w];
        block_sum[blockIdx.x] = t;
    }
}

// exclusive scan of nb block sums in place (rounds of kPrefixThreads x
// kPrefixItems, each thread a run of kPrefixItems), the total to *total
__global__ void __launch_bounds__(kPrefixThreads) k_block_prefix(int64_t nb, uint32_t *__restrict__ sums,
                                                                 uint32_t *__restrict__ total)
{
    pdl_enter();
    __shared__ uint32_t s_w[kPrefixThreads / 32];
    __shared__ uint32_t s_round;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t carry = 0;
    for (int64_t base = 0; base < nb; base += (int64_t)kPrefixThreads * kPrefixItems) {
        const int64_t i0 = base + (int64_t)tid * kPrefixItems;
        uint32_t v[kPrefixItems], acc = 0;
#pragma unroll
        for (int j = 0; j < kPrefixItems; j++) {
            v[j] = i0 + j < nb ? sums[i0 + j] : 0u;
            acc += v[j];
        }
        uint32_t x = acc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = s_w[lane];
            uint32_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            s_w[lane] = wi - w;
            if (lane == 31) s_round = wi;
        }
        __syncthreads();
        uint32_t run = carry + s_w[warp] + x - acc;
#pragma unroll
        for (int j = 0; j < kPrefixItems; j++) {
            if (i0 + j < nb) sums[i0 + j] = run;
            run += v[j];
        }
        carry += s_round;
        __syncthreads();  // s_w and s_round are rewritten by the next round
    }
    if (tid == 0) *total = carry;
}

// One warp per 32 consecutive depth-ordered Gaussians writes their
// super-tile entries (row-major over each Gaussian's super-tile rectangle),
// with coalesced stores as k_emit does for tile pairs: output slot s belongs
// to the last lane whose run starts at or before s. The CTA's first entry is
// its block offset; each warp adds the counts of the warps before it. Key:
// the super-tile index in the low `sbits` bits, above it the Gaussian's tile
// rectangle clipped to that super-tile (x0, x1 in 3 bits each, y0, y1 in 2
// bits each). Entries at or past `capacity` are not written (the status
// word records it), so every entry below it is valid.
__global__ void __launch_bounds__(kEmitBlock) k_emit_super(int64_t n, const uint32_t *__restrict__ order,
                                                           const uint32_t *__restrict__ scs,
                                                           const uint32_t *__restrict__ block_pre,
                                                           const uint2 *__restrict__ rect, int nsx, int sbits,
                                                           uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                                           uint64_t capacity, uint32_t *__restrict__ status)
{
    pdl_enter();
    constexpr uint32_t kFull = 0xffffffffu;
    __shared__ uint32_t s_w[kEmitBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r = (int64_t)blockIdx.x * kEmitBlock + threadIdx.x;
    uint32_t g = 0, cnt = 0, rx = 0, ry = 0;
    if (r < n) {
        g = order[r];
        cnt = scs[r];
        if (cnt) {
            const uint2 rc = rect[g];
            rx = rc.x;
            ry = rc.y;
        }
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[warp] = incl;
    uint64_t wpre = block_pre[blockIdx.x];
    __syncthreads();
    for (int w = 0; w < warp; w++) wpre += s_w[w];
    const uint32_t loc = incl - cnt;
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (wpre + total > capacity && lane == 0) atomicOr(status, kStatusCapacity);
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t s = base + lane;
        int j = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t lj = __shfl_sync(kFull, loc, j + step);
            if (lj <= s) j += step;
        }
        const uint32_t og = __shfl_sync(kFull, g, j), orx = __shfl_sync(kFull, rx, j), ory = __shfl_sync(kFull, ry, j);
        const uint32_t oloc = __shfl_sync(kFull, loc, j);
        const uint64_t slot = wpre + s;
        if (s < total && slot < capacity) {
            const uint32_t tx0 = orx & 0xffffu, tx1 = orx >> 16, ty0 = ory & 0xffffu, ty1 = ory >> 16;
            const uint32_t sx0 = tx0 / kSuperW, sx1 = tx1 / kSuperW, sy0 = ty0 / kSuperH;
            const uint32_t k = s - oloc, sw = sx1 - sx0 + 1, dy = k / sw, dx = k - dy * sw;
            const uint32_t sxi = sx0 + dx, syi = sy0 + dy;
            const uint32_t bx = sxi * kSuperW, by = syi * kSuperH;
            const uint32_t lx0 = max(tx0, bx) - bx, lx1 = min(tx1, bx + kSuperW - 1) - bx;
            const uint32_t ly0 = max(ty0, by) - by, ly1 = min(ty1, by + kSuperH - 1) - by;
            const uint32_t lr = lx0 | (lx1 << 3) | (ly0 << 6) | (ly1 << 8);
            keys[slot] = (syi * (uint32_t)nsx + sxi) | (lr << sbits);
            vals[slot] = og;
        }
    }
}

// ---- tile lists from the sorted super-tile lists. Each list is cut into
// chunks of kChunk consecutive entries; every entry's clipped rectangle is a
// 32-bit mask over its super-tile's tiles (bit 8 y + x). A count pass takes
// the per-(chunk, tile) counts, a prefix pass turns them into each chunk's
// offset within each tile's list (and the tiles' counts into their ranges),
// and a scatter pass writes every entry into the lists of the tiles it
// covers, in entry order.
constexpr int kChunk = 256;    // entries per chunk (one warp each: 8 groups of 32)
constexpr int kGroups = kChunk / 32;
static_assert(kGroups <= 15, "four count planes");
constexpr int kChunkWarps = 4; // chunks per CTA
constexpr int kRecWords = (kGroups + 2 + 3) / 4 * 4;  // the scatter's per-tile record: masks, position, limit

__device__ __forceinline__ uint32_t tile_mask(uint32_t lr)
{
    const uint32_t lx0 = lr & 7u, lx1 = (lr >> 3) & 7u, ly0 = (lr >> 6) & 3u, ly1 = (lr >> 8) & 3u;
    const uint32_t row = (0xffu >> (7u - lx1)) & (0xffu << lx0);                          // columns lx0..lx1
    const uint32_t rows = (0xffffffffu >> (8u * (3u - ly1))) & (0xffffffffu << (8u * ly0));  // bytes ly0..ly1
    return (row * 0x01010101u) & rows;
}

// Transpose of a 32 x 32 bit matrix held one row per lane (bit c of lane l's
// word = element (l, c)): returns column `lane` (bit l = element (l, lane)).
// Five exchange steps swap ever smaller blocks between lane pairs (the
// recursive block transpose written for a warp).
__device__ __forceinline__ uint32_t warp_transpose(uint32_t w, int lane)
{
    uint32_t m = 0x0000ffffu;
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        const uint32_t p = __shfl_xor_sync(0xffffffffu, w, j);
        w = (lane & j) ? w ^ (((p >> j) ^ w) & m) : w ^ ((((w >> j) ^ p) & m) << j);
        m ^= m << (j >> 1);
    }
    return w;
}

// the super-tile whose chunks contain chunk c: the last s with cb[s] <= c
__device__ __forceinline__ int chunk_super(const uint32_t *__restrict__ cb, int nsuper, uint32_t c)
{
    int lo = 0, hi = nsuper;  // cb[lo] <= c < cb[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (cb[mid] <= c) lo = mid;
        else hi = mid;
    }
    return lo;
}

// one CTA: cb[s] = first chunk of super-tile s (exclusive scan of the chunk
// counts), cb[nsuper] = all chunks. With `off` (the one-pass super-tile
// sort's exclusive digit offsets: the digit is the super-tile index) it first
// writes every super-tile's list range, [off[s], off[s + 1]), the last one
// ending at the sorted entry count.
__global__ void __launch_bounds__(1024) k_chunk_map(uint2 *__restrict__ sranges, const uint32_t *__restrict__ off,
                                                    int64_t total_host, const uint32_t *__restrict__ total_dev,
                                                    int nsuper, uint32_t *__restrict__ cb)
{
    pdl_enter();
    __shared__ uint32_t s_w[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (nsuper + 1023) / 1024;
    const int s0 = min(nsuper, tid * per), s1 = min(nsuper, s0 + per);
    uint32_t local = 0;
    if (off) {
        const uint32_t total = total_dev ? *total_dev : (uint32_t)total_host;
        for (int q = s0; q < s1; q++) {
            const uint2 r = make_uint2(off[q], q + 1 < nsuper ? off[q + 1] : total);
            sranges[q] = r;
            local += (r.y - r.x + kChunk - 1) / kChunk;
        }
    } else {
        for (int q = s0; q < s1; q++) {
            const uint2 r = sranges[q];
            local += (r.y - r.x + kChunk - 1) / kChunk;
        }
    }
    uint32_t x = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    uint32_t base = 0;
    for (int w = 0; w < warp; w++) base += s_w[w];
    uint32_t run = base + x - local;
    for (int q = s0; q < s1; q++) {
        const uint2 r = sranges[q];
        cb[q] = run;
        run += (r.y - r.x + kChunk - 1) / kChunk;
    }
    if (tid == 1023) cb[nsuper] = base + x;
}

// One warp per chunk, lane t = tile t of the chunk's super-tile. The
// chunk's groups of 32 entries are loaded first (one entry per lane and
// group, all loads in flight together) and turned into tile masks.
// cnt[c][t] = the entries covering tile t.
__global__ void __launch_bounds__(kChunkWarps * 32) k_super_count(const uint32_t *__restrict__ skeys,
                                                                  const uint2 *__restrict__ sranges,
                                                                  const uint32_t *__restrict__ cb, int nsuper, int sbits,
                                                                  uint32_t *__restrict__ cnt)
{
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const uint32_t c = blockIdx.x * kChunkWarps + (threadIdx.x >> 5);
    if (c >= cb[nsuper]) return;  // uniform over the warp
    const int s = chunk_super(cb, nsuper, c);
    const uint2 sr = sranges[s];
    const uint32_t beg = sr.x + (c - cb[s]) * kChunk, end = min(beg + kChunk, sr.y);
    uint32_t m[kGroups];
#pragma unroll
    for (int g = 0; g < kGroups; g++) {
        const uint32_t idx = beg + (uint32_t)(g * 32 + lane);
        m[g] = idx < end ? skeys[idx] : 0u;
    }
#pragma unroll
    for (int g = 0; g < kGroups; g++) m[g] = beg + (uint32_t)(g * 32 + lane) < end ? tile_mask(m[g] >> sbits) : 0u;
    // per lane, the count over its groups of each tile bit, bit-sliced into
    // four planes (counts up to 8); the column sums of the planes over the
    // warp's lanes are the tile counts
    uint32_t p0 = 0, p1 = 0, p2 = 0, p3 = 0;
#pragma unroll
    for (int g = 0; g < kGroups; g++) {
        const uint32_t c0 = m[g], c1 = p0 & c0;
        p0 ^= c0;
        const uint32_t c2 = p1 & c1;
        p1 ^= c1;
        const uint32_t c3 = p2 & c2;
        p2 ^= c2;
        p3 ^= c3;
    }
    const uint32_t acc = __popc(warp_transpose(p0, lane)) + 2u * __popc(warp_transpose(p1, lane)) +
                         4u * __popc(warp_transpose(p2, lane)) + 8u * __popc(warp_transpose(p3, lane));
    cnt[(size_t)c * 32 + lane] = acc;
}

// one warp per super-tile, lane = tile: each chunk's count replaced by its
// exclusive prefix over the super-tile's chunks; the totals are the tiles' counts
__global__ void __launch_bounds__(256) k_super_prefix(const uint32_t *__restrict__ cb, int nsuper, int nsx, int tiles_x,
                                                      int tiles_y, uint32_t *__restrict__ cnt,
                                                      uint32_t *__restrict__ tile_count)
{
    pdl_enter();
    const int s = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (s >= nsuper) return;  // uniform over the warp
    const uint32_t c0 = cb[s], c1 = cb[s + 1];
    uint32_t acc = 0;
    for (uint32_t c = c0; c < c1; c += 32) {
        uint32_t v[32];
#pragma unroll
        for (int k = 0; k < 32; k++) v[k] = c + k < c1 ? cnt[(size_t)(c + k) * 32 + lane] : 0u;
#pragma unroll
        for (int k = 0; k < 32; k++)
            if (c + k < c1) {
                cnt[(size_t)(c + k) * 32 + lane] = acc;
                acc += v[k];
            }
    }
    const int sx = s % nsx, sy = s / nsx;
    const int tx = sx * kSuperW + (lane & 7), ty = sy * kSuperH + (lane >> 3);
    if (tx < tiles_x && ty < tiles_y) tile_count[ty * tiles_x + tx] = acc;
}

// one CTA: exclusive scan of the tile counts in tile order: ranges, clamped
// to `cap` slots (a total past it is reported); *total = the pairs
__global__ void __launch_bounds__(kCountScanThreads) k_tile_scan(const uint32_t *__restrict__ tile_count, int ntiles,
                                                                 uint2 *__restrict__ ranges, uint32_t cap,
                                                                 uint32_t *__restrict__ total, uint32_t *__restrict__ status)
{
    pdl_enter();
    __shared__ uint32_t s_w[kCountScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (ntiles + kCountScanThreads - 1) / kCountScanThreads;
    const int t0 = min(ntiles, tid * per), t1 = min(ntiles, t0 + per);
    uint32_t local = 0;
    for (int t = t0; t < t1; t++) local += tile_count[t];
    uint32_t x = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    uint32_t base = 0;
    for (int w = 0; w < warp; w++) base += s_w[w];
    uint32_t run = base + x - local;
    for (int t = t0; t < t1; t++) {
        const uint32_t c = tile_count[t];
        ranges[t] = make_uint2(min(run, cap), min(run + c, cap));
        run += c;
    }
    if (tid == kCountScanThreads - 1) {  // its run ends at the total
        if (total) *total = run;
        if (run > cap) atomicOr(status, kStatusCapacity);
    }
}

// One warp per chunk: its entries (keys and values) are loaded first, one
// per lane and group, and each group's tile masks transposed (lane t then
// holds the lanes covering tile t). Tile by tile, the entries covering the
// tile fill consecutive slots of its list in entry order, from the tile's
// start plus the chunk's offset (k_super_prefix); they are gathered in a
// per-warp shared buffer first, so that each store instruction writes up to
// 32 contiguous slots. A slot past a tile's range is reported and not written.
__global__ void __launch_bounds__(kChunkWarps * 32) k_super_scatter(
    const uint32_t *__restrict__ skeys, const uint32_t *__restrict__ svals, const uint2 *__restrict__ sranges,
    const uint32_t *__restrict__ cb, int nsuper, int nsx, int sbits, int tiles_x, int tiles_y,
    const uint32_t *__restrict__ cnt, const uint2 *__restrict__ ranges, uint32_t *__restrict__ gauss_ids,
    uint32_t *__restrict__ status)
{
    pdl_enter();
    const int lane = threadIdx.x & 31;
    __shared__ uint32_t s_slot[kChunkWarps][kChunk];
    __shared__ __align__(16) uint32_t s_rec[kChunkWarps][32][kRecWords];
    const uint32_t c = blockIdx.x * kChunkWarps + (threadIdx.x >> 5);
    if (c >= cb[nsuper]) return;  // uniform over the warp
    const int s = chunk_super(cb, nsuper, c);
    const uint2 sr = sranges[s];
    const uint32_t beg = sr.x + (c - cb[s]) * kChunk, end = min(beg + kChunk, sr.y);
    const int tx = (s % nsx) * kSuperW + (lane & 7), ty = (s / nsx) * kSuperH + (lane >> 3);
    uint2 rg = make_uint2(0u, 0u);
    if (tx < tiles_x && ty < tiles_y) rg = ranges[ty * tiles_x + tx];
    const uint32_t base = rg.x + cnt[(size_t)c * 32 + lane];
    uint32_t m[kGroups], v[kGroups];
#pragma unroll
    for (int g = 0; g < kGroups; g++) {
        const uint32_t idx = beg + (uint32_t)(g * 32 + lane);
        const bool in = idx < end;
        m[g] = in ? skeys[idx] : 0u;
        v[g] = in ? svals[idx] : 0u;
    }
    // per group, the transpose of the lanes' tile masks: lane t holds the
    // lanes whose entry covers tile t
#pragma unroll
    for (int g = 0; g < kGroups; g++)
        m[g] = warp_transpose(beg + (uint32_t)(g * 32 + lane) < end ? tile_mask(m[g] >> sbits) : 0u, lane);
    // lane t's record for tile t (its masks, list position and limit) goes
    // to shared memory: the tile loop reads it with broadcast 16-byte loads,
    // three per tile instead of ten shuffles (the shuffle rate bounds this loop)
    uint32_t(*rec)[kRecWords] = s_rec[threadIdx.x >> 5];
    {
        uint32_t w[kRecWords];
#pragma unroll
        for (int g = 0; g < kGroups; g++) w[g] = m[g];
        w[kGroups] = base;
        w[kGroups + 1] = rg.y;
#pragma unroll
        for (int q = kGroups + 2; q < kRecWords; q++) w[q] = 0u;
#pragma unroll
        for (int q = 0; q < kRecWords; q += 4)
            *reinterpret_cast<uint4 *>(&rec[lane][q]) = make_uint4(w[q], w[q + 1], w[q + 2], w[q + 3]);
    }
    __syncwarp();
    bool bad = false;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t *buf = s_slot[threadIdx.x >> 5];
    for (int t = 0; t < 32; t++) {
        // the tile's hits in this chunk, in entry order: group g's covering
        // lanes put their values in slots pre_g + rank of the warp's buffer,
        // then the warp stores the slots 32 at a time, contiguously
        uint32_t w[kRecWords];
#pragma unroll
        for (int q = 0; q < kRecWords; q += 4) {
            const uint4 u = *reinterpret_cast<const uint4 *>(&rec[t][q]);
            w[q] = u.x;
            w[q + 1] = u.y;
            w[q + 2] = u.z;
            w[q + 3] = u.w;
        }
        const uint32_t pos = w[kGroups], lim = w[kGroups + 1];
        uint32_t pre = 0;
#pragma unroll
        for (int g = 0; g < kGroups; g++) {
            const uint32_t b = w[g];  // the lanes covering tile t
            if ((b >> lane) & 1u) buf[pre + __popc(b & lt)] = v[g];
            pre += __popc(b);
        }
        __syncwarp();
        for (uint32_t i = lane; i < pre; i += 32) {
            if (pos + i < lim) gauss_ids[pos + i] = buf[i];
            else bad = true;
        }
        __syncwarp();  // the buffer is refilled for the next tile
    }
    if (bad) atomicOr(status, kStatusCapacity);
}

}  // namespace

int super_bits(const TileGeom &tg, int *nsx)
{
    *nsx = (tg.tx + kSuperW - 1) / kSuperW;
    const int64_t ns = (int64_t)*nsx * ((tg.ty + kSuperH - 1) / kSuperH);
    int b = 1;
    while (((int64_t)1 << b) < ns) b++;
    return b;
}

int64_t chunk_bound(int64_t n_super_entries, int nsuper) { return (n_super_entries + kChunk - 1) / kChunk + nsuper; }

size_t binning_scratch_words(int64_t n_super_entries, int nsuper, int ntiles)
{
    return (size_t)nsuper + 1 + 32 * (size_t)chunk_bound(n_super_entries, nsuper) + (size_t)ntiles;
}

BinningScratch binning_scratch_carve(uint32_t *base, int64_t n_super_entries, int nsuper)
{
    BinningScratch bs;
    bs.chunk_base = base;
    bs.chunk_count = base + nsuper + 1;
    bs.tile_count = bs.chunk_count + 32 * chunk_bound(n_super_entries, nsuper);
    return bs;
}

void launch_pair_totals(int64_t n, const uint32_t *tt, const uint2 *rect, uint32_t *sc, void *scratch,
                        uint64_t *host_out, const uint32_t *status, cudaStream_t s)
{
    ulonglong2 *part = static_cast<ulonglong2 *>(scratch);
    uint32_t *ticket = reinterpret_cast<uint32_t *>(part + kPairTotalBlocksMax);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, kPairTotalBlocksMax));
    launch_pdl(k_pair_totals, blocks, 256, 0, s, std::max<int64_t>(n, 0), tt, rect, sc, part, ticket,
               reinterpret_cast<unsigned long long *>(host_out), status);
    count_launch();
}

int64_t emit_blocks(int64_t n) { return (std::max<int64_t>(n, 0) + kEmitBlock - 1) / kEmitBlock; }

void launch_super_scan(int64_t n, const uint32_t *order, const uint32_t *sc, uint32_t *scs, uint32_t *block_pre,
                       uint32_t *total, cudaStream_t s)
{
    const int64_t nb = emit_blocks(n);
    if (nb > 0) {
        launch_pdl(k_gather_counts, (unsigned)nb, kEmitBlock, 0, s, n, order, sc, scs, block_pre);
        count_launch();
    }
    launch_pdl(k_block_prefix, 1, kPrefixThreads, 0, s, nb, block_pre, total);
    count_launch();
}

void launch_emit_super(int64_t n, const uint32_t *order, const uint32_t *scs, const uint32_t *block_pre,
                       const uint2 *rect, int nsx, int sbits, uint32_t *keys, uint32_t *vals, uint64_t capacity,
                       uint32_t *status, cudaStream_t s)
{
    if (n <= 0) return;
    launch_pdl(k_emit_super, (unsigned)emit_blocks(n), kEmitBlock, 0, s, n, order, scs, block_pre, rect, nsx, sbits,
               keys, vals, capacity, status);
    count_launch();
}

void launch_tile_lists(const TileGeom &tg, int nsx, int sbits, int64_t n_super_entries, const uint32_t *skeys,
                       const uint32_t *svals, uint2 *sranges, const BinningScratch &bs, uint2 *ranges,
                       uint32_t *gauss_ids, uint32_t *status, cudaStream_t s, uint32_t cap, uint32_t *total,
                       const uint32_t *digit_off, const uint32_t *n_sorted_dev)
{
    // plain launches: started early behind one another (programmatic launch)
    // these kernels made the forward 0.17 ms slower on the B300
    const int nsuper = nsx * ((tg.ty + kSuperH - 1) / kSuperH), ntiles = tg.tx * tg.ty;
    const unsigned chunks = (unsigned)chunk_bound(n_super_entries, nsuper);
    k_chunk_map<<<1, 1024, 0, s>>>(sranges, digit_off, n_super_entries, n_sorted_dev, nsuper, bs.chunk_base);
    count_launch();
    const unsigned ctas = (chunks + kChunkWarps - 1) / kChunkWarps;
    k_super_count<<<ctas, kChunkWarps * 32, 0, s>>>(skeys, sranges, bs.chunk_base, nsuper, sbits, bs.chunk_count);
    count_launch();
    k_super_prefix<<<(unsigned)(((int64_t)nsuper * 32 + 255) / 256), 256, 0, s>>>(bs.chunk_base, nsuper, nsx, tg.tx,
               tg.ty, bs.chunk_count, bs.tile_count);
    count_launch();
    k_tile_scan<<<1, kCountScanThreads, 0, s>>>(bs.tile_count, ntiles, ranges, cap, total, status);
    count_launch();
    k_super_scatter<<<ctas, kChunkWarps * 32, 0, s>>>(skeys, svals, sranges, bs.chunk_base, nsuper, nsx, sbits,
               tg.tx, tg.ty, bs.chunk_count, ranges, gauss_ids, status);
    count_launch();
}

}  // namespace splash
