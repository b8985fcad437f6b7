// Stable LSD radix sort of (uint32 key, uint32 value) pairs, onesweep form:
// one kernel reads all keys once to build the digit histograms of every
// pass; then one kernel per digit (8 bits, or 9 where that saves a pass)
// ranks a partition of 256 x ITEMS keys in shared memory, learns its global
// offset by decoupled look-back over the partitions before it, and scatters.
// Each pass reads and writes every pair once (16 B per pair per pass).
//
// The rasterizer needs the per-tile lists ordered by depth (Sec. III-A: the
// Gaussians of a pixel are composited in increasing depth). It sorts the
// Gaussians by FP32 depth bits once (minus the bits of z_near: 26
// significant bits for (0.2, 20] m, 3 passes of 9/9/8 bits) and then the
// (tile, Gaussian) pairs emitted in that order by tile index only
// (ceil(log2 tiles) bits); stability makes the result identical to one
// sort of 64-bit (tile << 32 | depth bits) keys emitted in index order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "internal.cuh"

namespace splash {
namespace {

constexpr uint32_t kFlagAgg = 1u << 30;  // partition aggregate published
constexpr uint32_t kFlagInc = 2u << 30;  // inclusive prefix published
constexpr uint32_t kValMask = (1u << 30) - 1u;
constexpr int kWarps = kSortThreads / 32;

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p) { return *reinterpret_cast<const volatile uint32_t *>(p); }
__device__ __forceinline__ void st_volatile(uint32_t *p, uint32_t v) { *reinterpret_cast<volatile uint32_t *>(p) = v; }

// exclusive scan of one pass's r <= 512 digit counts by a 256-thread CTA,
// two consecutive digits per thread (the counts were added by other CTAs'
// atomics: read from L2, not L1)
__device__ __forceinline__ void scan_digits(uint32_t *h, int r, uint32_t *s_w)
{
    const int t = threadIdx.x;
    const uint32_t v0 = 2 * t < r ? ld_volatile(h + 2 * t) : 0u;
    const uint32_t v1 = 2 * t + 1 < r ? ld_volatile(h + 2 * t + 1) : 0u;
    const uint32_t v = v0 + v1;
    const int lane = t & 31, w = t >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    uint32_t base = 0;
    for (int i = 0; i < w; i++) base += s_w[i];
    base += x - v;
    if (2 * t < r) h[2 * t] = base;
    if (2 * t + 1 < r) h[2 * t + 1] = base + v0;
    __syncthreads();
}

// Digit histograms of every pass. The last CTA to finish (a ticket taken
// after its counts are flushed and fenced; nothing waits) turns them into
// the per-pass exclusive digit offsets.
__global__ void __launch_bounds__(256) k_hist(const uint32_t *__restrict__ keys, int64_t n_host,
                                              const uint32_t *__restrict__ n_dev, DigitPlan plan,
                                              uint32_t *__restrict__ hist, uint32_t *__restrict__ done)
{
    pdl_enter();
    __shared__ uint32_t s[4][kRadixMax];
    const int passes = plan.passes;
    for (int e = threadIdx.x; e < 4 * kRadixMax; e += blockDim.x) (&s[0][0])[e] = 0u;
    __syncthreads();
    uint32_t pmask[4];
    int pshift[4];
    for (int p = 0; p < 4; p++) {
        pmask[p] = p < passes ? (1u << plan.width[p]) - 1u : 0u;
        pshift[p] = p < passes ? plan.shift[p] : 0;
    }
    const int64_t n = n_dev ? (int64_t)*n_dev : n_host;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // 16-byte loads only from a 16-byte-aligned base; otherwise all scalar
    const int64_t n4 = (reinterpret_cast<uintptr_t>(keys) & 15) ? 0 : (n >> 2);
    const uint4 *k4 = reinterpret_cast<const uint4 *>(keys);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const uint4 v = k4[i];
        const uint32_t kk[4] = {v.x, v.y, v.z, v.w};
        for (int p = 0; p < passes; p++)
#pragma unroll
            for (int q = 0; q < 4; q++) atomicAdd(&s[p][(kk[q] >> pshift[p]) & pmask[p]], 1u);
    }
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t k = keys[i];
        for (int p = 0; p < passes; p++) atomicAdd(&s[p][(k >> pshift[p]) & pmask[p]], 1u);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < passes * kRadixMax; e += blockDim.x) {
        const uint32_t c = (&s[0][0])[e];
        if (c) atomicAdd(&hist[e], c);
    }
    __threadfence();
    __shared__ uint32_t s_last;
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;  // uniform over the CTA
    __threadfence();
    __shared__ uint32_t s_w[256 / 32];
    for (int p = 0; p < passes; p++) scan_digits(hist + p * kRadixMax, 1 << plan.width[p], s_w);
}

// BITS: the digit width of this pass (its number of ballots per key);
// ITEMS: keys per thread (the partition is kSortThreads * ITEMS keys, staged
// for the scatter in dynamic shared memory)
template <int BITS, int ITEMS>
__global__ void __launch_bounds__(kSortThreads) k_onesweep(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, int64_t n_host, const uint32_t *__restrict__ n_dev, int shift, uint32_t mask,
    const uint32_t *__restrict__ goff, uint32_t *__restrict__ lookback, uint32_t *__restrict__ counter,
    uint32_t *__restrict__ status, int spin_limit, uint32_t stall_part)
{
    pdl_enter();
    // digits per thread in the per-digit steps: RA = max(256, 2^BITS) table entries
    constexpr int RA = (1 << BITS) > kSortThreads ? (1 << BITS) : kSortThreads;
    constexpr int DPT = RA / kSortThreads;
    __shared__ uint32_t s_whist[kWarps][RA];  // per-warp digit counts, then warp offsets
    __shared__ uint32_t s_doff[RA];           // block-local exclusive digit offsets
    __shared__ uint32_t s_gbase[RA];          // global position of each digit's first key
    __shared__ uint32_t s_wsum[kWarps];
    __shared__ uint32_t s_part;
    extern __shared__ uint32_t s_stage[];
    constexpr int kTile = kSortThreads * ITEMS;
    uint32_t *s_keys = s_stage, *s_vals = s_stage + kTile;

    if (threadIdx.x == 0) s_part = atomicAdd(counter, 1u);  // partitions start in ticket order
    for (int e = threadIdx.x; e < kWarps * RA; e += kSortThreads) (&s_whist[0][0])[e] = 0u;
    __syncthreads();
    const uint32_t part = s_part;
    const int64_t n = n_dev ? (int64_t)*n_dev : n_host;
    const int64_t base = (int64_t)part * kTile;
    if (base >= n) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t wbase = base + (int64_t)warp * 32 * ITEMS;
    const uint32_t lt = (1u << lane) - 1u;

    // warp-striped loads: item j of lane l is key wbase + 32 j + l (input order)
    uint32_t k[ITEMS], v[ITEMS], rank[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        const int64_t idx = wbase + 32 * j + lane;
        const bool ok = idx < n;
        k[j] = ok ? kin[idx] : 0xffffffffu;  // past the end: largest digit, ranked last
        v[j] = ok ? (vin ? vin[idx] : (uint32_t)idx) : 0u;
    }
    // stable rank within the warp: lanes with equal digits, from one ballot per digit bit
    uint32_t *wh = s_whist[warp];
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        const uint32_t d = (k[j] >> shift) & mask;
        uint32_t peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < BITS; b++) {
            const uint32_t bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bal : ~bal;
        }
        const uint32_t old = wh[d];  // every peer reads the same word (a broadcast)
        __syncwarp();
        rank[j] = old + __popc(peers & lt);
        if ((peers >> lane) == 1u) wh[d] = rank[j] + 1u;  // the last peer: old + the peer count
        __syncwarp();
    }
    __syncthreads();

    // per digit (DPT per thread): warp offsets, block totals and their
    // block-wide exclusive scan
    uint32_t carry = 0;
#pragma unroll
    for (int i = 0; i < DPT; i++) {
        const uint32_t d0 = threadIdx.x + i * kSortThreads;
        uint32_t total = 0;
#pragma unroll
        for (int w = 0; w < kWarps; w++) {
            const uint32_t c = s_whist[w][d0];
            s_whist[w][d0] = total;
            total += c;
        }
        uint32_t x = total;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wsum[warp] = x;
        __syncthreads();
        uint32_t wpre = 0, all = 0;
#pragma unroll
        for (int w = 0; w < kWarps; w++) {
            wpre += w < warp ? s_wsum[w] : 0u;
            all += s_wsum[w];
        }
        s_doff[d0] = carry + wpre + x - total;
        carry += all;
        __syncthreads();  // s_wsum is reused by the next digit
        // decoupled look-back for this digit (digits the pass cannot produce take no part:
        // every partition of the pass skips the same ones)
        uint32_t *lb = lookback + (int64_t)part * RA + d0;
        uint32_t excl = 0;
        const bool publish = stall_part == 0u || part != stall_part;  // test hook: a partition that never reports
        if (d0 >= (1u << BITS)) {
            // no key of this pass has digit d0
        } else if (part == 0) {
            st_volatile(lb, kFlagInc | total);
        } else {
            if (publish) st_volatile(lb, kFlagAgg | total);
            int64_t p = (int64_t)part - 1;
            int spins = 0;
            while (true) {
                const uint32_t w = ld_volatile(lookback + p * RA + d0);
                const uint32_t flag = w & ~kValMask;
                if (flag == 0u) {
                    if (++spins > spin_limit) {  // give up: report, keep offsets in range
                        atomicOr(status, kStatusTimeout);
                        break;
                    }
                    continue;
                }
                excl += w & kValMask;
                if (flag == kFlagInc || p == 0) break;
                --p;
            }
            if (publish) st_volatile(lb, kFlagInc | (excl + total));
        }
        if (d0 < (1u << BITS)) s_gbase[d0] = goff[d0] + excl;
    }
    __syncthreads();

    // scatter into shared memory in block-sorted order
#pragma unroll
    for (int j = 0; j < ITEMS; j++) {
        const uint32_t d = (k[j] >> shift) & mask;
        const uint32_t slot = s_doff[d] + s_whist[warp][d] + rank[j];
        s_keys[slot] = k[j];
        s_vals[slot] = v[j];
    }
    __syncthreads();
    // runs of equal digits go to consecutive global addresses
    const int nvalid = (int)min((int64_t)kTile, n - base);
    for (int s = threadIdx.x; s < nvalid; s += kSortThreads) {
        const uint32_t kk = s_keys[s];
        const uint32_t d = (kk >> shift) & mask;
        const uint32_t dst = s_gbase[d] + (uint32_t)s - s_doff[d];
        kout[dst] = kk;
        vout[dst] = s_vals[s];
    }
}

__global__ void k_iota_copy(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
                            uint32_t *__restrict__ vout, int64_t n_host, const uint32_t *__restrict__ n_dev)
{
    pdl_enter();
    const int64_t n = n_dev ? (int64_t)*n_dev : n_host;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        kout[i] = kin[i];
        vout[i] = vin ? vin[i] : (uint32_t)i;
    }
}

}  // namespace

DigitPlan digit_plan(int bits)
{
    DigitPlan pl{};
    if (bits <= 0) return pl;
    const int p8 = (bits + 7) / 8, p9 = (bits + kRadixBitsMax - 1) / kRadixBitsMax;
    if (p9 < p8) {
        // spread the bits evenly: the first (bits % passes) passes get one more
        pl.passes = p9;
        for (int p = 0, sh = 0; p < p9; p++) {
            pl.width[p] = bits / p9 + (p < bits % p9 ? 1 : 0);
            pl.shift[p] = sh;
            sh += pl.width[p];
        }
    } else {
        pl.passes = p8;
        for (int p = 0; p < p8; p++) {
            pl.width[p] = std::min(kRadixBits, bits - kRadixBits * p);
            pl.shift[p] = kRadixBits * p;
        }
    }
    return pl;
}

int depth_key_bits(float z_near, float z_far)
{
    uint32_t a, b;
    std::memcpy(&a, &z_near, 4);
    std::memcpy(&b, &z_far, 4);
    const uint32_t span = b > a ? b - a : 0xffffffffu;
    int bits = 0;
    while (bits < 32 && (span >> bits) != 0) bits++;
    return std::max(bits, 1);
}

size_t sort_scratch_bytes(int64_t n_max)
{
    const int64_t parts = (n_max + kSortTile - 1) / kSortTile + 1;
    return sizeof(uint32_t) * (size_t)(4 * kRadixMax + 64 + kLookbackPerPart * parts);
}

void sort_scratch_carve(void *base, int64_t n_max, SortScratch *s)
{
    const int64_t parts = (n_max + kSortTile - 1) / kSortTile + 1;
    uint32_t *p = static_cast<uint32_t *>(base);
    s->hist = p;
    s->counters = p + 4 * kRadixMax;
    s->lookback = p + 4 * kRadixMax + 64;
    s->max_parts = parts;
}

namespace {

using OnesweepFn = void (*)(const uint32_t *, const uint32_t *, uint32_t *, uint32_t *, int64_t, const uint32_t *, int,
                           uint32_t, const uint32_t *, uint32_t *, uint32_t *, uint32_t *, int, uint32_t);

template <int ITEMS>
OnesweepFn onesweep_for(int pbits)
{
    switch (pbits) {
    case 1: return k_onesweep<1, ITEMS>;
    case 2: return k_onesweep<2, ITEMS>;
    case 3: return k_onesweep<3, ITEMS>;
    case 4: return k_onesweep<4, ITEMS>;
    case 5: return k_onesweep<5, ITEMS>;
    case 6: return k_onesweep<6, ITEMS>;
    case 7: return k_onesweep<7, ITEMS>;
    case 8: return k_onesweep<8, ITEMS>;
    default: return k_onesweep<9, ITEMS>;
    }
}

// the partition's key and value staging (dynamic shared memory)
OnesweepFn onesweep_kernel(int pbits, int items, size_t *smem)
{
    *smem = sizeof(uint32_t) * 2 * (size_t)kSortThreads * (size_t)items;
    return items == kDepthSortItems ? onesweep_for<kDepthSortItems>(pbits) : onesweep_for<kSortItems>(pbits);
}

// lookback entries per partition of a pass of this width
int lookback_stride(int pbits) { return std::max(kSortThreads, 1 << pbits); }

}  // namespace

cudaError_t sort_prepare_device()
{
    // with its static arrays the wide form passes the default 48 KB window
    const int smem = (int)(sizeof(uint32_t) * 2 * (size_t)kSortThreads * (size_t)kDepthSortItems);
    for (int pbits = 1; pbits <= kRadixBitsMax; pbits++) {
        for (const OnesweepFn f : {onesweep_for<kDepthSortItems>(pbits), onesweep_for<kSortItems>(pbits)}) {
            const cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(f),
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

int sort_pairs(const uint32_t *keys_in, const uint32_t *vals_in, uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1,
               int64_t n_host, const uint32_t *n_dev, int bits, const SortScratch &s, uint32_t *status, int spin_limit,
               int stall_part, cudaStream_t stream, int items)
{
    if (n_host <= 0) return 0;
    const DigitPlan plan = digit_plan(bits);
    const int passes = plan.passes;
    if (passes == 0) {
        const int blocks = (int)std::min<int64_t>((n_host + 255) / 256, 148 * 16);
        launch_pdl(k_iota_copy, blocks, 256, 0, stream, keys_in, vals_in, k0, v0, n_host, n_dev);
        count_launch();
        return 0;
    }
    if (items != kDepthSortItems) items = kSortItems;
    const int64_t tile = (int64_t)kSortThreads * items;
    const int64_t parts = (n_host + tile - 1) / tile;  // at most the scratch's kSortTile-sized count
    // histograms, tickets and the look-back flags of every pass (one block of
    // parts x stride words per pass) are contiguous: one memset clears them
    size_t lb_words = 0;
    for (int p = 0; p < passes; p++) lb_words += (size_t)parts * lookback_stride(plan.width[p]);
    cudaMemsetAsync(s.hist, 0, sizeof(uint32_t) * (size_t)(s.lookback - s.hist) + sizeof(uint32_t) * lb_words, stream);
    // every CTA flushes its shared counters with global atomics onto the same
    // addresses: 4 CTAs per SM keeps that contention below the cost of reading
    const int hblocks = (int)std::min<int64_t>((n_host / 4 + 255) / 256 + 1, 148 * 4);
    launch_pdl(k_hist, hblocks, 256, 0, stream, keys_in, n_host, n_dev, plan, s.hist, s.counters + 4);  // zeroed above
    count_launch();
    const uint32_t *ki = keys_in, *vi = vals_in;
    uint32_t *lb = s.lookback;
    for (int p = 0; p < passes; p++) {
        uint32_t *ko = (p & 1) ? k1 : k0, *vo = (p & 1) ? v1 : v0;
        const int pbits = plan.width[p];
        const uint32_t mask = (1u << pbits) - 1u;
        size_t smem = 0;
        const OnesweepFn kern = onesweep_kernel(pbits, items, &smem);
        launch_pdl(kern, (unsigned)parts, kSortThreads, smem, stream, ki, vi, ko, vo, n_host, n_dev, plan.shift[p], mask,
                                                              s.hist + kRadixMax * p, lb, s.counters + p, status,
                                                              spin_limit, (uint32_t)stall_part);
        count_launch();
        lb += (size_t)parts * lookback_stride(pbits);
        ki = ko;
        vi = vo;
    }
    return (passes - 1) & 1;
}

}  // namespace splash
