// Backscatter estimate behind the L_best prior (Sec. IV-B, Eq. 7-9), after
// the appendix's Alg. 1 ("Estimate Backscatter") and Alg. 2 ("Get
// backscatter by curve fitting"): dark pixels per depth cluster of an
// observed view, their per-interval minima, and a bounded per-channel fit of
// B_inf (1 - exp(-beta_B z)).
//
//   k_bs_resize  -- area-average resize of image + depth (FP64 accumulation,
//                   one rounding to FP32), darkness keys, depth min/max
//   k_bs_cluster -- depth cluster of every pixel, per-block cluster counts
//   k_bs_offsets -- where each (block, cluster) run starts in the partition
//   k_bs_scatter -- stable partition of (darkness key, index) by cluster
//   k_bs_select  -- one block per cluster segment: radix select of the
//                   ceil(p_dark n)-th darkest key, then the kept pixels
//   k_bs_fit     -- one block per channel: interval minima of the kept
//                   pixels (the fit points), then an FP32 residual scan over
//                   beta and two sign scans of the profiled derivative
//   k_bs_prior   -- Eq. 9's lambda_est L_best loss and gradient
//
// The estimate runs once every few hundred training iterations on a
// ~135k-pixel image, so it is latency-bound; its integer decisions (cluster,
// rank, interval, argmin) are all taken on values that are either the exact
// FP32 rounding of an FP64 quantity or FP32 sums in a fixed order, so they do
// not depend on the launch shape.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "host.h"
#include "internal.cuh"

using namespace splash_host;

namespace splash {
namespace {

constexpr int kMaxClusters = 64;                     // edges <= 65
constexpr int kMaxIntervals = SPLASH_BS_MAX_POINTS;  // intervals <= 65
constexpr int kGrid = 1024;                          // FP32 beta scan points

struct BsCounters {      // cleared by one memset per estimate
    uint32_t zmax_bits;  // max over resized depths of the FP32 bits (values >= 0)
    uint32_t zmin_inv;   // max of ~bits, i.e. ~(min bits)
    uint32_t n_dark;
    uint32_t pad;
    uint32_t count[kMaxClusters];  // cluster sizes
    uint32_t start[kMaxClusters];  // segment starts of the cluster-major partition
};

__device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// Lanes of the (full) warp whose `bits`-bit value equals this lane's: one
// ballot per bit (cheaper than match.any on this GPU for a few bits; the
// 11-bit digits of the select use match.any).
__device__ __forceinline__ unsigned peers_of(uint32_t v, int bits)
{
    unsigned peers = 0xffffffffu;
    for (int b = 0; b < bits; b++) {
        const unsigned bal = __ballot_sync(0xffffffffu, (v >> b) & 1u);
        peers &= ((v >> b) & 1u) ? bal : ~bal;
    }
    return peers;
}

__device__ __forceinline__ uint32_t block_max_u32(uint32_t v, uint32_t *s_red)
{
    v = __reduce_max_sync(0xffffffffu, v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    uint32_t r = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) r = max(r, s_red[i]);
    __syncthreads();
    return r;
}

// Output pixel i = (o, p) of the h x w grid averages the source rectangle
// [o H / h, (o+1) H / h) x [p W / w, (p+1) W / w). In units of 1/h of a row,
// output row o is [o H, (o+1) H) and source row r is [r h, (r+1) h), so the
// row weights are integer overlap lengths (columns alike), the weights of a
// cell sum to H W, and every product wx * v is exact in FP64.
__global__ void __launch_bounds__(256) k_bs_resize(const float *__restrict__ img, const float *__restrict__ depth,
                                                   int W, int H, int w, int h, float *__restrict__ out,
                                                   uint32_t *__restrict__ key, BsCounters *__restrict__ cnt)
{
    __shared__ uint32_t s_red[8];
    const int64_t N = (int64_t)h * w;
    const int64_t HW = (int64_t)H * W;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t zbits = 0, zinv = 0;
    if (i < N) {
        const int o = (int)(i / w), p = (int)(i - (int64_t)o * w);
        const int64_t ya = (int64_t)o * H, yb = ya + H;
        const int64_t xa = (int64_t)p * W, xb = xa + W;
        const int r0 = (int)(ya / h), r1 = (int)min64(H, (yb + h - 1) / h);
        const int c0 = (int)(xa / w), c1 = (int)min64(W, (xb + w - 1) / w);
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int r = r0; r < r1; r++) {
            const double wy = (double)(min64(yb, (int64_t)(r + 1) * h) - max64(ya, (int64_t)r * h));
            double row[4] = {0.0, 0.0, 0.0, 0.0};
            const float *src = img + (int64_t)r * W;
            const float *zs = depth + (int64_t)r * W;
            for (int c = c0; c < c1; c++) {
                const double wx =
                    (double)(min64(xb, (int64_t)(c + 1) * w) - max64(xa, (int64_t)c * w));
                row[0] = fma(wx, (double)src[c], row[0]);
                row[1] = fma(wx, (double)src[HW + c], row[1]);
                row[2] = fma(wx, (double)src[2 * HW + c], row[2]);
                row[3] = fma(wx, (double)zs[c], row[3]);
            }
#pragma unroll
            for (int k = 0; k < 4; k++) acc[k] = fma(wy, row[k], acc[k]);
        }
        const double area = (double)H * (double)W;
        float v[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float f = __double2float_rn(acc[k] / area);
            v[k] = f > 0.f ? f : 0.f;  // negatives (and -0) to +0
            out[k * N + i] = v[k];
        }
        key[i] = __float_as_uint(__fadd_rn(__fadd_rn(v[0], v[1]), v[2]));
        zbits = __float_as_uint(v[3]);
        zinv = ~zbits;
    }
    zbits = block_max_u32(zbits, s_red);
    zinv = block_max_u32(zinv, s_red);
    if (threadIdx.x == 0) {
        atomicMax(&cnt->zmax_bits, zbits);
        atomicMax(&cnt->zmin_inv, zinv);
    }
}

// Evenly spaced FP64 bounds lo + ((hi - lo) i) / (count - 1), turned into the
// smallest FP32 value >= each bound: for an FP32 z, z >= bound exactly when
// z >= that value.
__device__ __forceinline__ float bound_ru(double lo, double hi, int i, int count)
{
    const double e = __dadd_rn(lo, __ddiv_rn(__dmul_rn(__dsub_rn(hi, lo), (double)i), (double)(count - 1)));
    return __double2float_ru(e);
}

constexpr int kPartThreads = 256;
constexpr int kPartItems = 4;
constexpr int kPartTile = kPartThreads * kPartItems;  // pixels per partition block

// Alg. 2: cluster = the largest i <= E-2 with z >= e_i. One block per 1024
// consecutive pixels; also its per-cluster counts (for the stable partition)
// and the cluster sizes.
__global__ void __launch_bounds__(kPartThreads) k_bs_cluster(const float *__restrict__ z, int64_t N, int E,
                                                             BsCounters *__restrict__ cnt, uint8_t *__restrict__ cl,
                                                             uint32_t *__restrict__ blk_cnt, uint8_t *__restrict__ dark)
{
    __shared__ float s_t[kMaxClusters];
    __shared__ uint32_t s_cnt[kMaxClusters];
    const double zmin = (double)__uint_as_float(~cnt->zmin_inv), zmax = (double)__uint_as_float(cnt->zmax_bits);
    if ((int)threadIdx.x < E - 2) s_t[threadIdx.x] = bound_ru(zmin, zmax, threadIdx.x + 1, E);
    if ((int)threadIdx.x < E - 1) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kPartTile;
#pragma unroll
    for (int r = 0; r < kPartItems; r++) {
        const int64_t i = base + r * kPartThreads + threadIdx.x;
        int c = kMaxClusters;  // past the end: a cluster no pixel has
        if (i < N) {
            const float zi = z[i];
            c = 0;
            for (int k = 0; k < E - 2; k++) c += zi >= s_t[k];
            cl[i] = (uint8_t)c;
            if (dark) dark[i] = 0;
        }
        // one shared atomic per distinct cluster in the warp
        const unsigned peers = peers_of((uint32_t)c, 7);
        if (c < kMaxClusters && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&s_cnt[c], (uint32_t)__popc(peers));
    }
    __syncthreads();
    if ((int)threadIdx.x < E - 1) {
        const uint32_t v = s_cnt[threadIdx.x];
        blk_cnt[(int64_t)blockIdx.x * (E - 1) + threadIdx.x] = v;
        if (v) atomicAdd(&cnt->count[threadIdx.x], v);
    }
}

// Start of every (block, cluster) run in the cluster-major partition: warp c
// scans column c of blk_cnt over the blocks, after the sizes of the clusters
// before c. Also the segment start of each cluster.
__global__ void __launch_bounds__(1024) k_bs_offsets(int nblk, int E, BsCounters *__restrict__ cnt,
                                                     uint32_t *__restrict__ blk_cnt)
{
    const int lane = threadIdx.x & 31;
    for (int c = threadIdx.x >> 5; c < E - 1; c += 32) {
    uint32_t carry = 0;
    for (int k = 0; k < c; k++) carry += cnt->count[k];
    if (lane == 0) cnt->start[c] = carry;
    for (int b0 = 0; b0 < nblk; b0 += 32) {
        const int b = b0 + lane;
        const uint32_t v = b < nblk ? blk_cnt[(int64_t)b * (E - 1) + c] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (b < nblk) blk_cnt[(int64_t)b * (E - 1) + c] = carry + x - v;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    }
}

// Stable partition by cluster: every pixel's (key, index) goes to its
// cluster's segment, in index order.
__global__ void __launch_bounds__(kPartThreads) k_bs_scatter(const uint32_t *__restrict__ key, const uint8_t *__restrict__ cl,
                                                             int64_t N, int E, const uint32_t *__restrict__ blk_off,
                                                             uint32_t *__restrict__ seg_key, uint32_t *__restrict__ seg_idx)
{
    constexpr int kWarps = kPartThreads / 32;
    __shared__ uint32_t s_run[kMaxClusters];           // pixels of each cluster placed so far
    __shared__ uint32_t s_wc[kWarps][kMaxClusters];    // this round's count per warp and cluster
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if ((int)threadIdx.x < E - 1) s_run[threadIdx.x] = blk_off[(int64_t)blockIdx.x * (E - 1) + threadIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kPartTile;
    for (int r = 0; r < kPartItems; r++) {
        for (int k = threadIdx.x; k < kWarps * kMaxClusters; k += kPartThreads) (&s_wc[0][0])[k] = 0;
        __syncthreads();
        const int64_t i = base + r * kPartThreads + threadIdx.x;
        const bool ok = i < N;
        int c = ok ? cl[i] : kMaxClusters;  // past the end: a cluster no pixel has
        const unsigned peers = peers_of((uint32_t)c, 7);
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        if (ok && lane == __ffs(peers) - 1) s_wc[wid][c] = __popc(peers);
        __syncthreads();
        if (ok) {
            uint32_t pos = s_run[c] + rank;
            for (int w2 = 0; w2 < wid; w2++) pos += s_wc[w2][c];
            seg_key[pos] = key[i];
            seg_idx[pos] = (uint32_t)i;
        }
        __syncthreads();
        if ((int)threadIdx.x < E - 1) {
            uint32_t t = 0;
            for (int w2 = 0; w2 < kWarps; w2++) t += s_wc[w2][threadIdx.x];
            s_run[threadIdx.x] += t;
        }
        __syncthreads();
    }
}

constexpr int kSelThreads = 1024;

// Inclusive block scan of one value per thread (kSelThreads threads).
__device__ __forceinline__ uint32_t block_incl_scan(uint32_t v, uint32_t *s_w)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) s_w[wid] = v;
    __syncthreads();
    if (wid == 0) {
        uint32_t x = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        s_w[lane] = x;
    }
    __syncthreads();
    const uint32_t r = v + (wid ? s_w[wid - 1] : 0u);
    __syncthreads();
    return r;
}

// Block c keeps the k = ceil(p_dark n_c) smallest (key, index) pairs of
// cluster c's segment (index order): three radix rounds (11, 11, 10 bits)
// find the k-th smallest key t, then every key < t is kept together with the
// first keys == t needed to reach k.
__global__ void __launch_bounds__(kSelThreads) k_bs_select(const uint32_t *__restrict__ seg_key,
                                                           const uint32_t *__restrict__ seg_idx, double p_dark,
                                                           BsCounters *__restrict__ cnt, uint32_t *__restrict__ list,
                                                           uint8_t *__restrict__ dark)
{
    __shared__ uint32_t hist[2048];
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_pick[2];
    const int c = blockIdx.x;
    const uint32_t n = cnt->count[c];
    if (n == 0) return;
    const uint32_t *keys = seg_key + cnt->start[c];
    const uint32_t *idxs = seg_idx + cnt->start[c];
    uint32_t krem = (uint32_t)ceil(__dmul_rn(p_dark, (double)n));
    krem = min(max(krem, 1u), n);
    uint32_t prefix = 0, pmask = 0;
    for (int round = 0; round < 3; round++) {
        const int shift = round == 0 ? 21 : (round == 1 ? 10 : 0);
        const uint32_t dmask = round == 2 ? 0x3ffu : 0x7ffu;
        for (int b = threadIdx.x; b < 2048; b += kSelThreads) hist[b] = 0;
        __syncthreads();
        for (uint32_t j0 = 0; j0 < n; j0 += kSelThreads) {
            const uint32_t j = j0 + threadIdx.x;
            const uint32_t u = j < n ? keys[j] : 0u;
            const bool in = j < n && (u & pmask) == prefix;
            const uint32_t d = in ? (u >> shift) & dmask : 0xffffffffu;
            // one shared atomic per distinct digit in the warp (neighbouring keys share digits)
            // (11-bit digits: one match.any beats twelve ballots here)
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            if (in && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[d], (uint32_t)__popc(peers));
        }
        __syncthreads();
        // thread t owns bins 2t, 2t+1; find the bin where the running count reaches krem
        const uint32_t h0 = hist[2 * threadIdx.x], h1 = hist[2 * threadIdx.x + 1];
        const uint32_t incl = block_incl_scan(h0 + h1, s_w);
        const uint32_t excl = incl - h0 - h1;
        if (excl < krem && incl >= krem) {
            const bool first = excl + h0 >= krem;
            s_pick[0] = 2 * threadIdx.x + (first ? 0 : 1);
            s_pick[1] = first ? excl : excl + h0;
        }
        __syncthreads();
        prefix |= s_pick[0] << shift;
        pmask |= dmask << shift;
        krem -= s_pick[1];
        __syncthreads();
    }
    const uint32_t t = prefix, need = krem;  // keys < t all kept; `need` of the keys == t
    const uint32_t chunk = (n + kSelThreads - 1) / kSelThreads;
    const uint32_t a = min(n, threadIdx.x * chunk), b = min(n, a + chunk);
    uint32_t ties = 0;
    for (uint32_t j = a; j < b; j++) ties += keys[j] == t;
    uint32_t before = block_incl_scan(ties, s_w) - ties;
    for (uint32_t j = a; j < b; j++) {
        const uint32_t u = keys[j];
        bool take = u < t;
        if (u == t) take = before++ < need;
        if (take) {
            const uint32_t i = idxs[j];
            list[atomicAdd(&cnt->n_dark, 1u)] = i;
            if (dark) dark[i] = 1;
        }
    }
}

// Profiled residual of one channel: for a given beta the best B is the
// clipped linear least-squares value B(beta) = clip(sum m f / sum f f), and
// by the envelope theorem dS/dbeta = -2 B (sum m f' - B sum f f'), with
// f = 1 - exp(-beta z) and f' = z exp(-beta z). FP32; one thread per beta.
__device__ __forceinline__ float dS32(float beta, const float *z, const float *m, int n, float bmax)
{
    float smf = 0.f, sff = 0.f, smp = 0.f, sfp = 0.f;
    for (int j = 0; j < n; j++) {
        const float em1 = expm1f(-beta * z[j]), f = -em1, fp = z[j] * (1.f + em1);
        smf = fmaf(m[j], f, smf);
        sff = fmaf(f, f, sff);
        smp = fmaf(m[j], fp, smp);
        sfp = fmaf(f, fp, sfp);
    }
    const float B = sff > 0.f ? fminf(bmax, fmaxf(0.f, smf / sff)) : 0.f;
    return -2.f * B * (smp - B * sfp);
}

__device__ __forceinline__ float B32(float beta, const float *z, const float *m, int n, float bmax)
{
    float smf = 0.f, sff = 0.f;
    for (int j = 0; j < n; j++) {
        const float f = -expm1f(-beta * z[j]);
        smf = fmaf(m[j], f, smf);
        sff = fmaf(f, f, sff);
    }
    return sff > 0.f ? fminf(bmax, fmaxf(0.f, smf / sff)) : 0.f;
}

__device__ __forceinline__ float S32(float beta, float B, const float *z, const float *m, int n)
{
    float S = 0.f;
    for (int j = 0; j < n; j++) {
        const float r = m[j] + B * expm1f(-beta * z[j]);
        S = fmaf(r, r, S);
    }
    return S;
}

// Block-wide: the first thread whose flag is set (kGrid if none), and
// whether any thread's `any` is set.
__device__ __forceinline__ int block_first(bool flag, bool any, int *s_i, int *s_any)
{
    int v = __reduce_min_sync(0xffffffffu, flag ? (int)threadIdx.x : kGrid);
    const unsigned a = __reduce_or_sync(0xffffffffu, any ? 1u : 0u);
    if ((threadIdx.x & 31) == 0) {
        s_i[threadIdx.x >> 5] = v;
        s_any[threadIdx.x >> 5] = (int)a;
    }
    __syncthreads();
    int r = kGrid, an = 0;
    for (int w = 0; w < kGrid / 32; w++) {
        r = min(r, s_i[w]);
        an |= s_any[w];
    }
    __syncthreads();
    return an ? r : -1;
}

// Bounded fit of one channel (block = channel): level 1 scans the residual
// at kGrid betas over [0, beta_max] for the global minimum; levels 2 and 3
// scan the sign of dS/dbeta at kGrid betas inside the best cell pair and
// then inside the bracketing sub-cell, locating the zero to about the FP32
// noise of dS (a few 1e-6 relative). Where dS keeps one sign across a cell
// the minimum is on the cell's edge (a bound of the box, or the level-1
// point when dS vanishes identically).
__global__ void __launch_bounds__(kGrid) k_bs_fit(const float *__restrict__ res, int64_t N, int w, int h, int M,
                                                  const BsCounters *__restrict__ cnt, const uint32_t *__restrict__ list,
                                                  splash_backscatter_result *__restrict__ out, float bmax, float beta_max)
{
    __shared__ float s_z[kMaxIntervals], s_m[kMaxIntervals];
    __shared__ unsigned long long s_min[32];
    __shared__ unsigned long long s_best[kMaxIntervals];
    __shared__ float s_f[kMaxIntervals];
    __shared__ uint32_t s_red[32];
    __shared__ int s_i[32], s_any[32];
    __shared__ int s_g, s_n;
    const int ch = blockIdx.x, t = threadIdx.x;
    // Alg. 1 steps 6-8 for this channel: interval bounds over the kept
    // depths, then per interval the kept pixel with the smallest (value, index)
    const uint32_t nd = cnt->n_dark;
    const float *zres = res + 3 * N, *vres = res + ch * N;
    uint32_t hi_b = 0, lo_inv = 0;
    for (uint32_t j = t; j < nd; j += blockDim.x) {
        const uint32_t zb = __float_as_uint(zres[list[j]]);
        hi_b = max(hi_b, zb);
        lo_inv = max(lo_inv, ~zb);
    }
    hi_b = block_max_u32(hi_b, s_red);
    lo_inv = block_max_u32(lo_inv, s_red);
    if (t < M - 2) s_f[t] = bound_ru(__uint_as_float(~lo_inv), __uint_as_float(hi_b), t + 1, M);
    if (t < kMaxIntervals) s_best[t] = ~0ull;
    __syncthreads();
    for (uint32_t j = t; j < nd; j += blockDim.x) {
        const uint32_t idx = list[j];
        const float zi = zres[idx];
        int iv = 0;
        for (int k = 0; k < M - 2; k++) iv += zi >= s_f[k];
        atomicMin(&s_best[iv], ((unsigned long long)__float_as_uint(vres[idx]) << 32) | idx);
    }
    __syncthreads();
    if (t == 0) {
        int np = 0;
        for (int iv = 0; iv < M - 1; iv++) {
            const unsigned long long b = s_best[iv];
            if (b == ~0ull) continue;
            s_z[np] = zres[(uint32_t)(b & 0xffffffffu)];
            s_m[np] = __uint_as_float((uint32_t)(b >> 32));
            np++;
        }
        s_n = np;
        out->n_points[ch] = np;
        if (ch == 0) {
            out->n_dark = (int32_t)nd;
            out->width = w;
            out->height = h;
            out->pad = 0;
        }
    }
    __syncthreads();
    const int n = s_n;
    for (int j = t; j < kMaxIntervals; j += blockDim.x) {
        out->point_z[ch][j] = j < n ? s_z[j] : 0.f;
        out->point_v[ch][j] = j < n ? s_m[j] : 0.f;
    }
    if (n <= 0) {
        if (t == 0) out->beta_b[ch] = out->b_inf[ch] = out->residual[ch] = 0.f;
        return;
    }
    // level 1: residual at beta_g = beta_max g / (kGrid - 1)
    auto grid1 = [&](int g) { return beta_max * (float)g / (float)(kGrid - 1); };
    {
        const float beta = grid1(t);
        const float S = S32(beta, B32(beta, s_z, s_m, n, bmax), s_z, s_m, n);
        unsigned long long v = ((unsigned long long)__float_as_uint(S) << 32) | (uint32_t)t;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
        if ((t & 31) == 0) s_min[t >> 5] = v;
        __syncthreads();
        if (t < 32) {
            unsigned long long u = s_min[t];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) u = min(u, __shfl_xor_sync(0xffffffffu, u, o));
            if (t == 0) s_g = (int)(u & 0xffffffffu);
        }
        __syncthreads();
    }
    const int g = s_g;
    float lo = grid1(max(g - 1, 0)), hi = grid1(min(g + 1, kGrid - 1));
    float beta = grid1(g);
    // levels 2 and 3: first point of the cell where dS > 0
    for (int level = 0; level < 2; level++) {
        const float b = lo + (hi - lo) * (float)t / (float)(kGrid - 1);
        const float d = dS32(b, s_z, s_m, n, bmax);
        const int first = block_first(d > 0.f, d != 0.f, s_i, s_any);
        if (first < 0) break;  // dS vanishes on the whole cell: keep the level-1 point
        if (first == 0) {      // rising from the left edge: the minimum is at that edge
            beta = lo;
            break;
        }
        const float l2 = lo + (hi - lo) * (float)(first - 1) / (float)(kGrid - 1);
        const float h2 = first == kGrid ? hi : lo + (hi - lo) * (float)first / (float)(kGrid - 1);
        if (first == kGrid) {  // falling across the whole cell: the minimum is at the right edge
            beta = hi;
            break;
        }
        lo = l2;
        hi = h2;
        beta = 0.5f * (lo + hi);
    }
    if (t == 0) {
        const float B = B32(beta, s_z, s_m, n, bmax);
        out->beta_b[ch] = beta;
        out->b_inf[ch] = B;
        out->residual[ch] = S32(beta, B, s_z, s_m, n);
    }
}

__global__ void k_bs_prior(const float *__restrict__ medium, const float *__restrict__ prior, float lam,
                           float *__restrict__ grad, float *__restrict__ loss)
{
    const int j = threadIdx.x;
    float l = 0.f;
    if (j < 6) {
        const float d = medium[3 + j] - prior[j];
        l = lam * fabsf(d);
        if (grad) grad[3 + j] += d > 0.f ? lam : (d < 0.f ? -lam : 0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (j == 0 && loss) *loss += l;
}

}  // namespace
}  // namespace splash

using namespace splash;

extern "C" splash_status splash_backscatter_estimate(splash_ctx *ctx, const float *image, const float *depth,
                                                     int32_t width, int32_t height,
                                                     const splash_backscatter_options *opt,
                                                     splash_backscatter_result *result, float *resized, uint8_t *dark,
                                                     void *stream)
{
    if (!ctx || !image || !depth || !result) return fail(SPLASH_ERR_INVALID_ARG, "null context, image, depth or result");
    if (reinterpret_cast<uintptr_t>(result) & 15) return fail(SPLASH_ERR_INVALID_ARG, "result must be 16-byte aligned");
    splash_backscatter_options o{300, 10, 25, 0, 0.01, 1.0f, 5.0f};
    if (opt) o = *opt;
    if (width <= 0 || height <= 0 || (int64_t)width * height >= ((int64_t)1 << 31))
        return fail(SPLASH_ERR_INVALID_ARG, "image size must be positive and below 2^31 pixels");
    if (o.resized_height < 1 || o.resized_height > 4096) return fail(SPLASH_ERR_INVALID_ARG, "resized_height must be 1..4096");
    if (o.edges < 2 || o.edges > kMaxClusters + 1) return fail(SPLASH_ERR_INVALID_ARG, "edges must be 2..65");
    if (o.intervals < 2 || o.intervals > kMaxIntervals + 1) return fail(SPLASH_ERR_INVALID_ARG, "intervals must be 2..65");
    if (!(o.p_dark > 0.0 && o.p_dark <= 1.0)) return fail(SPLASH_ERR_INVALID_ARG, "p_dark must be in (0, 1]");
    if (!(o.b_max > 0.f && o.b_max < 1e30f) || !(o.beta_max > 0.f && o.beta_max < 1e30f))
        return fail(SPLASH_ERR_INVALID_ARG, "fit bounds must be positive and finite");
    const int h = o.resized_height;
    const int w = (int)std::max<int64_t>(1, (2 * (int64_t)width * h + height) / (2 * (int64_t)height));
    const int64_t N = (int64_t)h * w;
    if (N > ((int64_t)1 << 24)) return fail(SPLASH_ERR_INVALID_ARG, "resized image above 2^24 pixels");
    cudaStream_t s = (cudaStream_t)stream;
    // scratch: counters | keys [N] | clusters [N] | kept list [N] | partition keys, indices [N] |
    // per-block cluster counts | resized [4N] (when not given)
    const int nblk = (int)((N + kPartTile - 1) / kPartTile);
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t off_key = up(sizeof(BsCounters)), off_cl = off_key + up(4 * N), off_list = off_cl + up(N),
                 off_sk = off_list + up(4 * N), off_si = off_sk + up(4 * N), off_blk = off_si + up(4 * N),
                 off_res = off_blk + up(4 * (size_t)nblk * (o.edges - 1)), total = off_res + (resized ? 0 : up(16 * N));
    ENSURE(ctx->bs_scratch, total);
    char *base = ctx->bs_scratch.as<char>();
    BsCounters *cnt = reinterpret_cast<BsCounters *>(base);
    uint32_t *key = reinterpret_cast<uint32_t *>(base + off_key);
    uint8_t *cl = reinterpret_cast<uint8_t *>(base + off_cl);
    uint32_t *list = reinterpret_cast<uint32_t *>(base + off_list);
    uint32_t *seg_key = reinterpret_cast<uint32_t *>(base + off_sk);
    uint32_t *seg_idx = reinterpret_cast<uint32_t *>(base + off_si);
    uint32_t *blk = reinterpret_cast<uint32_t *>(base + off_blk);
    float *res = resized ? resized : reinterpret_cast<float *>(base + off_res);
    const unsigned blocks = (unsigned)((N + 255) / 256);
    {
        Stage t(ctx->prof, SPLASH_STAGE_BS_RESIZE, s);
        SPLASH_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(BsCounters), s));
        k_bs_resize<<<blocks, 256, 0, s>>>(image, depth, width, height, w, h, res, key, cnt);
    }
    {
        Stage t(ctx->prof, SPLASH_STAGE_BACKSCATTER, s);
        k_bs_cluster<<<nblk, kPartThreads, 0, s>>>(res + 3 * N, N, o.edges, cnt, cl, blk, dark);
        k_bs_offsets<<<1, 1024, 0, s>>>(nblk, o.edges, cnt, blk);
        k_bs_scatter<<<nblk, kPartThreads, 0, s>>>(key, cl, N, o.edges, blk, seg_key, seg_idx);
        k_bs_select<<<o.edges - 1, kSelThreads, 0, s>>>(seg_key, seg_idx, o.p_dark, cnt, list, dark);
        k_bs_fit<<<3, kGrid, 0, s>>>(res, N, w, h, o.intervals, cnt, list, result, o.b_max, o.beta_max);
        count_launch(6);
    }
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}

extern "C" splash_status splash_backscatter_prior(const float *medium, const float *prior, float lambda_est,
                                                  float *grad_medium, float *loss, void *stream)
{
    if (!medium || !prior) return fail(SPLASH_ERR_INVALID_ARG, "null medium or prior");
    if (!(lambda_est >= 0.f)) return fail(SPLASH_ERR_INVALID_ARG, "lambda_est must be >= 0");
    if (!grad_medium && !loss) return SPLASH_OK;
    k_bs_prior<<<1, 32, 0, (cudaStream_t)stream>>>(medium, prior, lambda_est, grad_medium, loss);
    count_launch();
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}
