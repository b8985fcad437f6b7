// Backscatter estimate behind the L_best prior (Sec. IV-B, Eq. 7-9), after
// the appendix's Alg. 1 ("Estimate Backscatter") and Alg. 2 ("Get
// backscatter by curve fitting"): dark pixels per depth cluster of an
// observed view, their per-interval minima, and a bounded per-channel fit of
// B_inf (1 - exp(-beta_B z)).
//
//   k_bs_resize  -- area-average resize of image + depth (FP64 accumulation,
//                   one rounding to FP32), darkness keys, depth min/max
//   k_bs_cluster -- depth cluster of every pixel, cluster sizes
//   k_bs_select  -- one block per cluster: radix select of the
//                   ceil(p_dark n)-th darkest key, then the kept pixels
//   k_bs_minima  -- interval minima of the kept pixels -> fit points
//   k_bs_fit     -- one block per channel: FP32 scan over beta, FP64
//                   root of the profiled residual's derivative
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
    uint32_t count[kMaxClusters];
};

__device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

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

// Alg. 2: cluster = the largest i <= E-2 with z >= e_i.
__global__ void __launch_bounds__(256) k_bs_cluster(const float *__restrict__ z, int64_t N, int E,
                                                    BsCounters *__restrict__ cnt, uint8_t *__restrict__ cl,
                                                    uint8_t *__restrict__ dark)
{
    __shared__ float s_t[kMaxClusters];
    __shared__ uint32_t s_cnt[kMaxClusters];
    const double zmin = (double)__uint_as_float(~cnt->zmin_inv), zmax = (double)__uint_as_float(cnt->zmax_bits);
    if ((int)threadIdx.x < E - 2) s_t[threadIdx.x] = bound_ru(zmin, zmax, threadIdx.x + 1, E);
    if ((int)threadIdx.x < E - 1) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        const float zi = z[i];
        int c = 0;
        for (int k = 0; k < E - 2; k++) c += zi >= s_t[k];
        cl[i] = (uint8_t)c;
        if (dark) dark[i] = 0;
        atomicAdd(&s_cnt[c], 1u);
    }
    __syncthreads();
    if ((int)threadIdx.x < E - 1 && s_cnt[threadIdx.x]) atomicAdd(&cnt->count[threadIdx.x], s_cnt[threadIdx.x]);
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
// cluster c: three radix rounds (11, 11, 10 bits) find the k-th smallest key
// t, then every key < t is kept together with the first (in index order)
// keys == t needed to reach k.
__global__ void __launch_bounds__(kSelThreads) k_bs_select(const uint32_t *__restrict__ key, const uint8_t *__restrict__ cl,
                                                           int64_t N, double p_dark, BsCounters *__restrict__ cnt,
                                                           uint32_t *__restrict__ list, uint8_t *__restrict__ dark)
{
    __shared__ uint32_t hist[2048];
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_pick[2];
    const int c = blockIdx.x;
    const uint32_t n = cnt->count[c];
    if (n == 0) return;
    uint32_t krem = (uint32_t)ceil(__dmul_rn(p_dark, (double)n));
    krem = min(max(krem, 1u), n);
    uint32_t prefix = 0, pmask = 0;
    for (int round = 0; round < 3; round++) {
        const int shift = round == 0 ? 21 : (round == 1 ? 10 : 0);
        const uint32_t dmask = round == 2 ? 0x3ffu : 0x7ffu;
        for (int b = threadIdx.x; b < 2048; b += kSelThreads) hist[b] = 0;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < N; i += kSelThreads) {
            if (cl[i] != c) continue;
            const uint32_t u = key[i];
            if ((u & pmask) == prefix) atomicAdd(&hist[(u >> shift) & dmask], 1u);
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
    const int64_t chunk = (N + kSelThreads - 1) / kSelThreads;
    const int64_t a = min64(N, (int64_t)threadIdx.x * chunk), b = min64(N, a + chunk);
    uint32_t ties = 0;
    for (int64_t i = a; i < b; i++) ties += (cl[i] == c && key[i] == t);
    uint32_t before = block_incl_scan(ties, s_w) - ties;
    for (int64_t i = a; i < b; i++) {
        if (cl[i] != c) continue;
        const uint32_t u = key[i];
        bool take = u < t;
        if (u == t) take = before++ < need;
        if (take) {
            list[atomicAdd(&cnt->n_dark, 1u)] = (uint32_t)i;
            if (dark) dark[i] = 1;
        }
    }
}

// Alg. 1 steps 6-8: interval bounds over the kept depths; per channel and
// interval, the kept pixel with the smallest (value, index).
__global__ void __launch_bounds__(1024) k_bs_minima(const float *__restrict__ res, int64_t N, int w, int h, int M,
                                                    const BsCounters *__restrict__ cnt, const uint32_t *__restrict__ list,
                                                    splash_backscatter_result *__restrict__ out)
{
    __shared__ uint32_t s_red[32];
    __shared__ float s_f[kMaxIntervals];
    __shared__ unsigned long long s_best[3][kMaxIntervals];
    const uint32_t nd = cnt->n_dark;
    const float *zres = res + 3 * N;
    uint32_t hi = 0, loinv = 0;
    for (uint32_t j = threadIdx.x; j < nd; j += blockDim.x) {
        const uint32_t zb = __float_as_uint(zres[list[j]]);
        hi = max(hi, zb);
        loinv = max(loinv, ~zb);
    }
    hi = block_max_u32(hi, s_red);
    loinv = block_max_u32(loinv, s_red);
    if ((int)threadIdx.x < M - 2) s_f[threadIdx.x] = bound_ru(__uint_as_float(~loinv), __uint_as_float(hi), threadIdx.x + 1, M);
    for (int k = threadIdx.x; k < 3 * kMaxIntervals; k += blockDim.x) (&s_best[0][0])[k] = ~0ull;
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < nd; j += blockDim.x) {
        const uint32_t idx = list[j];
        const float zi = zres[idx];
        int iv = 0;
        for (int k = 0; k < M - 2; k++) iv += zi >= s_f[k];
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            const unsigned long long v = ((unsigned long long)__float_as_uint(res[ch * N + idx]) << 32) | idx;
            atomicMin(&s_best[ch][iv], v);
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int ch = threadIdx.x;
        int np = 0;
        for (int iv = 0; iv < M - 1; iv++) {
            const unsigned long long b = s_best[ch][iv];
            if (b == ~0ull) continue;
            const uint32_t idx = (uint32_t)(b & 0xffffffffu);
            out->point_z[ch][np] = zres[idx];
            out->point_v[ch][np] = __uint_as_float((uint32_t)(b >> 32));
            np++;
        }
        out->n_points[ch] = np;
    }
    if (threadIdx.x == 0) {
        out->n_dark = (int32_t)nd;
        out->width = w;
        out->height = h;
        out->pad = 0;
    }
}

// Profiled residual of one channel: for a given beta the best B is the
// clipped linear least-squares value, and by the envelope theorem
// dS/dbeta = -2 B (sum m f' - B sum f f'), f = 1 - exp(-beta z),
// f' = z exp(-beta z). Lanes hold the points; FP64.
struct Prof64 {
    double B, dS;
};

__device__ Prof64 profile64(double beta, const float *z, const float *m, int n, double bmax)
{
    double smf = 0, sff = 0, smp = 0, sfp = 0;
    for (int j = threadIdx.x & 31; j < n; j += 32) {
        const double zj = z[j], mj = m[j];
        const double e = exp(-beta * zj), f = 1.0 - e, fp = zj * e;
        smf = fma(mj, f, smf);
        sff = fma(f, f, sff);
        smp = fma(mj, fp, smp);
        sfp = fma(f, fp, sfp);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        smf += __shfl_xor_sync(0xffffffffu, smf, o);
        sff += __shfl_xor_sync(0xffffffffu, sff, o);
        smp += __shfl_xor_sync(0xffffffffu, smp, o);
        sfp += __shfl_xor_sync(0xffffffffu, sfp, o);
    }
    Prof64 r;
    r.B = sff > 0 ? fmin(bmax, fmax(0.0, smf / sff)) : 0.0;
    r.dS = -2.0 * r.B * (smp - r.B * sfp);
    return r;
}

__global__ void __launch_bounds__(kGrid) k_bs_fit(splash_backscatter_result *__restrict__ out, float bmax, float beta_max)
{
    __shared__ float s_z[kMaxIntervals], s_m[kMaxIntervals];
    __shared__ unsigned long long s_min[32];
    __shared__ int s_g;
    const int ch = blockIdx.x;
    const int n = out->n_points[ch];
    if (n <= 0) {
        if (threadIdx.x == 0) out->beta_b[ch] = out->b_inf[ch] = out->residual[ch] = 0.f;
        return;
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        s_z[j] = out->point_z[ch][j];
        s_m[j] = out->point_v[ch][j];
    }
    __syncthreads();
    // FP32 scan: beta_g = beta_max g / (kGrid - 1), residual with the best B
    {
        const int g = threadIdx.x;
        const float beta = beta_max * (float)g / (float)(kGrid - 1);
        float smf = 0.f, sff = 0.f;
        for (int j = 0; j < n; j++) {
            const float f = -expm1f(-beta * s_z[j]);
            smf = fmaf(s_m[j], f, smf);
            sff = fmaf(f, f, sff);
        }
        const float B = sff > 0.f ? fminf(bmax, fmaxf(0.f, smf / sff)) : 0.f;
        float S = 0.f;
        for (int j = 0; j < n; j++) {
            const float r = s_m[j] + B * expm1f(-beta * s_z[j]);
            S = fmaf(r, r, S);
        }
        unsigned long long v = ((unsigned long long)__float_as_uint(S) << 32) | (uint32_t)g;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
        if ((threadIdx.x & 31) == 0) s_min[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x < 32) {
            unsigned long long u = s_min[threadIdx.x];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) u = min(u, __shfl_xor_sync(0xffffffffu, u, o));
            if (threadIdx.x == 0) s_g = (int)(u & 0xffffffffu);
        }
        __syncthreads();
    }
    if (threadIdx.x >= 32) return;
    // FP64: zero of dS/dbeta next to the best scan point (the bracket moves
    // outward one scan cell at a time if the FP32 scan was off by a cell)
    const double bm = bmax, top = beta_max;
    auto grid = [&](int g) { return top * (double)g / (double)(kGrid - 1); };
    int g = s_g;
    double x = grid(g);
    Prof64 px = profile64(x, s_z, s_m, n, bm);
    double beta = x;
    if (px.dS != 0.0) {
        double lo, hi, flo, fhi;
        bool bracketed = false;
        if (px.dS < 0.0) {  // descending at x: the minimum lies to the right
            lo = x, flo = px.dS;
            int gh = g;
            hi = x, fhi = px.dS;
            while (gh < kGrid - 1) {
                hi = grid(++gh);
                fhi = profile64(hi, s_z, s_m, n, bm).dS;
                if (fhi > 0.0) { bracketed = true; break; }
                if (fhi == 0.0) break;
                lo = hi, flo = fhi;
            }
            if (!bracketed) beta = hi;  // at the upper bound, or an exact stationary point
        } else {
            hi = x, fhi = px.dS;
            int gl = g;
            lo = x, flo = px.dS;
            while (gl > 0) {
                lo = grid(--gl);
                flo = profile64(lo, s_z, s_m, n, bm).dS;
                if (flo < 0.0) { bracketed = true; break; }
                if (flo == 0.0) break;
                hi = lo, fhi = flo;
            }
            if (!bracketed) beta = lo;
        }
        if (bracketed) {
            // Illinois regula falsi on flo < 0 < fhi
            int side = 0;
            for (int it = 0; it < 200; it++) {
                double c = hi - fhi * (hi - lo) / (fhi - flo);
                if (!(c > lo && c < hi)) c = 0.5 * (lo + hi);
                if (!(c > lo && c < hi)) break;  // no representable point left inside
                const double fc = profile64(c, s_z, s_m, n, bm).dS;
                if (fc == 0.0) {
                    lo = hi = c;
                    break;
                }
                if (fc < 0.0) {
                    lo = c, flo = fc;
                    if (side == -1) fhi *= 0.5;
                    side = -1;
                } else {
                    hi = c, fhi = fc;
                    if (side == 1) flo *= 0.5;
                    side = 1;
                }
                if (hi - lo <= 2e-16 * hi) break;
            }
            beta = -flo <= fhi ? lo : hi;
        }
    }
    const Prof64 pf = profile64(beta, s_z, s_m, n, bm);
    double S = 0.0;
    for (int j = threadIdx.x; j < n; j += 32) {
        const double r = (double)s_m[j] - pf.B * (1.0 - exp(-beta * (double)s_z[j]));
        S = fma(r, r, S);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
    if (threadIdx.x == 0) {
        out->beta_b[ch] = (float)beta;
        out->b_inf[ch] = (float)pf.B;
        out->residual[ch] = (float)S;
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
    // scratch: counters | keys [N] | clusters [N] | kept list [N] | resized [4N] (when not given)
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t off_key = up(sizeof(BsCounters)), off_cl = off_key + up(4 * N), off_list = off_cl + up(N),
                 off_res = off_list + up(4 * N), total = off_res + (resized ? 0 : up(16 * N));
    ENSURE(ctx->bs_scratch, total);
    char *base = ctx->bs_scratch.as<char>();
    BsCounters *cnt = reinterpret_cast<BsCounters *>(base);
    uint32_t *key = reinterpret_cast<uint32_t *>(base + off_key);
    uint8_t *cl = reinterpret_cast<uint8_t *>(base + off_cl);
    uint32_t *list = reinterpret_cast<uint32_t *>(base + off_list);
    float *res = resized ? resized : reinterpret_cast<float *>(base + off_res);
    {
        Stage t(ctx->prof, SPLASH_STAGE_BACKSCATTER, s);
        SPLASH_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(BsCounters), s));
        const unsigned blocks = (unsigned)((N + 255) / 256);
        k_bs_resize<<<blocks, 256, 0, s>>>(image, depth, width, height, w, h, res, key, cnt);
        k_bs_cluster<<<blocks, 256, 0, s>>>(res + 3 * N, N, o.edges, cnt, cl, dark);
        k_bs_select<<<o.edges - 1, kSelThreads, 0, s>>>(key, cl, N, o.p_dark, cnt, list, dark);
        k_bs_minima<<<1, 1024, 0, s>>>(res, N, w, h, o.intervals, cnt, list, result);
        k_bs_fit<<<3, kGrid, 0, s>>>(result, o.b_max, o.beta_max);
        count_launch(5);
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
