// MCMC densification (Sec. IV-D adopts the sampling form of 3DGS-MCMC in
// place of clone / split / prune; Sec. VI ablates the choice): relocation of
// dead Gaussians and the position noise.
//   k_mcmc_weights  -- w = sigmoid(o) of live Gaussians (0 for dead ones), FP64
//   k_f64_scan_*    -- the running sum C of w in index order, FP64
//   k_mcmc_draw     -- each dead Gaussian's source: the first g with C_g > u C_total
//   k_mcmc_sources  -- a source drawn c times stands for N = min(c + 1, 51)
//                      Gaussians: o' = 1 - (1 - o)^(1/N), s' = s o / Z(N, o')
//   k_mcmc_copies   -- each dead Gaussian takes its source's new parameters;
//                      the moments of sources and copies are zeroed
//   k_mcmc_noise    -- mu += lambda lr sigmoid(-k (o - t)) Sigma eta
#include <cuda_runtime.h>
#include <math.h>

#include "host.h"
#include "internal.cuh"

using namespace splash_host;

namespace splash {
namespace {

constexpr int kMcmcNMax = 51;
constexpr int kScanChunk = 1024;  // elements per block of the FP64 running sum (256 threads x 4)

__global__ void k_mcmc_weights(const float *__restrict__ logits, int64_t n, double min_opacity, double *__restrict__ w,
                               uint32_t *__restrict__ n_dead)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double o = 1.0 / (1.0 + exp(-(double)logits[i]));
        const bool dead = o <= min_opacity;
        w[i] = dead ? 0.0 : o;
        if (dead) atomicAdd(n_dead, 1u);
    }
}

__device__ __forceinline__ double warp_incl_scan(double x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// in place: C[i] = inclusive running sum within the block's chunk; sums[b] = the chunk's total
__global__ void __launch_bounds__(256) k_f64_scan_chunks(double *__restrict__ c, int64_t n, double *__restrict__ sums)
{
    __shared__ double s_w[8];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + 4 * threadIdx.x;
    double v[4], t = 0.0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        v[j] = base + j < n ? c[base + j] : 0.0;
        t += v[j];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double incl = warp_incl_scan(t, lane);
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    double pre = 0.0;
    for (int w = 0; w < warp; w++) pre += s_w[w];
    double run = pre + incl - t;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        run += v[j];
        if (base + j < n) c[base + j] = run;
    }
    if (threadIdx.x == 255) sums[blockIdx.x] = run;
}

// one CTA: exclusive running sum of the chunk totals, chunk after chunk of 256
__global__ void __launch_bounds__(256) k_f64_scan_top(double *__restrict__ sums, int64_t nchunks)
{
    __shared__ double s_w[8];
    __shared__ double s_carry;
    if (threadIdx.x == 0) s_carry = 0.0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t b0 = 0; b0 < nchunks; b0 += 256) {
        const int64_t i = b0 + threadIdx.x;
        const double t = i < nchunks ? sums[i] : 0.0;
        const double incl = warp_incl_scan(t, lane);
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        double pre = s_carry;
        for (int w = 0; w < warp; w++) pre += s_w[w];
        if (i < nchunks) sums[i] = pre + incl - t;
        __syncthreads();
        if (threadIdx.x == 255) s_carry = pre + incl;
        __syncthreads();
    }
}

__global__ void k_f64_scan_add(double *__restrict__ c, int64_t n, const double *__restrict__ sums)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c[i] += sums[i / kScanChunk];
}

// each dead Gaussian (w = 0 and its opacity at or below the minimum) draws its
// source: the first g with C_g > u C_total (C is non-decreasing)
__global__ void k_mcmc_draw(const float *__restrict__ logits, const float *__restrict__ u, const double *__restrict__ c,
                            int64_t n, double min_opacity, int32_t *__restrict__ src, uint32_t *__restrict__ cnt)
{
    const double total = c[n - 1];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double o = 1.0 / (1.0 + exp(-(double)logits[i]));
        if (!(o <= min_opacity) || !(total > 0.0)) {
            src[i] = -1;
            continue;
        }
        const double target = (double)u[i] * total;
        int64_t lo = 0, hi = n - 1;  // the answer lies in [lo, hi]: C_{n-1} = total > target for u < 1
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (c[mid] > target) hi = mid;
            else lo = mid + 1;
        }
        // the blocked running sum is monotone to within rounding: never take a
        // dead Gaussian (an opacity at or below the minimum) as the source
        while (lo < n - 1 && 1.0 / (1.0 + exp(-(double)logits[lo])) <= min_opacity) lo++;
        src[i] = (int32_t)lo;
        atomicAdd(cnt + lo, 1u);
    }
}

struct McmcParams {
    float *p[5], *m[5], *v[5];  // means, log_scales, quats, opacity_logits, sh
    int width[5];               // floats per Gaussian in each group
};

__device__ __forceinline__ void zero_moments(const McmcParams &d, int64_t i)
{
#pragma unroll
    for (int g = 0; g < 5; g++)
        for (int k = 0; k < d.width[g]; k++) {
            d.m[g][i * d.width[g] + k] = 0.f;
            d.v[g][i * d.width[g] + k] = 0.f;
        }
}

// the sources drawn at least once: the shared opacity and scale of a source and its copies
__global__ void k_mcmc_sources(McmcParams d, int64_t n, const uint32_t *__restrict__ cnt)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = cnt[g];
        if (c == 0) continue;
        const int N = (int)min(c + 1u, (uint32_t)kMcmcNMax);
        const double o = 1.0 / (1.0 + exp(-(double)d.p[3][g]));
        const double on = 1.0 - pow(1.0 - o, 1.0 / N);
        // Z = sum_{i=1}^{N} sum_{k=0}^{i-1} C(i-1, k) (-1)^k on^(k+1) / sqrt(k+1)
        double z = 0.0;
        for (int i = 1; i <= N; i++) {
            double binom = 1.0, pw = on;
            for (int k = 0; k < i; k++) {
                z += ((k & 1) ? -binom : binom) * pw / sqrt((double)(k + 1));
                binom = binom * (double)(i - 1 - k) / (double)(k + 1);
                pw *= on;
            }
        }
        d.p[3][g] = (float)log(on / (1.0 - on));
        const double lf = log(o / z);
#pragma unroll
        for (int k = 0; k < 3; k++) d.p[1][3 * g + k] = (float)((double)d.p[1][3 * g + k] + lf);
        zero_moments(d, g);
    }
}

__global__ void k_mcmc_copies(McmcParams d, int64_t n, const int32_t *__restrict__ src)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = src[i];
        if (s < 0) continue;
#pragma unroll
        for (int g = 0; g < 5; g++)
            for (int k = 0; k < d.width[g]; k++) d.p[g][i * d.width[g] + k] = d.p[g][(int64_t)s * d.width[g] + k];
        zero_moments(d, i);
    }
}

__global__ void k_mcmc_noise(float *__restrict__ means, const float *__restrict__ log_scales,
                             const float *__restrict__ quats, const float *__restrict__ logits,
                             const float *__restrict__ eta, int64_t n, float step, float k_gate, float t_gate)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float o = 1.f / (1.f + expf(-logits[i]));
        const float gate = 1.f / (1.f + expf(k_gate * (o - t_gate)));  // sigmoid(-k (o - t))
        const float4 q = reinterpret_cast<const float4 *>(quats)[i];
        const float qi = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
        const float w = q.x * qi, x = q.y * qi, y = q.z * qi, z = q.w * qi;
        const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                            2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                            2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
        const float e[3] = {eta[3 * i], eta[3 * i + 1], eta[3 * i + 2]};
        // Sigma eta = R diag(s^2) R^T eta
        float a[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float s2 = expf(2.f * log_scales[3 * i + c]);
            a[c] = s2 * (R[c] * e[0] + R[3 + c] * e[1] + R[6 + c] * e[2]);
        }
        const float f = step * gate;
#pragma unroll
        for (int r = 0; r < 3; r++) means[3 * i + r] += f * (R[3 * r] * a[0] + R[3 * r + 1] * a[1] + R[3 * r + 2] * a[2]);
    }
}

}  // namespace
}  // namespace splash

using namespace splash;

extern "C" splash_status splash_mcmc_relocate(splash_ctx *ctx, const splash_param_buffers *params,
                                              const splash_param_buffers *m, const splash_param_buffers *v, int64_t n,
                                              int32_t sh_degree, const float *uniforms, float min_opacity,
                                              int64_t *n_dead, void *stream)
{
    if (!ctx || !params || !m || !v) return fail(SPLASH_ERR_INVALID_ARG, "null argument");
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(SPLASH_ERR_INVALID_ARG, "n must be in [0, 2^31)");
    if (sh_degree < 0 || sh_degree > 3) return fail(SPLASH_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (!(min_opacity > 0.f && min_opacity < 1.f)) return fail(SPLASH_ERR_INVALID_ARG, "min_opacity must be in (0, 1)");
    if (n == 0) {
        if (n_dead) *n_dead = 0;
        return SPLASH_OK;
    }
    if (!uniforms) return fail(SPLASH_ERR_INVALID_ARG, "null uniforms");
    McmcParams d{};
    const splash_param_buffers *src[3] = {params, m, v};
    for (int w = 0; w < 3; w++) {
        float *in[5] = {src[w]->means, src[w]->log_scales, src[w]->quats, src[w]->opacity_logits, src[w]->sh};
        for (int g = 0; g < 5; g++) {
            if (!in[g]) return fail(SPLASH_ERR_INVALID_ARG, "null parameter or moment buffer");
            (w == 0 ? d.p : (w == 1 ? d.m : d.v))[g] = in[g];
        }
    }
    if (reinterpret_cast<uintptr_t>(params->quats) & 15) return fail(SPLASH_ERR_INVALID_ARG, "quats must be 16-byte aligned");
    const int widths[5] = {3, 3, 4, 1, 3 * (sh_degree + 1) * (sh_degree + 1)};
    for (int g = 0; g < 5; g++) d.width[g] = widths[g];
    const int64_t nchunks = (n + kScanChunk - 1) / kScanChunk;
    ENSURE(ctx->mcmc_c, 8 * (size_t)n);
    ENSURE(ctx->mcmc_sums, 8 * (size_t)(nchunks + 1));
    ENSURE(ctx->mcmc_src, 4 * (size_t)n);
    ENSURE(ctx->mcmc_cnt, 4 * (size_t)n + 16);
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *cnt = ctx->mcmc_cnt.as<uint32_t>();
    uint32_t *nd = cnt + n;  // the dead count, after the per-Gaussian counts
    SPLASH_CUDA_TRY(cudaMemsetAsync(cnt, 0, 4 * (size_t)n + 16, s));
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
    const double mo = (double)min_opacity;
    double *c = ctx->mcmc_c.as<double>();
    k_mcmc_weights<<<blocks, 256, 0, s>>>(d.p[3], n, mo, c, nd);
    k_f64_scan_chunks<<<(unsigned)nchunks, 256, 0, s>>>(c, n, ctx->mcmc_sums.as<double>());
    k_f64_scan_top<<<1, 256, 0, s>>>(ctx->mcmc_sums.as<double>(), nchunks);
    k_f64_scan_add<<<blocks, 256, 0, s>>>(c, n, ctx->mcmc_sums.as<double>());
    k_mcmc_draw<<<blocks, 256, 0, s>>>(d.p[3], uniforms, c, n, mo, ctx->mcmc_src.as<int32_t>(), cnt);
    k_mcmc_sources<<<blocks, 256, 0, s>>>(d, n, cnt);
    k_mcmc_copies<<<blocks, 256, 0, s>>>(d, n, ctx->mcmc_src.as<int32_t>());
    count_launch(7);
    SPLASH_CUDA_TRY(cudaGetLastError());
    if (n_dead) {
        uint32_t h = 0;
        SPLASH_CUDA_TRY(cudaMemcpyAsync(&h, nd, 4, cudaMemcpyDeviceToHost, s));
        SPLASH_CUDA_TRY(cudaStreamSynchronize(s));
        *n_dead = h;
    }
    return SPLASH_OK;
}

extern "C" splash_status splash_mcmc_noise(float *means, const float *log_scales, const float *quats,
                                           const float *opacity_logits, const float *eta, int64_t n, float lr,
                                           float lambda_noise, void *stream)
{
    if (n < 0) return fail(SPLASH_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0) return SPLASH_OK;
    if (!means || !log_scales || !quats || !opacity_logits || !eta) return fail(SPLASH_ERR_INVALID_ARG, "null buffer");
    if (reinterpret_cast<uintptr_t>(quats) & 15) return fail(SPLASH_ERR_INVALID_ARG, "quats must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
    k_mcmc_noise<<<blocks, 256, 0, s>>>(means, log_scales, quats, opacity_logits, eta, n, lambda_noise * lr, 100.f,
                                        0.005f);
    count_launch();
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}
