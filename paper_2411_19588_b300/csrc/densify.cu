// Densification step of the training loop (appendix, "Experimental Setup":
// every 100 iterations from 1,500 to 15,000, gradient threshold 0.0002,
// minimum opacity 0.1; the 3DGS clone / split / prune procedure the paper
// keeps). The per-Gaussian statistics (NDC norm of the screen-space centre
// gradient, visible count) are gathered by the fused adjoint + Adam kernel.
//   k_densify_classify -- action and output count per Gaussian
//   (count scan)       -- where each Gaussian's outputs start
//   k_densify_apply    -- gather the surviving, cloned and split Gaussians
//                         (and their Adam moments) into the new arrays
#include <cuda_runtime.h>
#include <math.h>

#include "host.h"
#include "internal.cuh"

using namespace splash_host;

namespace splash {
namespace {

enum : uint8_t { kPrune = 0, kKeep = 1, kClone = 2, kSplit = 3 };

__global__ void k_iota(uint32_t *__restrict__ out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (uint32_t)i;
}

// decisions in FP32 on the stored values: opacity below the minimum as a
// logit compare, size as a log-scale compare, selection on the mean statistic
__global__ void k_densify_classify(const float *__restrict__ log_scales, const float *__restrict__ logits,
                                   const float2 *__restrict__ stats, int64_t n, float thr, float min_logit,
                                   float log_dense, uint32_t *__restrict__ count, uint8_t *__restrict__ action)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float ls = fmaxf(log_scales[3 * i], fmaxf(log_scales[3 * i + 1], log_scales[3 * i + 2]));
        const float2 st = stats[i];
        const bool sel = __fdiv_rn(st.x, fmaxf(st.y, 1.f)) >= thr;
        uint8_t a = kKeep;
        if (logits[i] < min_logit) a = kPrune;
        else if (sel) a = ls > log_dense ? kSplit : kClone;
        action[i] = a;
        count[i] = a == kPrune ? 0u : (a == kKeep ? 1u : 2u);
    }
}

struct DensParams {
    const float *p[5], *m[5], *v[5];  // means, log_scales, quats, opacity_logits, sh
    float *np[5], *nm[5], *nv[5];
    int width[5];                     // floats per Gaussian in each group
};

__device__ __forceinline__ void copy_one(const DensParams &d, int64_t src, int64_t dst, bool moments)
{
#pragma unroll
    for (int g = 0; g < 5; g++) {
        const int w = d.width[g];
        for (int k = 0; k < w; k++) {
            d.np[g][dst * w + k] = d.p[g][src * w + k];
            d.nm[g][dst * w + k] = moments ? d.m[g][src * w + k] : 0.f;
            d.nv[g][dst * w + k] = moments ? d.v[g][src * w + k] : 0.f;
        }
    }
}

__global__ void k_densify_apply(DensParams d, int64_t n, const uint8_t *__restrict__ action,
                                const uint32_t *__restrict__ offsets, const float *__restrict__ noise, float log_shrink)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t a = action[i];
        if (a == kPrune) continue;
        const int64_t o = offsets[i];
        if (a == kKeep || a == kClone) {
            copy_one(d, i, o, true);
            if (a == kClone) copy_one(d, i, o + 1, false);
            continue;
        }
        // split: two samples of the Gaussian, scales divided by 1.6
        const float *q4 = d.p[2] + 4 * i;
        const float qn = rsqrtf(q4[0] * q4[0] + q4[1] * q4[1] + q4[2] * q4[2] + q4[3] * q4[3]);
        const float w = q4[0] * qn, x = q4[1] * qn, y = q4[2] * qn, z = q4[3] * qn;
        const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                            2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                            2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
        const float s[3] = {expf(d.p[1][3 * i]), expf(d.p[1][3 * i + 1]), expf(d.p[1][3 * i + 2])};
        for (int k = 0; k < 2; k++) {
            const int64_t t = o + k;
            copy_one(d, i, t, false);
            const float *e = noise + 6 * i + 3 * k;
            const float u[3] = {s[0] * e[0], s[1] * e[1], s[2] * e[2]};
#pragma unroll
            for (int r = 0; r < 3; r++) {
                d.np[0][3 * t + r] = d.p[0][3 * i + r] + fmaf(R[3 * r], u[0], fmaf(R[3 * r + 1], u[1], R[3 * r + 2] * u[2]));
                d.np[1][3 * t + r] = d.p[1][3 * i + r] - log_shrink;
            }
        }
    }
}

}  // namespace
}  // namespace splash

using namespace splash;

extern "C" splash_status splash_densify_plan(splash_ctx *ctx, const float *log_scales, const float *opacity_logits,
                                             const float *stats, int64_t n, const splash_densify_options *opt,
                                             int64_t *n_new, void *stream)
{
    if (!ctx || !opt || !n_new) return fail(SPLASH_ERR_INVALID_ARG, "null context, options or output");
    if (n < 0 || n >= ((int64_t)1 << 31)) return fail(SPLASH_ERR_INVALID_ARG, "n must be in [0, 2^31)");
    if (n > 0 && (!log_scales || !opacity_logits || !stats)) return fail(SPLASH_ERR_INVALID_ARG, "null buffer");
    if (!(opt->min_opacity > 0.f && opt->min_opacity < 1.f) || !(opt->percent_dense > 0.f) || !(opt->extent > 0.f) ||
        !(opt->grad_threshold >= 0.f))
        return fail(SPLASH_ERR_INVALID_ARG, "densify options out of range");
    cudaStream_t s = (cudaStream_t)stream;
    ctx->dens_n = -1;
    if (n == 0) {
        *n_new = 0;
        ctx->dens_n = 0;
        return SPLASH_OK;
    }
    ENSURE(ctx->dens_count, 4 * (size_t)n);
    ENSURE(ctx->dens_action, (size_t)n);
    ENSURE(ctx->dens_off, 4 * (size_t)n);
    ENSURE(ctx->dens_iota, 4 * (size_t)n);
    ENSURE(ctx->dens_sums, 4 * (size_t)(n / 4096 + 2));
    ENSURE(ctx->dens_total, 4 * 2);
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
    const float min_logit = (float)log((double)opt->min_opacity / (1.0 - (double)opt->min_opacity));
    const float log_dense = (float)log((double)opt->percent_dense * (double)opt->extent);
    k_iota<<<blocks, 256, 0, s>>>(ctx->dens_iota.as<uint32_t>(), n);
    k_densify_classify<<<blocks, 256, 0, s>>>(log_scales, opacity_logits, reinterpret_cast<const float2 *>(stats), n,
                                              opt->grad_threshold, min_logit, log_dense, ctx->dens_count.as<uint32_t>(),
                                              ctx->dens_action.as<uint8_t>());
    count_launch(2);
    launch_count_scan(n, ctx->dens_iota.as<uint32_t>(), ctx->dens_count.as<uint32_t>(), ctx->dens_off.as<uint32_t>(),
                      ctx->dens_sums.as<uint32_t>(), ctx->dens_total.as<uint32_t>(), s);
    uint32_t total = 0;
    SPLASH_CUDA_TRY(cudaMemcpyAsync(&total, ctx->dens_total.p, 4, cudaMemcpyDeviceToHost, s));
    SPLASH_CUDA_TRY(cudaStreamSynchronize(s));
    *n_new = total;
    ctx->dens_n = n;
    return SPLASH_OK;
}

extern "C" splash_status splash_densify_apply(splash_ctx *ctx, const splash_param_buffers *params,
                                              const splash_param_buffers *m, const splash_param_buffers *v, int64_t n,
                                              int32_t sh_degree, const float *noise, const splash_param_buffers *new_params,
                                              const splash_param_buffers *new_m, const splash_param_buffers *new_v,
                                              int64_t n_new, void *stream)
{
    if (!ctx || !params || !m || !v || !new_params || !new_m || !new_v) return fail(SPLASH_ERR_INVALID_ARG, "null argument");
    if (ctx->dens_n != n) return fail(SPLASH_ERR_STATE, "no densification plan for this many Gaussians");
    if (sh_degree < 0 || sh_degree > 3) return fail(SPLASH_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (n == 0) return SPLASH_OK;
    if (!noise) return fail(SPLASH_ERR_INVALID_ARG, "null noise");
    DensParams d{};
    const splash_param_buffers *src[3] = {params, m, v};
    const splash_param_buffers *dst[3] = {new_params, new_m, new_v};
    for (int w = 0; w < 3; w++) {
        const float *in[5] = {src[w]->means, src[w]->log_scales, src[w]->quats, src[w]->opacity_logits, src[w]->sh};
        float *out[5] = {dst[w]->means, dst[w]->log_scales, dst[w]->quats, dst[w]->opacity_logits, dst[w]->sh};
        for (int g = 0; g < 5; g++) {
            if (!in[g] || (n_new > 0 && !out[g])) return fail(SPLASH_ERR_INVALID_ARG, "null parameter or moment buffer");
            (w == 0 ? d.p : (w == 1 ? d.m : d.v))[g] = in[g];
            (w == 0 ? d.np : (w == 1 ? d.nm : d.nv))[g] = out[g];
        }
    }
    const int widths[5] = {3, 3, 4, 1, 3 * (sh_degree + 1) * (sh_degree + 1)};
    for (int g = 0; g < 5; g++) d.width[g] = widths[g];
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
    k_densify_apply<<<blocks, 256, 0, s>>>(d, n, ctx->dens_action.as<uint8_t>(), ctx->dens_off.as<uint32_t>(), noise,
                                           (float)log(1.6));
    count_launch();
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}
