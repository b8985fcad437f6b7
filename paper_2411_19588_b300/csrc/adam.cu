// One Adam step (Kingma & Ba) over up to eight parameter groups in a single
// launch: Sec. IV-C optimises the Gaussian and medium parameters with Adam
// at per-group learning rates (appendix, "Experimental Setup"). A pure
// stream: per element it reads p, g, m, v and writes p, m, v (28 B), so it is
// HBM-bound; 16-byte vector accesses where the group allows.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace splash {
namespace {

constexpr int kAdamThreads = 256;
constexpr int kAdamVec = 4;
constexpr int kAdamPerBlock = kAdamThreads * kAdamVec * 4;  // elements per block

struct AdamTable {
    splash_adam_group g[SPLASH_ADAM_MAX_GROUPS];
    int64_t block_start[SPLASH_ADAM_MAX_GROUPS + 1];
    int n;
    AdamHyper h;
};

__device__ __forceinline__ void adam1(float &p, float g, float &m, float &v, float lr, const AdamTable &t,
                                      const splash_adam_group &G)
{
    adam_update(p, g, m, v, lr, t.h);
    if (G.has_clamp) p = fmaxf(p, G.clamp_min);
}

__global__ void __launch_bounds__(kAdamThreads) k_adam(AdamTable t)
{
    int gi = 0;
    while (gi + 1 < t.n && (int64_t)blockIdx.x >= t.block_start[gi + 1]) gi++;
    const splash_adam_group &G = t.g[gi];
    const int64_t base = ((int64_t)blockIdx.x - t.block_start[gi]) * kAdamPerBlock;
    const bool vec = ((reinterpret_cast<uintptr_t>(G.param) | reinterpret_cast<uintptr_t>(G.grad) |
                       reinterpret_cast<uintptr_t>(G.m) | reinterpret_cast<uintptr_t>(G.v)) & 15) == 0;
    const float lr = G.lr;
    if (vec) {
#pragma unroll
        for (int it = 0; it < 4; it++) {
            const int64_t i = base + ((int64_t)it * kAdamThreads + threadIdx.x) * kAdamVec;
            if (i + kAdamVec <= G.n) {
                float4 p = *reinterpret_cast<float4 *>(G.param + i);
                const float4 g = *reinterpret_cast<const float4 *>(G.grad + i);
                float4 m = *reinterpret_cast<float4 *>(G.m + i);
                float4 v = *reinterpret_cast<float4 *>(G.v + i);
                adam1(p.x, g.x, m.x, v.x, lr, t, G);
                adam1(p.y, g.y, m.y, v.y, lr, t, G);
                adam1(p.z, g.z, m.z, v.z, lr, t, G);
                adam1(p.w, g.w, m.w, v.w, lr, t, G);
                *reinterpret_cast<float4 *>(G.param + i) = p;
                *reinterpret_cast<float4 *>(G.m + i) = m;
                *reinterpret_cast<float4 *>(G.v + i) = v;
            } else {
                for (int64_t e = i; e < G.n; e++) adam1(G.param[e], G.grad[e], G.m[e], G.v[e], lr, t, G);
            }
        }
    } else {
        for (int64_t e = base + threadIdx.x; e < min(G.n, base + kAdamPerBlock); e += kAdamThreads)
            adam1(G.param[e], G.grad[e], G.m[e], G.v[e], lr, t, G);
    }
}

}  // namespace
}  // namespace splash

extern "C" splash_status splash_adam_step(const splash_adam_group *groups, int32_t n_groups, int32_t step, float beta1,
                                          float beta2, float eps, void *stream)
{
    using namespace splash;
    if (!groups || n_groups < 1 || n_groups > SPLASH_ADAM_MAX_GROUPS || step < 1) {
        splash_set_error("splash_adam_step: bad group table or step");
        return SPLASH_ERR_INVALID_ARG;
    }
    AdamTable t{};
    t.n = n_groups;
    t.h = make_adam_hyper(beta1, beta2, eps, step);
    int64_t blocks = 0;
    for (int i = 0; i < n_groups; i++) {
        const splash_adam_group &G = groups[i];
        if (G.n < 0 || (G.n > 0 && (!G.param || !G.grad || !G.m || !G.v))) {
            splash_set_error("splash_adam_step: group with null buffer or negative size");
            return SPLASH_ERR_INVALID_ARG;
        }
        t.g[i] = G;
        t.block_start[i] = blocks;
        blocks += (G.n + kAdamPerBlock - 1) / kAdamPerBlock;
    }
    t.block_start[n_groups] = blocks;
    if (blocks == 0) return SPLASH_OK;
    k_adam<<<(unsigned)blocks, kAdamThreads, 0, (cudaStream_t)stream>>>(t);
    count_launch();
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}

// Opacity reset of the appendix's schedule (every 3,000 iterations in the
// paper, as in 3DGS): opacities above max_opacity are set to it (a cap on the
// logit), and the opacity group's Adam moments restart at zero.
namespace {
__global__ void k_opacity_reset(float *__restrict__ logits, float *__restrict__ m, float *__restrict__ v, int64_t n,
                                float cap)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        logits[i] = fminf(logits[i], cap);
        if (m) m[i] = 0.f;
        if (v) v[i] = 0.f;
    }
}
}  // namespace

extern "C" splash_status splash_opacity_reset(float *logits, float *adam_m, float *adam_v, int64_t n, float max_opacity,
                                              void *stream)
{
    using namespace splash;
    if (n < 0 || (n > 0 && !logits)) {
        splash_set_error("splash_opacity_reset: null logits or negative n");
        return SPLASH_ERR_INVALID_ARG;
    }
    if (!(max_opacity > 0.f && max_opacity < 1.f)) {
        splash_set_error("splash_opacity_reset: max_opacity must be in (0, 1)");
        return SPLASH_ERR_INVALID_ARG;
    }
    if (n == 0) return SPLASH_OK;
    const float cap = (float)log((double)max_opacity / (1.0 - (double)max_opacity));
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 8);
    k_opacity_reset<<<blocks, 256, 0, (cudaStream_t)stream>>>(logits, adam_m, adam_v, n, cap);
    count_launch();
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}
