// The paper-literal pixel form of the water (Eq. 5 with the Eq. 6 depth):
//   C = J e^{-beta_D z} + B_inf (1 - e^{-beta_B z}),
//   J = sum_i c_i alpha_i T_i,  z = sum_i d_i alpha_i T_i / sum_i alpha_i T_i (z_far if empty).
// J and z are what the rasterizer produces with a zero medium (every
// effective colour is then the plain colour and no backscatter term is
// left), so this form reuses the render and its adjoint unchanged:
//   forward:  zero-medium render, then k_pixel_epilogue per pixel;
//   backward: k_pixel_adjoint turns dL/dC into the upstream of the
//             zero-medium render, dL/dJ = G e^{-beta_D z} and the depth
//             gradient dL/dz += sum_ch G (B_inf beta_B e^{-beta_B z} -
//             beta_D J e^{-beta_D z}) (where something composites), and
//             reduces the medium gradient per block; then the zero-medium
//             backward (with its depth path) and a fixed-order medium sum.
#include <cuda_runtime.h>
#include <math.h>

#include "host.h"
#include "internal.cuh"

using namespace splash_host;

namespace splash {
namespace {

constexpr int kPixThreads = 256;
constexpr int kPixBlocksMax = 148 * 8;

__global__ void __launch_bounds__(kPixThreads) k_pixel_epilogue(float *__restrict__ image, const float *__restrict__ zhat,
                                                                const float *__restrict__ medium, int64_t HW,
                                                                float *__restrict__ J)
{
    float bD[3], bB[3], B[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        bD[c] = __ldg(medium + c);
        bB[c] = __ldg(medium + 3 + c);
        B[c] = __ldg(medium + 6 + c);
    }
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += (int64_t)gridDim.x * blockDim.x) {
        const float z = zhat[p];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float j = image[c * HW + p];
            J[c * HW + p] = j;
            image[c * HW + p] = fmaf(j, expf(-bD[c] * z), B[c] * -expm1f(-bB[c] * z));
        }
    }
}

// Per pixel: the zero-medium upstream (G a, depth gradient) and the medium
// gradient terms; per block: the nine medium sums (fixed order) to block_med.
__global__ void __launch_bounds__(kPixThreads) k_pixel_adjoint(
    const float *__restrict__ G, const float *__restrict__ gdepth, const float *__restrict__ J,
    const float *__restrict__ zhat, const float *__restrict__ acc_alpha, const float *__restrict__ medium, int64_t HW,
    float *__restrict__ G_out, float *__restrict__ gz_out, float *__restrict__ block_med)
{
    __shared__ float s_w[kPixThreads / 32][9];
    float bD[3], bB[3], B[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        bD[c] = __ldg(medium + c);
        bB[c] = __ldg(medium + 3 + c);
        B[c] = __ldg(medium + 6 + c);
    }
    float m[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += (int64_t)gridDim.x * blockDim.x) {
        const float z = zhat[p];
        float dz = 0.f;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float g = G[c * HW + p], j = J[c * HW + p];
            const float a = expf(-bD[c] * z), em1 = expm1f(-bB[c] * z), b = 1.f + em1;
            G_out[c * HW + p] = g * a;
            dz = fmaf(g, B[c] * bB[c] * b - bD[c] * j * a, dz);
            m[c] = fmaf(-g * z, j * a, m[c]);      // beta_D
            m[3 + c] = fmaf(g * B[c], z * b, m[3 + c]);  // beta_B
            m[6 + c] = fmaf(g, -em1, m[6 + c]);    // B_inf
        }
        // with nothing composited z = z_far does not move
        gz_out[p] = (acc_alpha[p] > 0.f ? dz : 0.f) + (gdepth ? gdepth[p] : 0.f);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 9; k++) {
        float v = m[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_w[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < kPixThreads / 32; w++) v += s_w[w][threadIdx.x];
        block_med[blockIdx.x * 9 + threadIdx.x] = v;
    }
}

// d_medium[j] = sum over blocks of block_med[b][j]: warp j, lane l adds
// blocks l, l + 32, ... in order, then a fixed butterfly (deterministic)
__global__ void __launch_bounds__(9 * 32) k_pixel_medium_final(const float *__restrict__ block_med, int nblocks,
                                                               float *__restrict__ d_medium)
{
    const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float v = 0.f;
    for (int b = lane; b < nblocks; b += 32) v += block_med[b * 9 + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) d_medium[j] = v;
}

int pixel_blocks(int64_t HW) { return (int)std::min<int64_t>((HW + kPixThreads - 1) / kPixThreads, kPixBlocksMax); }

splash_status zero_medium(splash_ctx *ctx, cudaStream_t s, const float **out)
{
    if (!ctx->zero16.p) {
        ENSURE(ctx->zero16, 16 * sizeof(float));
        SPLASH_CUDA_TRY(cudaMemsetAsync(ctx->zero16.p, 0, 16 * sizeof(float), s));
    }
    *out = ctx->zero16.as<float>();
    return SPLASH_OK;
}

}  // namespace

void launch_pixel_medium_final(const float *partials, int nblocks, float *d_medium, cudaStream_t s)
{
    k_pixel_medium_final<<<1, 9 * 32, 0, s>>>(partials, nblocks, d_medium);
    count_launch();
}

}  // namespace splash

using namespace splash;

extern "C" splash_status splash_render_forward_pixel(splash_ctx *ctx, splash_state *st, const splash_gaussians *g,
                                                     const float *medium, const splash_camera *cam, float *image,
                                                     float *depth, float *depth01, void *stream)
{
    if (!ctx || !st || st->ctx != ctx) return fail(SPLASH_ERR_INVALID_ARG, "bad context or state");
    if (!medium || !image) return fail(SPLASH_ERR_INVALID_ARG, "null medium or image");
    if (!cam) return fail(SPLASH_ERR_INVALID_ARG, "null camera");
    cudaStream_t s = (cudaStream_t)stream;
    const float *zero = nullptr;
    splash_status rc;
    if ((rc = zero_medium(ctx, s, &zero)) != SPLASH_OK) return rc;
    if ((rc = splash_render_forward(ctx, st, g, zero, cam, image, depth, depth01, stream)) != SPLASH_OK) return rc;
    const int64_t HW = (int64_t)cam->width * cam->height;
    ENSURE(st->pixJ, 12 * (size_t)HW);
    k_pixel_epilogue<<<pixel_blocks(HW), kPixThreads, 0, s>>>(image, st->zh.as<float>(), medium, HW, st->pixJ.as<float>());
    count_launch();
    SPLASH_CUDA_TRY(cudaGetLastError());
    st->pixel_forward = true;
    return SPLASH_OK;
}

extern "C" splash_status splash_render_backward_pixel(splash_ctx *ctx, splash_state *st, const splash_gaussians *g,
                                                      const float *medium, const splash_camera *cam,
                                                      const float *dL_dimage, const float *dL_ddepth,
                                                      const float *dL_ddepth01, const splash_grads *grads,
                                                      void *stream)
{
    if (!ctx || !st || st->ctx != ctx) return fail(SPLASH_ERR_INVALID_ARG, "bad context or state");
    if (!medium || !dL_dimage || !grads || !cam) return fail(SPLASH_ERR_INVALID_ARG, "null medium, dL_dimage, grads or camera");
    if (!st->has_forward || !st->pixel_forward || st->W != cam->width || st->H != cam->height)
        return fail(SPLASH_ERR_STATE, "backward does not match the last pixel-form forward on this state");
    cudaStream_t s = (cudaStream_t)stream;
    const float *zero = nullptr;
    splash_status rc;
    if ((rc = zero_medium(ctx, s, &zero)) != SPLASH_OK) return rc;
    const int64_t HW = (int64_t)cam->width * cam->height;
    const int nb = pixel_blocks(HW);
    ENSURE(st->pixG, 12 * (size_t)HW);
    ENSURE(st->pixgz, 4 * (size_t)HW);
    ENSURE(st->pixmed, 4 * 9 * (size_t)nb);
    k_pixel_adjoint<<<nb, kPixThreads, 0, s>>>(dL_dimage, dL_ddepth, st->pixJ.as<float>(), st->zh.as<float>(),
                                               st->aA.as<float>(), medium, HW, st->pixG.as<float>(),
                                               st->pixgz.as<float>(), st->pixmed.as<float>());
    count_launch();
    SPLASH_CUDA_TRY(cudaGetLastError());
    splash_grads gs = *grads;
    gs.medium = nullptr;  // the zero-medium render's own water terms do not apply
    if ((rc = render_backward_impl(ctx, st, g, zero, cam, st->pixG.as<float>(), st->pixgz.as<float>(), dL_ddepth01,
                                   &gs, stream)) != SPLASH_OK)
        return rc;
    if (grads->medium) launch_pixel_medium_final(st->pixmed.as<float>(), nb, grads->medium, s);
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}

extern "C" splash_status splash_render_backward_adam_pixel(splash_ctx *ctx, splash_state *st,
                                                           const splash_param_buffers *params, int64_t n,
                                                           int32_t sh_degree, const splash_camera *cam,
                                                           const float *dL_dimage, const float *dL_ddepth,
                                                           const float *dL_ddepth01, const splash_adam_config *adam,
                                                           float *grad_medium, void *stream)
{
    if (!ctx || !st || st->ctx != ctx) return fail(SPLASH_ERR_INVALID_ARG, "bad context or state");
    if (!params || !params->medium || !dL_dimage || !cam || !adam)
        return fail(SPLASH_ERR_INVALID_ARG, "null params, medium, dL_dimage, camera or adam config");
    if (!st->has_forward || !st->pixel_forward || st->W != cam->width || st->H != cam->height)
        return fail(SPLASH_ERR_STATE, "backward does not match the last pixel-form forward on this state");
    cudaStream_t s = (cudaStream_t)stream;
    const float *zero = nullptr;
    splash_status rc;
    if ((rc = zero_medium(ctx, s, &zero)) != SPLASH_OK) return rc;
    const int64_t HW = (int64_t)cam->width * cam->height;
    const int nb = pixel_blocks(HW);
    ENSURE(st->pixG, 12 * (size_t)HW);
    ENSURE(st->pixgz, 4 * (size_t)HW);
    ENSURE(st->pixmed, 4 * 9 * (size_t)nb);
    k_pixel_adjoint<<<nb, kPixThreads, 0, s>>>(dL_dimage, dL_ddepth, st->pixJ.as<float>(), st->zh.as<float>(),
                                               st->aA.as<float>(), params->medium, HW, st->pixG.as<float>(),
                                               st->pixgz.as<float>(), st->pixmed.as<float>());
    count_launch();
    SPLASH_CUDA_TRY(cudaGetLastError());
    return backward_adam_impl(ctx, st, params, n, sh_degree, cam, st->pixG.as<float>(), st->pixgz.as<float>(),
                              dL_ddepth01, adam, grad_medium, stream, zero, st->pixmed.as<float>(), nb);
}
