// Water removal from a depth map (the application of Sec. I / Sec. V: the
// clean colour behind the water): the per-pixel image formation of Eq. 5,
// I = J exp(-beta_D z) + B_inf (1 - exp(-beta_B z)), inverted for J with the
// direct signal clipped at 0. A pure stream: 16 B read and 12 B written per
// pixel, float4 accesses over each plane.
#include <cuda_runtime.h>
#include <math.h>

#include "host.h"
#include "internal.cuh"

using namespace splash_host;

namespace splash {
namespace {

__device__ __forceinline__ float restore1(float I, float z, float bD, float bB, float B)
{
    const float direct = fmaxf(I - B * (-expm1f(-bB * z)), 0.f);
    return direct * expf(bD * z);
}

// Thread i handles pixels 4i .. 4i+3 of every channel (n4 = HW / 4 when HW
// and the pointers allow float4 access), then a scalar tail.
__global__ void __launch_bounds__(256) k_restore(const float *__restrict__ img, const float *__restrict__ depth,
                                                 const float *__restrict__ medium, int64_t HW, int vec,
                                                 float *__restrict__ out)
{
    float bD[3], bB[3], B[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        bD[c] = __ldg(medium + c);
        bB[c] = __ldg(medium + 3 + c);
        B[c] = __ldg(medium + 6 + c);
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n4 = vec ? HW / 4 : 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 z = reinterpret_cast<const float4 *>(depth)[i];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float4 v = reinterpret_cast<const float4 *>(img + c * HW)[i];
            float4 r;
            r.x = restore1(v.x, z.x, bD[c], bB[c], B[c]);
            r.y = restore1(v.y, z.y, bD[c], bB[c], B[c]);
            r.z = restore1(v.z, z.z, bD[c], bB[c], B[c]);
            r.w = restore1(v.w, z.w, bD[c], bB[c], B[c]);
            reinterpret_cast<float4 *>(out + c * HW)[i] = r;
        }
    }
    for (int64_t p = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += stride) {
        const float z = depth[p];
#pragma unroll
        for (int c = 0; c < 3; c++) out[c * HW + p] = restore1(img[c * HW + p], z, bD[c], bB[c], B[c]);
    }
}

}  // namespace
}  // namespace splash

using namespace splash;

extern "C" splash_status splash_restore(const float *image, const float *depth, const float *medium, int32_t width,
                                        int32_t height, float *out, void *stream)
{
    if (!image || !depth || !medium || !out) return fail(SPLASH_ERR_INVALID_ARG, "null image, depth, medium or out");
    if (width <= 0 || height <= 0 || (int64_t)width * height >= ((int64_t)1 << 31))
        return fail(SPLASH_ERR_INVALID_ARG, "image size must be positive and below 2^31 pixels");
    const int64_t HW = (int64_t)width * height;
    const bool vec = HW % 4 == 0 && ((reinterpret_cast<uintptr_t>(image) | reinterpret_cast<uintptr_t>(depth) |
                                      reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    const int64_t work = vec ? HW / 4 : HW;
    const int blocks = (int)std::min<int64_t>((work + 255) / 256, 148 * 16);
    k_restore<<<blocks, 256, 0, (cudaStream_t)stream>>>(image, depth, medium, HW, vec ? 1 : 0, out);
    count_launch();
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}
