// Photometric loss of the training step and its gradient in two tiled
// passes: L = mean|x - y| + lam (1 - mean SSIM(x, y)) (the Eq. 7 form,
// Sec. IV-C), SSIM with an 11x11 Gaussian window (sigma 1.5) and zero
// padding.
//   pass 1: blurred statistics mu_x, mu_y, E[x^2], E[y^2], E[xy] by a
//           separable convolution from a haloed shared-memory tile; per pixel
//           SSIM and its partials w.r.t. (mu_x, E[x^2], E[xy]), scaled by
//           dL/dSSIM_p = -lam / count; block partial sums of |x-y| and SSIM.
//   pass 2: dL/dx = blur(d_mu) + 2 x blur(d_xx) + y blur(d_xy) + sign(x-y)/count
//           (the window is symmetric, so the adjoint blur is the same blur).
// Both passes are HBM-bound streams over a few [C,H,W] maps.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.cuh"

namespace splash {
namespace {

constexpr int kR = 5;             // window radius
constexpr int kTX = 32, kTY = 16; // output tile
constexpr int kHX = kTX + 2 * kR, kHY = kTY + 2 * kR;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct Win {
    float w[2 * kR + 1];
};

__device__ __forceinline__ float load0(const float *p, int x, int y, int W, int H)
{
    return (x >= 0 && x < W && y >= 0 && y < H) ? p[y * W + x] : 0.f;
}

__global__ void __launch_bounds__(256) k_ssim_pass1(const float *__restrict__ X, const float *__restrict__ Y, int W, int H,
                                                    Win win, float wscale, float *__restrict__ d_mu,
                                                    float *__restrict__ d_xx, float *__restrict__ d_xy,
                                                    float *__restrict__ partial)
{
    __shared__ float sx[kHY][kHX], sy[kHY][kHX];
    __shared__ float h[5][kHY][kTX];
    __shared__ float s_red[2][8];
    const int c = blockIdx.z;
    const float *x = X + (size_t)c * W * H, *y = Y + (size_t)c * W * H;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int tid = threadIdx.x;
    for (int e = tid; e < kHY * kHX; e += 256) {
        const int r = e / kHX, q = e - r * kHX;
        sx[r][q] = load0(x, x0 - kR + q, y0 - kR + r, W, H);
        sy[r][q] = load0(y, x0 - kR + q, y0 - kR + r, W, H);
    }
    __syncthreads();
    for (int e = tid; e < kHY * kTX; e += 256) {
        const int r = e / kTX, q = e - r * kTX;
        float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * kR; k++) {
            const float u = sx[r][q + k], v = sy[r][q + k], w = win.w[k];
            a = fmaf(w, u, a);
            b = fmaf(w, v, b);
            aa = fmaf(w, u * u, aa);
            bb = fmaf(w, v * v, bb);
            ab = fmaf(w, u * v, ab);
        }
        h[0][r][q] = a; h[1][r][q] = b; h[2][r][q] = aa; h[3][r][q] = bb; h[4][r][q] = ab;
    }
    __syncthreads();
    float l1 = 0.f, ss = 0.f;
    for (int e = tid; e < kTY * kTX; e += 256) {
        const int r = e / kTX, q = e - r * kTX;
        const int gx = x0 + q, gy = y0 + r;
        if (gx >= W || gy >= H) continue;
        float m1 = 0.f, m2 = 0.f, e11 = 0.f, e22 = 0.f, e12 = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * kR; k++) {
            const float w = win.w[k];
            m1 = fmaf(w, h[0][r + k][q], m1);
            m2 = fmaf(w, h[1][r + k][q], m2);
            e11 = fmaf(w, h[2][r + k][q], e11);
            e22 = fmaf(w, h[3][r + k][q], e22);
            e12 = fmaf(w, h[4][r + k][q], e12);
        }
        const float sxx = e11 - m1 * m1, syy = e22 - m2 * m2, sxy = e12 - m1 * m2;
        const float A1 = 2.f * m1 * m2 + kC1, A2 = 2.f * sxy + kC2;
        const float B1 = m1 * m1 + m2 * m2 + kC1, B2 = sxx + syy + kC2;
        const float inv = 1.f / (B1 * B2);
        const float S = A1 * A2 * inv;
        // partials of S(m1, e11, e12) with m2, e22 fixed
        const float dm1 = (2.f * m2 * (A2 - A1) - 2.f * m1 * S * (B2 - B1)) * inv;
        const float de11 = -S / B2;
        const float de12 = 2.f * A1 * inv;
        const size_t p = (size_t)c * W * H + (size_t)gy * W + gx;
        d_mu[p] = wscale * dm1;
        d_xx[p] = wscale * de11;
        d_xy[p] = wscale * de12;
        l1 += fabsf(sx[r + kR][q + kR] - sy[r + kR][q + kR]);
        ss += S;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l1 += __shfl_xor_sync(0xffffffffu, l1, o);
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
    }
    if ((tid & 31) == 0) {
        s_red[0][tid >> 5] = l1;
        s_red[1][tid >> 5] = ss;
    }
    __syncthreads();
    if (tid < 2) {
        float v = 0.f;
#pragma unroll
        for (int i = 0; i < 8; i++) v += s_red[tid][i];
        const int b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partial[2 * b + tid] = v;
    }
}

__global__ void __launch_bounds__(256) k_ssim_pass2(const float *__restrict__ X, const float *__restrict__ Y, int W, int H,
                                                    Win win, float l1scale, const float *__restrict__ d_mu,
                                                    const float *__restrict__ d_xx, const float *__restrict__ d_xy,
                                                    float *__restrict__ grad)
{
    __shared__ float s[3][kHY][kHX];
    __shared__ float h[3][kHY][kTX];
    const int c = blockIdx.z;
    const size_t off = (size_t)c * W * H;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int tid = threadIdx.x;
    for (int e = tid; e < kHY * kHX; e += 256) {
        const int r = e / kHX, q = e - r * kHX;
        const int gx = x0 - kR + q, gy = y0 - kR + r;
        s[0][r][q] = load0(d_mu + off, gx, gy, W, H);
        s[1][r][q] = load0(d_xx + off, gx, gy, W, H);
        s[2][r][q] = load0(d_xy + off, gx, gy, W, H);
    }
    __syncthreads();
    for (int e = tid; e < kHY * kTX; e += 256) {
        const int r = e / kTX, q = e - r * kTX;
        float a = 0.f, b = 0.f, d = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * kR; k++) {
            const float w = win.w[k];
            a = fmaf(w, s[0][r][q + k], a);
            b = fmaf(w, s[1][r][q + k], b);
            d = fmaf(w, s[2][r][q + k], d);
        }
        h[0][r][q] = a; h[1][r][q] = b; h[2][r][q] = d;
    }
    __syncthreads();
    for (int e = tid; e < kTY * kTX; e += 256) {
        const int r = e / kTX, q = e - r * kTX;
        const int gx = x0 + q, gy = y0 + r;
        if (gx >= W || gy >= H) continue;
        float a = 0.f, b = 0.f, d = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * kR; k++) {
            const float w = win.w[k];
            a = fmaf(w, h[0][r + k][q], a);
            b = fmaf(w, h[1][r + k][q], b);
            d = fmaf(w, h[2][r + k][q], d);
        }
        const size_t p = off + (size_t)gy * W + gx;
        const float xv = X[p], yv = Y[p];
        const float diff = xv - yv;
        const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
        grad[p] = a + 2.f * xv * b + yv * d + sgn * l1scale;
    }
}

// Final stage: the kColsumParts partial rows of (sum |x-y|, sum SSIM) in a
// fixed order, then the loss.
__global__ void k_loss_final(const float *__restrict__ part, double inv_count, float lam, float *__restrict__ loss)
{
    if (threadIdx.x != 0) return;
    double l1 = 0.0, ss = 0.0;
    for (int p = 0; p < kColsumParts; p++) {
        l1 += part[2 * p];
        ss += part[2 * p + 1];
    }
    *loss = (float)(l1 * inv_count + (double)lam * (1.0 - ss * inv_count));
}

Win make_window()
{
    Win w;
    double sum = 0.0, g[2 * kR + 1];
    for (int k = 0; k <= 2 * kR; k++) {
        const double t = k - kR;
        g[k] = exp(-t * t / (2.0 * 1.5 * 1.5));
        sum += g[k];
    }
    for (int k = 0; k <= 2 * kR; k++) w.w[k] = (float)(g[k] / sum);
    return w;
}

}  // namespace

size_t ssim_scratch_floats(int C, int H, int W)
{
    const size_t nb = (size_t)((W + kTX - 1) / kTX) * ((H + kTY - 1) / kTY) * C;
    return 3 * (size_t)C * H * W + 2 * nb + 2 * kColsumParts + 64;
}

void launch_ssim_loss(const float *img, const float *tgt, int C, int H, int W, float lam, float *loss, float *grad,
                      float *scratch, cudaStream_t s)
{
    const dim3 grid((W + kTX - 1) / kTX, (H + kTY - 1) / kTY, C);
    const size_t n = (size_t)C * H * W;
    float *d_mu = scratch, *d_xx = scratch + n, *d_xy = scratch + 2 * n, *partial = scratch + 3 * n;
    const Win win = make_window();
    const double inv = 1.0 / (double)n;
    k_ssim_pass1<<<grid, 256, 0, s>>>(img, tgt, W, H, win, (float)(-lam * inv), d_mu, d_xx, d_xy, partial);
    count_launch();
    const int nb = grid.x * grid.y * grid.z;
    float *part2 = partial + 2 * nb;
    launch_colsum_partial(partial, nb, 2, part2, s);
    k_loss_final<<<1, 32, 0, s>>>(part2, inv, lam, loss);
    count_launch();
    if (grad) k_ssim_pass2<<<grid, 256, 0, s>>>(img, tgt, W, H, win, (float)inv, d_mu, d_xx, d_xy, grad);
    if (grad) count_launch();
}

}  // namespace splash
