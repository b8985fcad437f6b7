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
// Each 1-D window pass is register-blocked: a thread slides the 11 taps over
// four consecutive outputs, so a few shared loads feed many FMAs.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.cuh"

namespace splash {
namespace {

constexpr int kR = 5;             // window radius
constexpr int kTX = 32, kTY = 32; // output tile
constexpr int kHX = kTX + 2 * kR, kHY = kTY + 2 * kR;  // haloed tile (42 x 42)
constexpr int kSX = 44;           // row stride of the haloed tile: float4 rows, conflict-free
constexpr int kRun = 4;           // consecutive outputs per thread in each 1-D pass
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

struct Win {
    float w[2 * kR + 1];
};

__device__ __forceinline__ float load0(const float *p, int x, int y, int W, int H)
{
    return (x >= 0 && x < W && y >= 0 && y < H) ? p[(size_t)y * W + x] : 0.f;
}

// kRun horizontal window sums starting at column 4j of row r of a haloed tile:
// the 14 inputs come in as four float4 loads.
__device__ __forceinline__ void hrun(const float (*t)[kSX], int r, int j, float (&u)[16])
{
    const float4 *row = reinterpret_cast<const float4 *>(&t[r][4 * j]);
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const float4 v = row[i];
        u[4 * i] = v.x;
        u[4 * i + 1] = v.y;
        u[4 * i + 2] = v.z;
        u[4 * i + 3] = v.w;
    }
}

// Pass 1: blurred statistics (separable, register-blocked), per-pixel SSIM
// and its partials w.r.t. (mu_x, E[x^2], E[xy]) scaled by dL/dSSIM_p, block
// sums of |x - y| and SSIM.
__global__ void __launch_bounds__(256) k_ssim_pass1(const float *__restrict__ X, const float *__restrict__ Y, int W, int H,
                                                    Win win, float wscale, float *__restrict__ d_mu,
                                                    float *__restrict__ d_xx, float *__restrict__ d_xy,
                                                    float *__restrict__ partial)
{
    __shared__ __align__(16) float sx[kHY][kSX];
    __shared__ __align__(16) float sy[kHY][kSX];
    __shared__ float h[5][kHY][kTX + 1];
    __shared__ float s_red[2][8];
    const int c = blockIdx.z;
    const float *x = X + (size_t)c * W * H, *y = Y + (size_t)c * W * H;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int tid = threadIdx.x;
    {  // haloed tiles: every load of this thread in flight before any store
        constexpr int NL = (kHY * kSX + 255) / 256;
        float lx[NL], ly[NL];
#pragma unroll
        for (int t = 0; t < NL; t++) {
            const int e = tid + 256 * t, r = e / kSX, q = e - r * kSX;
            const bool in = e < kHY * kSX && q < kHX;
            lx[t] = in ? load0(x, x0 - kR + q, y0 - kR + r, W, H) : 0.f;
            ly[t] = in ? load0(y, x0 - kR + q, y0 - kR + r, W, H) : 0.f;
        }
#pragma unroll
        for (int t = 0; t < NL; t++) {
            const int e = tid + 256 * t, r = e / kSX, q = e - r * kSX;
            if (e < kHY * kSX) {
                sx[r][q] = lx[t];
                sy[r][q] = ly[t];
            }
        }
    }
    __syncthreads();
    // horizontal: kHY rows x (kTX / kRun) runs
    for (int e = tid; e < kHY * (kTX / kRun); e += 256) {
        const int r = e / (kTX / kRun), j = e - r * (kTX / kRun);
        float u[16], v[16], uu[16], vv[16], uv[16];
        hrun(sx, r, j, u);
        hrun(sy, r, j, v);
#pragma unroll
        for (int i = 0; i < kRun + 2 * kR; i++) {
            uu[i] = u[i] * u[i];
            vv[i] = v[i] * v[i];
            uv[i] = u[i] * v[i];
        }
#pragma unroll
        for (int i = 0; i < kRun; i++) {
            float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
            for (int k = 0; k <= 2 * kR; k++) {
                const float w = win.w[k];
                a = fmaf(w, u[i + k], a);
                b = fmaf(w, v[i + k], b);
                aa = fmaf(w, uu[i + k], aa);
                bb = fmaf(w, vv[i + k], bb);
                ab = fmaf(w, uv[i + k], ab);
            }
            const int q = kRun * j + i;
            h[0][r][q] = a; h[1][r][q] = b; h[2][r][q] = aa; h[3][r][q] = bb; h[4][r][q] = ab;
        }
    }
    __syncthreads();
    // vertical: thread (column q, run b) makes rows kRun b .. kRun b + kRun - 1
    const int q = tid & (kTX - 1), rb = tid / kTX;
    float st[5][kRun];
#pragma unroll
    for (int m = 0; m < 5; m++) {
        float col[kRun + 2 * kR];
#pragma unroll
        for (int i = 0; i < kRun + 2 * kR; i++) col[i] = h[m][kRun * rb + i][q];
#pragma unroll
        for (int i = 0; i < kRun; i++) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k <= 2 * kR; k++) acc = fmaf(win.w[k], col[i + k], acc);
            st[m][i] = acc;
        }
    }
    float l1 = 0.f, ss = 0.f;
    const int gx = x0 + q;
#pragma unroll
    for (int i = 0; i < kRun; i++) {
        const int r = kRun * rb + i, gy = y0 + r;
        if (gx >= W || gy >= H) continue;
        const float m1 = st[0][i], m2 = st[1][i], e11 = st[2][i], e22 = st[3][i], e12 = st[4][i];
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

// Pass 2: dL/dx = blur(d_mu) + 2 x blur(d_xx) + y blur(d_xy) + sign(x - y) / count
// (the window is symmetric, so the adjoint blur is the same blur).
__global__ void __launch_bounds__(256) k_ssim_pass2(const float *__restrict__ X, const float *__restrict__ Y, int W, int H,
                                                    Win win, float l1scale, const float *__restrict__ d_mu,
                                                    const float *__restrict__ d_xx, const float *__restrict__ d_xy,
                                                    float *__restrict__ grad)
{
    __shared__ __align__(16) float s[3][kHY][kSX];
    __shared__ float h[3][kHY][kTX + 1];
    const int c = blockIdx.z;
    const size_t off = (size_t)c * W * H;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int tid = threadIdx.x;
    {  // haloed tiles: every load of this thread in flight before any store
        constexpr int NL = (kHY * kSX + 255) / 256;
        float l0[NL], l1[NL], l2[NL];
#pragma unroll
        for (int t = 0; t < NL; t++) {
            const int e = tid + 256 * t, r = e / kSX, q = e - r * kSX;
            const int gx = x0 - kR + q, gy = y0 - kR + r;
            const bool in = e < kHY * kSX && q < kHX;
            l0[t] = in ? load0(d_mu + off, gx, gy, W, H) : 0.f;
            l1[t] = in ? load0(d_xx + off, gx, gy, W, H) : 0.f;
            l2[t] = in ? load0(d_xy + off, gx, gy, W, H) : 0.f;
        }
#pragma unroll
        for (int t = 0; t < NL; t++) {
            const int e = tid + 256 * t, r = e / kSX, q = e - r * kSX;
            if (e < kHY * kSX) {
                s[0][r][q] = l0[t];
                s[1][r][q] = l1[t];
                s[2][r][q] = l2[t];
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < kHY * (kTX / kRun); e += 256) {
        const int r = e / (kTX / kRun), j = e - r * (kTX / kRun);
#pragma unroll
        for (int m = 0; m < 3; m++) {
            float u[16];
            hrun(s[m], r, j, u);
#pragma unroll
            for (int i = 0; i < kRun; i++) {
                float a = 0.f;
#pragma unroll
                for (int k = 0; k <= 2 * kR; k++) a = fmaf(win.w[k], u[i + k], a);
                h[m][r][kRun * j + i] = a;
            }
        }
    }
    __syncthreads();
    const int q = tid & (kTX - 1), rb = tid / kTX;
    float bl[3][kRun];
#pragma unroll
    for (int m = 0; m < 3; m++) {
        float col[kRun + 2 * kR];
#pragma unroll
        for (int i = 0; i < kRun + 2 * kR; i++) col[i] = h[m][kRun * rb + i][q];
#pragma unroll
        for (int i = 0; i < kRun; i++) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k <= 2 * kR; k++) acc = fmaf(win.w[k], col[i + k], acc);
            bl[m][i] = acc;
        }
    }
    const int gx = x0 + q;
#pragma unroll
    for (int i = 0; i < kRun; i++) {
        const int gy = y0 + kRun * rb + i;
        if (gx >= W || gy >= H) continue;
        const size_t p = off + (size_t)gy * W + gx;
        const float xv = X[p], yv = Y[p];
        const float diff = xv - yv;
        const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
        grad[p] = bl[0][i] + 2.f * xv * bl[1][i] + yv * bl[2][i] + sgn * l1scale;
    }
}

// Final stage: the kColsumParts partial rows of (sum |x-y|, sum SSIM) in a
// fixed order, then the loss.
// one warp: lane l adds partial rows l, l + 32, ... (FP64), then a fixed
// butterfly; the FP64 add chain stays short on this GPU's narrow FP64 pipe
__global__ void k_loss_final(const float *__restrict__ part, double inv_count, float lam, float *__restrict__ loss)
{
    const int lane = threadIdx.x;
    double l1 = 0.0, ss = 0.0;
    for (int p = lane; p < kColsumParts; p += 32) {
        l1 += part[2 * p];
        ss += part[2 * p + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l1 += __shfl_xor_sync(0xffffffffu, l1, o);
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
    }
    if (lane == 0) *loss = (float)(l1 * inv_count + (double)lam * (1.0 - ss * inv_count));
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
