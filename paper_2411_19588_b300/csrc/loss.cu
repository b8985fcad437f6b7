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
// four consecutive outputs, so a few shared loads feed many FMAs; pairs of
// statistics share one packed FP32x2 FMA per tap.
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

// Whether a CTA's haloed window lies inside the image with 16-byte aligned
// rows (the maps' base addresses a, b, c included): then it is read as the
// aligned columns x0 - 8 .. x0 + 39 (twelve 16-byte loads per row), with no
// per-element bounds checks.
__device__ __forceinline__ bool window_inside(int x0, int y0, int W, int H, const void *a, const void *b, const void *c)
{
    const uintptr_t base = reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(c);
    return x0 >= 8 && x0 + kTX + 8 <= W && y0 >= kR && y0 + kTY + kR <= H && (W & 3) == 0 && (base & 15) == 0;
}

// The haloed window of NMAP maps of an inside CTA into shared memory: every
// 16-byte load in flight before any store; element e of the load at aligned
// column m lands in window column 4 m - 3 + e (kept while inside the row).
template <int NMAP>
__device__ __forceinline__ void load_window_inside(const float *const (&src)[NMAP], float (*const (&dst)[NMAP])[kSX],
                                                   int x0, int y0, int W)
{
    constexpr int Q4 = 12;                  // 16-byte columns per window row
    constexpr int NV = kHY * Q4;            // per map
    constexpr int NI = (NV + 255) / 256;
    const int tid = threadIdx.x;
    float4 v[NMAP][NI];
#pragma unroll
    for (int t = 0; t < NI; t++) {
        const int idx = tid + 256 * t;
        if (idx >= NV) continue;
        const int r = idx / Q4, m = idx - r * Q4;
        const size_t o = (size_t)(y0 - kR + r) * W + (x0 - 8);
#pragma unroll
        for (int k = 0; k < NMAP; k++) v[k][t] = reinterpret_cast<const float4 *>(src[k] + o)[m];
    }
#pragma unroll
    for (int t = 0; t < NI; t++) {
        const int idx = tid + 256 * t;
        if (idx >= NV) continue;
        const int r = idx / Q4, m = idx - r * Q4;
#pragma unroll
        for (int k = 0; k < NMAP; k++) {
            const float e4[4] = {v[k][t].x, v[k][t].y, v[k][t].z, v[k][t].w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int q = 4 * m - 3 + e;
                if (q >= 0 && q < kSX) dst[k][r][q] = e4[e];
            }
        }
    }
}

// The window's taps as packed pairs (w_k, w_k); the window is symmetric
// (w_k = w_{2R-k} exactly), so six pairs serve all eleven taps.
struct WinPairs {
    F2 p[kR + 1];
    __device__ __forceinline__ explicit WinPairs(const Win &win)
    {
#pragma unroll
        for (int k = 0; k <= kR; k++) p[k] = f2(win.w[k], win.w[k]);
    }
    __device__ __forceinline__ F2 operator[](int k) const { return p[k <= kR ? k : 2 * kR - k]; }
};

// The 1-D passes are written in scatter form: each input is read (and its
// products formed) once and added into the kRun outputs it feeds. Every
// output still sums its taps in the order k = 0 .. 2R from zero, so the
// result is the same as the gather form, tap by tap.

// Pass 1: blurred statistics (separable, register-blocked), per-pixel SSIM
// and its partials w.r.t. (mu_x, E[x^2], E[xy]) scaled by dL/dSSIM_p, block
// sums of |x - y| and SSIM. The x and y statistics travel as packed pairs
// (mu_x, mu_y) and (E[x^2], E[y^2]); E[xy] is the scalar fifth.
__global__ void __launch_bounds__(256) k_ssim_pass1(const float *__restrict__ X, const float *__restrict__ Y, int W, int H,
                                                    Win win, float wscale, float *__restrict__ d_mu,
                                                    float *__restrict__ d_xx, float *__restrict__ d_xy,
                                                    float *__restrict__ partial)
{
    pdl_enter();
    __shared__ __align__(16) float sx[kHY][kSX];
    __shared__ __align__(16) float sy[kHY][kSX];
    __shared__ F2 hm[kHY][kTX + 1];   // horizontal (mu_x, mu_y)
    __shared__ F2 hs[kHY][kTX + 1];   // horizontal (E[x^2], E[y^2])
    __shared__ float hc[kHY][kTX + 1];  // horizontal E[xy]
    __shared__ float s_red[2][8];
    const int c = blockIdx.z;
    const float *x = X + (size_t)c * W * H, *y = Y + (size_t)c * W * H;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int tid = threadIdx.x;
    const WinPairs w2(win);
    if (window_inside(x0, y0, W, H, x, y, y)) {  // uniform over the CTA
        const float *const src[2] = {x, y};
        float (*const dst[2])[kSX] = {sx, sy};
        load_window_inside<2>(src, dst, x0, y0, W);
    } else {  // haloed tiles with zero padding: every load in flight before any store
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
    // horizontal: kHY rows x (kTX / kRun) runs; the 14 inputs of a run come
    // in as float4 loads (conflict-free at the 44-float row stride)
    for (int e = tid; e < kHY * (kTX / kRun); e += 256) {
        const int r = e / (kTX / kRun), j = e - r * (kTX / kRun);
        const float4 *rx = reinterpret_cast<const float4 *>(&sx[r][4 * j]);
        const float4 *ry = reinterpret_cast<const float4 *>(&sy[r][4 * j]);
        F2 a[kRun], b[kRun];
        float ab[kRun];
#pragma unroll
        for (int i = 0; i < kRun; i++) {
            a[i] = b[i] = f2(0.f, 0.f);
            ab[i] = 0.f;
        }
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const float4 fu = rx[t], fv = ry[t];
            const float u4[4] = {fu.x, fu.y, fu.z, fu.w}, v4[4] = {fv.x, fv.y, fv.z, fv.w};
#pragma unroll
            for (int l = 0; l < 4; l++) {
                const int jj = 4 * t + l;  // input column 4j + jj of the haloed row
                if (jj >= kRun + 2 * kR) continue;
                const F2 uv = f2(u4[l], v4[l]);
                const F2 sq = f2_mul(uv, uv);
                const float cr = u4[l] * v4[l];
#pragma unroll
                for (int i = 0; i < kRun; i++) {
                    const int k = jj - i;
                    if (k < 0 || k > 2 * kR) continue;
                    a[i] = f2_fma(w2[k], uv, a[i]);
                    b[i] = f2_fma(w2[k], sq, b[i]);
                    ab[i] = fmaf(win.w[k], cr, ab[i]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kRun; i++) {
            const int q = kRun * j + i;
            hm[r][q] = a[i];
            hs[r][q] = b[i];
            hc[r][q] = ab[i];
        }
    }
    __syncthreads();
    // vertical: thread (column q, run b) makes rows kRun b .. kRun b + kRun - 1
    const int q = tid & (kTX - 1), rb = tid / kTX;
    F2 mu[kRun], sq[kRun];
    float cr[kRun];
#pragma unroll
    for (int i = 0; i < kRun; i++) {
        mu[i] = sq[i] = f2(0.f, 0.f);
        cr[i] = 0.f;
    }
#pragma unroll
    for (int jj = 0; jj < kRun + 2 * kR; jj++) {
        const int rr = kRun * rb + jj;
        const F2 a = hm[rr][q], b = hs[rr][q];
        const float cc = hc[rr][q];
#pragma unroll
        for (int i = 0; i < kRun; i++) {
            const int k = jj - i;
            if (k < 0 || k > 2 * kR) continue;
            mu[i] = f2_fma(w2[k], a, mu[i]);
            sq[i] = f2_fma(w2[k], b, sq[i]);
            cr[i] = fmaf(win.w[k], cc, cr[i]);
        }
    }
    float l1 = 0.f, ss = 0.f;
    const int gx = x0 + q;
#pragma unroll
    for (int i = 0; i < kRun; i++) {
        const int r = kRun * rb + i, gy = y0 + r;
        if (gx >= W || gy >= H) continue;
        float m1, m2, e11, e22;
        f2_split(mu[i], m1, m2);
        f2_split(sq[i], e11, e22);
        const float e12 = cr[i];
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
// (the window is symmetric, so the adjoint blur is the same blur). d_mu and
// d_xx are blurred as one packed pair, d_xy as the scalar third.
__global__ void __launch_bounds__(256) k_ssim_pass2(const float *__restrict__ X, const float *__restrict__ Y, int W, int H,
                                                    Win win, float l1scale, const float *__restrict__ d_mu,
                                                    const float *__restrict__ d_xx, const float *__restrict__ d_xy,
                                                    float *__restrict__ grad)
{
    pdl_enter();
    __shared__ __align__(16) float s[3][kHY][kSX];
    __shared__ F2 hp[kHY][kTX + 1];     // horizontal (d_mu, d_xx)
    __shared__ float hq[kHY][kTX + 1];  // horizontal d_xy
    const int c = blockIdx.z;
    const size_t off = (size_t)c * W * H;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const int tid = threadIdx.x;
    const WinPairs w2(win);
    // this thread's image and target values, fetched with the window
    const int q = tid & (kTX - 1), rb = tid / kTX;
    const int gx = x0 + q;
    float xv[kRun], yv[kRun];
#pragma unroll
    for (int i = 0; i < kRun; i++) {
        const int gy = y0 + kRun * rb + i;
        const bool ok = gx < W && gy < H;
        const size_t p = off + (size_t)(ok ? gy : 0) * W + (ok ? gx : 0);
        xv[i] = ok ? X[p] : 0.f;
        yv[i] = ok ? Y[p] : 0.f;
    }
    if (window_inside(x0, y0, W, H, d_mu + off, d_xx + off, d_xy + off)) {  // uniform over the CTA
        const float *const src[3] = {d_mu + off, d_xx + off, d_xy + off};
        float (*const dst[3])[kSX] = {s[0], s[1], s[2]};
        load_window_inside<3>(src, dst, x0, y0, W);
    } else {  // haloed tiles with zero padding: every load in flight before any store
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
        const float4 *r0 = reinterpret_cast<const float4 *>(&s[0][r][4 * j]);
        const float4 *r1 = reinterpret_cast<const float4 *>(&s[1][r][4 * j]);
        const float4 *r2 = reinterpret_cast<const float4 *>(&s[2][r][4 * j]);
        F2 a[kRun];
        float b[kRun];
#pragma unroll
        for (int i = 0; i < kRun; i++) {
            a[i] = f2(0.f, 0.f);
            b[i] = 0.f;
        }
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const float4 f0 = r0[t], f1 = r1[t], f2v = r2[t];
            const float v0[4] = {f0.x, f0.y, f0.z, f0.w}, v1[4] = {f1.x, f1.y, f1.z, f1.w},
                        v2[4] = {f2v.x, f2v.y, f2v.z, f2v.w};
#pragma unroll
            for (int l = 0; l < 4; l++) {
                const int jj = 4 * t + l;
                if (jj >= kRun + 2 * kR) continue;
                const F2 pr = f2(v0[l], v1[l]);
#pragma unroll
                for (int i = 0; i < kRun; i++) {
                    const int k = jj - i;
                    if (k < 0 || k > 2 * kR) continue;
                    a[i] = f2_fma(w2[k], pr, a[i]);
                    b[i] = fmaf(win.w[k], v2[l], b[i]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kRun; i++) {
            hp[r][kRun * j + i] = a[i];
            hq[r][kRun * j + i] = b[i];
        }
    }
    __syncthreads();
    F2 bp[kRun];
    float bq[kRun];
#pragma unroll
    for (int i = 0; i < kRun; i++) {
        bp[i] = f2(0.f, 0.f);
        bq[i] = 0.f;
    }
#pragma unroll
    for (int jj = 0; jj < kRun + 2 * kR; jj++) {
        const int rr = kRun * rb + jj;
        const F2 a = hp[rr][q];
        const float bb = hq[rr][q];
#pragma unroll
        for (int i = 0; i < kRun; i++) {
            const int k = jj - i;
            if (k < 0 || k > 2 * kR) continue;
            bp[i] = f2_fma(w2[k], a, bp[i]);
            bq[i] = fmaf(win.w[k], bb, bq[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < kRun; i++) {
        const int gy = y0 + kRun * rb + i;
        if (gx >= W || gy >= H) continue;
        const size_t p = off + (size_t)gy * W + gx;
        const float diff = xv[i] - yv[i];
        const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
        float b0, b1;
        f2_split(bp[i], b0, b1);
        grad[p] = b0 + 2.f * xv[i] * b1 + yv[i] * bq[i] + sgn * l1scale;
    }
}

// Final stage: the kColsumParts partial rows of (sum |x-y|, sum SSIM) in a
// fixed order, then the loss.
// one warp: lane l adds partial rows l, l + 32, ... (FP64), then a fixed
// butterfly; the FP64 add chain stays short on this GPU's narrow FP64 pipe
__global__ void k_loss_final(const float *__restrict__ part, double inv_count, float lam, float *__restrict__ loss)
{
    pdl_enter();
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
    launch_pdl(k_ssim_pass1, grid, 256, 0, s, img, tgt, W, H, win, (float)(-lam * inv), d_mu, d_xx, d_xy, partial);
    count_launch();
    const int nb = grid.x * grid.y * grid.z;
    float *part2 = partial + 2 * nb;
    launch_colsum_partial(partial, nb, 2, part2, s);
    launch_pdl(k_loss_final, 1, 32, 0, s, part2, inv, lam, loss);
    count_launch();
    if (grad) launch_pdl(k_ssim_pass2, grid, 256, 0, s, img, tgt, W, H, win, (float)inv, d_mu, d_xx, d_xy, grad);
    if (grad) count_launch();
}

}  // namespace splash
