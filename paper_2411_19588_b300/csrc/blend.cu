// Per-tile front-to-back blending with the water model (forward) and its
// back-to-front adjoint (backward).
//
// Passages: Eq. 1 (alpha compositing over depth-sorted Gaussians), Eq. 2
// (alpha = sigmoid(o) e^{-q/2}), Sec. III-A (tiles, tile-parallel rendering),
// Eq. 3-5 (water), Eq. 6 (expected depth), Sec. IV-D (logistic depth map).
//
// Water model per pixel, Gaussians i = 1..m front to back with transmittance
// T_i in front of each, d_0 = 0 and the last segment ending at z_far:
//   C = sum_i c_i e^{-bD d_i} a_i T_i + B sum_{i=1}^{m+1} T_i (e^{-bB d_{i-1}} - e^{-bB d_i})
// Summation by parts turns the water sum into per-Gaussian terms:
//   C = sum_i a_i T_i ct_i + B (1 - T_final e^{-bB z_far}),  ct_i = c_i e^{-bD d_i} - B e^{-bB d_i}
// so the inner loop is plain compositing of the effective colour ct (made
// once per Gaussian in the preprocess) and the water costs one epilogue.
//
// Work decomposition: one CTA per tile, kPxFwd / kPxBwd pixels of one row per
// thread (they share the dy terms and, backward, one warp reduction of the
// gradient fields per Gaussian). Gaussians are staged in shared
// memory in batches of NB (64, 128 or 256); the local centre is formed once
// per (tile, Gaussian) from the doubled-precision record, relative to the
// 32-pixel-aligned corner that holds the tile (the same corner for every
// tile shape, so all shapes do identical per-pixel arithmetic). A warp skips
// a batch once all its pixels are done; the CTA stops when all are.
// Plain launches run one CTA per tile of one view; the persistent launches
// keep one wave of CTAs that pull (view, tile) items from a queue.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace splash {
namespace {

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x for x in [0.01, 1] (x = 1 - alpha with alpha <= 0.99): the hardware
// approximation, relative error below 2^-22
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// qs = A dx^2 + B dx dy + C dy^2 with the dy terms precomputed; used by both
// passes so that they take identical decisions
__device__ __forceinline__ float quad(float dx, float A, float Bdy, float Cdy2) { return fmaf(dx, fmaf(A, dx, Bdy), Cdy2); }

// pixels per thread, forward and backward
constexpr int kPxFwd = 2;
constexpr int kPxBwd = 4;

template <int TW, int TH, int PX>
struct Tile {
    static constexpr int NT = TW * TH / PX;  // threads per CTA
    static constexpr int HW = TW / PX;       // a thread's pixels are HW columns apart in one row
    static_assert(TW % PX == 0 && NT % 32 == 0, "tile width must split into PX pixels per thread");
};
template <int TW, int TH>
constexpr int fwd_threads() { return Tile<TW, TH, kPxFwd>::NT; }
template <int TW, int TH>
constexpr int bwd_threads() { return Tile<TW, TH, kPxBwd>::NT; }

// stage list entry `slot` of the batch: local centre, conic, log-opacity, colour, depth
__device__ __forceinline__ void stage_rec(const Rec *__restrict__ rec, uint32_t gid, int ox, int oy, float4 *s0, float4 *s1,
                                          float2 *s2, int slot)
{
    const Rec r = rec[gid];
    const float xl = (r.r0.x - (float)ox) + r.r0.z;
    const float yl = (r.r0.y - (float)oy) + r.r0.w;
    s0[slot] = make_float4(xl, yl, r.r1.x, r.r1.y);
    s1[slot] = make_float4(r.r1.z, r.r1.w, r.r2.y, r.r2.z);
    s2[slot] = make_float2(r.r2.w, r.r2.x);
}

template <int TW, int TH, int NB>
__device__ __forceinline__ void blend_tile_fwd(const BlendView &v, int tile, const float *__restrict__ medium)
{
    constexpr int PX = kPxFwd;
    constexpr int NT = Tile<TW, TH, PX>::NT, HW = Tile<TW, TH, PX>::HW;
    __shared__ float4 s0[NB];  // {x_loc, y_loc, A, B}
    __shared__ float4 s1[NB];  // {C, lo, ct_r, ct_g}
    __shared__ float2 s2[NB];  // {ct_b, d}
    const CamK &cam = v.cam;
    const int tyi = tile / v.tg.tx, txi = tile - tyi * v.tg.tx;
    const int x0 = txi * TW, y0 = tyi * TH;
    const int ox = x0 & ~31, oy = y0 & ~31;  // local origin shared by all tile shapes
    const int tid = threadIdx.x;
    const int row = tid / HW, col = tid - row * HW;
    const float pyl = (float)(y0 - oy + row) + 0.5f;
    const int W = cam.W, H = cam.H;
    const int gy = y0 + row;
    const uint2 rg = v.ranges[tile];
    const int n = (int)(rg.y - rg.x);

    float pxl[PX], T[PX], cr[PX], cg[PX], cb[PX], D[PX], A[PX];
    int last[PX], walk[PX];
    bool done[PX];
#pragma unroll
    for (int q = 0; q < PX; q++) {
        pxl[q] = (float)(x0 - ox + col + q * HW) + 0.5f;
        T[q] = 1.f;
        cr[q] = cg[q] = cb[q] = D[q] = A[q] = 0.f;
        last[q] = 0;
        done[q] = !(gy < H && x0 + col + q * HW < W);
        walk[q] = done[q] ? 0 : n;
    }

    for (int b0 = 0; b0 < n; b0 += NB) {
        bool all = true;
#pragma unroll
        for (int q = 0; q < PX; q++) all &= done[q];
        if (__syncthreads_count(!all) == 0) break;
        for (int sl = tid; sl < NB && b0 + sl < n; sl += NT) stage_rec(v.rec, v.gauss_ids[rg.x + b0 + sl], ox, oy, s0, s1, s2, sl);
        __syncthreads();
        const int nb = min(NB, n - b0);
        if (!__any_sync(0xffffffffu, !all)) continue;
        for (int k = 0; k < nb; k++) {
            const float4 a = s0[k];
            const float4 c = s1[k];
            const float dy = pyl - a.y;
            const float Bdy = a.w * dy;
            const float Cdy2 = c.x * dy * dy;
#pragma unroll
            for (int q = 0; q < PX; q++) {
                if (done[q]) continue;
                const float dx = pxl[q] - a.x;
                const float qs = quad(dx, a.z, Bdy, Cdy2);
                if (qs < kQsMin) continue;
                const float alpha = fminf(kAlphaMax, ex2_approx(qs + c.y));
                if (alpha < kAlphaMin) continue;
                const float tn = fmaf(-alpha, T[q], T[q]);
                if (tn < kTStop) {
                    done[q] = true;
                    walk[q] = b0 + k + 1;
                } else {
                    const float w = alpha * T[q];
                    const float2 e = s2[k];
                    cr[q] = fmaf(w, c.z, cr[q]);
                    cg[q] = fmaf(w, c.w, cg[q]);
                    cb[q] = fmaf(w, e.x, cb[q]);
                    D[q] = fmaf(w, e.y, D[q]);
                    A[q] += w;
                    T[q] = tn;
                    last[q] = b0 + k + 1;
                }
            }
        }
    }

    // epilogue: water behind the last Gaussian, depth, forward state
    const float zfar = cam.zfar;
    float binf[3], bfar[3];
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        binf[ch] = __ldg(medium + 6 + ch);
        bfar[ch] = expf(-__ldg(medium + 3 + ch) * zfar);
    }
    const int HWimg = W * H;
#pragma unroll
    for (int q = 0; q < PX; q++) {
        const int gx = x0 + col + q * HW;
        if (!(gy < H && gx < W)) continue;
        const int p = gy * W + gx;
        v.image[p] = cr[q] + binf[0] * (1.f - T[q] * bfar[0]);
        v.image[HWimg + p] = cg[q] + binf[1] * (1.f - T[q] * bfar[1]);
        v.image[2 * HWimg + p] = cb[q] + binf[2] * (1.f - T[q] * bfar[2]);
        const float z = A[q] > 0.f ? D[q] / A[q] : zfar;
        if (v.depth) v.depth[p] = z;
        if (v.depth01) v.depth01[p] = 2.f / (1.f + expf(-0.1f * z)) - 1.f;
        v.final_T[p] = T[q];
        v.acc_alpha[p] = A[q];
        v.zhat[p] = z;
        v.n_last[p] = (uint32_t)last[q];
        v.n_walk[p] = (uint32_t)walk[q];
    }
}

// ---------------------------------------------------------------------------
// Backward.

// Per-pixel state of the back-to-front walk.
struct PixB {
    float T;      // transmittance behind the current Gaussian (starts at T_final)
    float S;      // sum over Gaussians behind: w * (G.ct + gD d + gA), plus the water term
    float G0, G1, G2, gD, gA;
    int last;
};

// One warp-wide sum of 10 values by recursive halving: after five exchange
// steps lane L holds the warp total of field reduce10_field(L) (12 shuffles
// instead of 50 for ten separate butterflies).
template <int C>
__device__ __forceinline__ void rs_step(float *v, int m, bool hi)
{
    constexpr int H = (C + 1) / 2;
    float out[H];
#pragma unroll
    for (int i = 0; i < H; i++) {
        const float upper = (H + i < C) ? v[H + i] : 0.f;
        const float keep = hi ? upper : v[i];
        const float send = hi ? v[i] : upper;
        out[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
    }
#pragma unroll
    for (int i = 0; i < H; i++) v[i] = out[i];
}

__device__ __forceinline__ float warp_reduce10(float *v, int lane)
{
    rs_step<10>(v, 16, lane & 16);
    rs_step<5>(v, 8, lane & 8);
    rs_step<3>(v, 4, lane & 4);
    rs_step<2>(v, 2, lane & 2);
    rs_step<1>(v, 1, lane & 1);
    return v[0];
}

// which of the ten fields lane `lane` holds after warp_reduce10 (-1: none)
__device__ __forceinline__ int reduce10_field(int lane)
{
    int base = 0, nreal = 10, c = 10;
    const int masks[5] = {16, 8, 4, 2, 1};
#pragma unroll
    for (int s = 0; s < 5; s++) {
        const int h = (c + 1) / 2;
        if (lane & masks[s]) {
            base += h;
            nreal = max(0, nreal - h);
        } else {
            nreal = min(nreal, h);
        }
        c = h;
    }
    return nreal > 0 ? base : -1;
}

// adjoint of one pixel at one Gaussian that contributes to it (alpha = the
// clamped raw value araw, which is at least 1/255 here; dx its column offset).
// DG: the loss has a depth term (gD, gA non-zero); without it those terms vanish.
// The exponent's gradient gqs enters the centre and conic gradients only
// through its moments: acc[5] = sum gqs, acc[0] = sum gqs dx, acc[2] = sum
// gqs dx^2 over the thread's pixels (one row, so dy is shared); the dy
// moments and the conic coefficients are applied once per Gaussian.
template <bool DG>
__device__ __forceinline__ void pix_grad(PixB &p, float dx, float araw, float ctr, float ctg, float ctb, float d, float *acc)
{
    const float alpha = fminf(kAlphaMax, araw);
    const float inv = rcp_approx(1.f - alpha);
    const float Tj = p.T * inv;  // transmittance in front of this Gaussian
    const float w = alpha * Tj;
    const float u = DG ? fmaf(p.G0, ctr, fmaf(p.G1, ctg, fmaf(p.G2, ctb, fmaf(p.gD, d, p.gA))))
                       : fmaf(p.G0, ctr, fmaf(p.G1, ctg, p.G2 * ctb));
    // dL/dalpha = T_j u - S / (1 - alpha)
    const float galpha = fmaf(Tj, u, -p.S * inv);
    const float gqs = araw < kAlphaMax ? galpha * alpha * kLn2 : 0.f;
    const float gx = gqs * dx;
    acc[0] += gx;
    acc[2] = fmaf(gx, dx, acc[2]);
    acc[5] += gqs;
    if (DG) acc[6] = fmaf(p.gD, w, acc[6]);
    acc[7] = fmaf(p.G0, w, acc[7]);
    acc[8] = fmaf(p.G1, w, acc[8]);
    acc[9] = fmaf(p.G2, w, acc[9]);
    p.S = fmaf(w, u, p.S);
    p.T = Tj;
}

template <int TW, int TH, int NB, bool DG>
__device__ __forceinline__ void blend_tile_bwd(const BlendView &v, int tile, const float *__restrict__ medium)
{
    constexpr int PX = kPxBwd;
    constexpr int NT = Tile<TW, TH, PX>::NT, HW = Tile<TW, TH, PX>::HW;
    constexpr int NW = NT / 32;
    __shared__ float4 s0[NB];
    __shared__ float4 s1[NB];
    __shared__ float2 s2[NB];
    __shared__ uint32_t s_id[NB];
    __shared__ float s_g[10][NB + 1];  // padded: the ten fields of one Gaussian fall in ten banks
    __shared__ float s_med[NW][6];
    __shared__ int s_maxlast;

    const CamK &cam = v.cam;
    const int tyi = tile / v.tg.tx, txi = tile - tyi * v.tg.tx;
    const int x0 = txi * TW, y0 = tyi * TH;
    const int ox = x0 & ~31, oy = y0 & ~31;  // local origin shared by all tile shapes
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int row = tid / HW, col = tid - row * HW;
    const float pyl = (float)(y0 - oy + row) + 0.5f;
    const int W = cam.W, H = cam.H;
    const int gy = y0 + row;
    const uint2 rg = v.ranges[tile];
    const int HWimg = W * H;
    const float zfar = cam.zfar;
    float binf[3], bfar[3];
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        binf[ch] = __ldg(medium + 6 + ch);
        bfar[ch] = expf(-__ldg(medium + 3 + ch) * zfar);
    }
    if (tid == 0) s_maxlast = 0;

    // per-pixel set-up; medium terms that do not go through any Gaussian:
    //   dC/dB_inf = 1 - T_f b_far, dC/dbeta_B = B_inf T_f z_far b_far
    float mB[3] = {0.f, 0.f, 0.f}, mBB[3] = {0.f, 0.f, 0.f};
    float pxl[PX];
    PixB P[PX];
    int mylast = 0;
#pragma unroll
    for (int q = 0; q < PX; q++) {
        const int gx = x0 + col + q * HW;
        pxl[q] = (float)(x0 - ox + col + q * HW) + 0.5f;
        PixB &p = P[q];
        p.T = 1.f; p.S = 0.f; p.G0 = p.G1 = p.G2 = p.gD = p.gA = 0.f; p.last = 0;
        if (!(gy < H && gx < W)) continue;
        const int pix = gy * W + gx;
        p.T = v.final_T[pix];
        p.last = (int)v.n_last[pix];
        p.G0 = v.dL_dimage[pix];
        p.G1 = v.dL_dimage[HWimg + pix];
        p.G2 = v.dL_dimage[2 * HWimg + pix];
        if (DG) {
            const float A = v.acc_alpha[pix], z = v.zhat[pix];
            float gz = v.dL_ddepth ? v.dL_ddepth[pix] : 0.f;
            if (v.dL_ddepth01) {
                const float e = expf(-0.1f * z);
                gz += v.dL_ddepth01[pix] * 0.2f * e / ((1.f + e) * (1.f + e));
            }
            if (A > 0.f) {
                p.gD = gz / A;  // z = D / A
                p.gA = -gz * z / A;
            }
        }
        const float Gc[3] = {p.G0, p.G1, p.G2};
        float S = 0.f;
#pragma unroll
        for (int ch = 0; ch < 3; ch++) {
            mB[ch] += Gc[ch] * (1.f - p.T * bfar[ch]);
            mBB[ch] += Gc[ch] * binf[ch] * p.T * zfar * bfar[ch];
            S -= Gc[ch] * binf[ch] * bfar[ch] * p.T;  // the water behind the last Gaussian
        }
        p.S = S;
        mylast = max(mylast, p.last);
    }
    // per-tile medium partials {beta_B[3], B_inf[3]}, reduced now so that the
    // accumulators do not stay live through the main loop
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        float a = mBB[ch], b = mB[ch];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            s_med[warp][ch] = a;
            s_med[warp][3 + ch] = b;
        }
    }
    __syncthreads();
    atomicMax(&s_maxlast, mylast);
    if (tid < 6) {
        float acc = 0.f;
#pragma unroll
        for (int w = 0; w < NW; w++) acc += s_med[w][tid];
        v.tile_medium[6 * tile + tid] = acc;
    }
    const int my_field = reduce10_field(lane);
    __syncthreads();
    const int maxlast = s_maxlast;

    for (int bend = maxlast; bend > 0; bend -= NB) {
        const int b0 = max(0, bend - NB);
        const int nb = bend - b0;
        __syncthreads();  // the previous batch's flush has read s_g / s_id
        for (int sl = tid; sl < nb; sl += NT) {
            const uint32_t gid = v.gauss_ids[rg.x + b0 + sl];
            stage_rec(v.rec, gid, ox, oy, s0, s1, s2, sl);
            s_id[sl] = gid;
        }
        for (int sl = tid; sl < NB; sl += NT)
#pragma unroll
            for (int f = 0; f < 10; f++) s_g[f][sl] = 0.f;
        __syncthreads();
        if (__any_sync(0xffffffffu, mylast > b0)) {
            for (int k = nb - 1; k >= 0; k--) {
                const int j = b0 + k;
                const float4 a = s0[k];
                const float4 c = s1[k];
                const float2 e = s2[k];
                const float dy = pyl - a.y;
                const float Bdy = a.w * dy;
                const float Cdy2 = c.x * dy * dy;
                float acc[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                // the exponent and raw alpha of all the thread's pixels first, without
                // branches (independent chains the scheduler can overlap); a pixel
                // takes part if the Gaussian is in front of its last one, within
                // 3 sigma and at least 1/255 opaque there
                float dxv[PX], arv[PX];
                bool on[PX];
#pragma unroll
                for (int q = 0; q < PX; q++) {
                    dxv[q] = pxl[q] - a.x;
                    const float qs = quad(dxv[q], a.z, Bdy, Cdy2);
                    arv[q] = ex2_approx(qs + c.y);
                    on[q] = (j < P[q].last) & (qs >= kQsMin) & (fminf(kAlphaMax, arv[q]) >= kAlphaMin);
                }
                bool any = false;
#pragma unroll
                for (int q = 0; q < PX; q++) {
                    if (!on[q]) continue;
                    pix_grad<DG>(P[q], dxv[q], arv[q], c.z, c.w, e.x, e.y, acc);
                    any = true;
                }
                if (__any_sync(0xffffffffu, any)) {
                    // moments in y from the row's dy: sum gqs dy, sum gqs dx dy, sum gqs dy^2
                    acc[1] = acc[5] * dy;
                    acc[3] = acc[0] * dy;
                    acc[4] = acc[5] * (dy * dy);
                    const float r = warp_reduce10(acc, lane);
                    if (my_field >= 0) atomicAdd(&s_g[my_field][k], r);
                }
            }
        }
        __syncthreads();
        for (int sl = tid; sl < nb; sl += NT) {
            const float g[10] = {s_g[0][sl], s_g[1][sl], s_g[2][sl], s_g[3][sl], s_g[4][sl],
                                 s_g[5][sl], s_g[6][sl], s_g[7][sl], s_g[8][sl], s_g[9][sl]};
            bool nz = false;
#pragma unroll
            for (int f = 0; f < 10; f++) nz |= g[f] != 0.f;
            if (nz) {
                // centre gradient from the moments: dqs/dx = 2A dx + B dy, dqs/dy = B dx + 2C dy
                const float A = s0[sl].z, B = s0[sl].w, C = s1[sl].x;
                const float gmx = -fmaf(2.f * A, g[0], B * g[1]);
                const float gmy = -fmaf(B, g[0], 2.f * C * g[1]);
                GAcc *dst = v.gacc + s_id[sl];
                atomicAdd(&dst->a0, make_float4(gmx, gmy, g[2], g[3]));
                atomicAdd(&dst->a1, make_float4(g[4], g[5], g[6], 0.f));
                atomicAdd(&dst->a2, make_float4(g[7], g[8], g[9], 0.f));
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Kernels.

template <int TW, int TH, int NB>
__global__ void __launch_bounds__(fwd_threads<TW, TH>(), 1280 / fwd_threads<TW, TH>()) k_blend_fwd(BlendView v, const float *__restrict__ medium)
{
    blend_tile_fwd<TW, TH, NB>(v, blockIdx.x, medium);
}

// occupancy target: 14 blocks of 64 threads per SM without the depth terms
// (72 registers), 12 with them (80)
template <int TW, int TH, int NB, bool DG>
__global__ void __launch_bounds__(bwd_threads<TW, TH>(), (DG ? 768 : 896) / bwd_threads<TW, TH>()) k_blend_bwd(BlendView v, const float *__restrict__ medium)
{
    blend_tile_bwd<TW, TH, NB, DG>(v, blockIdx.x, medium);
}

// Persistent: one wave of CTAs; each takes the next (view, tile) item from the
// queue (items are ordered longest list first) until none is left. The only
// shared state is an atomic ticket counter: nothing waits on another CTA.
__device__ __forceinline__ bool next_item(int *counter, const uint32_t *n_items, int &it)
{
    __shared__ int s_item;
    __syncthreads();  // everyone is done with the previous item
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    it = s_item;
    return it < (int)*n_items;
}

template <int TW, int TH, int NB>
__global__ void __launch_bounds__(fwd_threads<TW, TH>(), 1152 / fwd_threads<TW, TH>()) k_blend_fwd_persistent(const BlendView *__restrict__ views,
                                                                  const uint32_t *__restrict__ items,
                                                                  const uint32_t *__restrict__ n_items, int *counter,
                                                                  const float *__restrict__ medium)
{
    int it;
    while (next_item(counter, n_items, it)) {
        const uint32_t code = items[it];
        blend_tile_fwd<TW, TH, NB>(views[code >> 24], (int)(code & 0xffffffu), medium);
    }
}

template <int TW, int TH, int NB>
__global__ void __launch_bounds__(bwd_threads<TW, TH>(), 768 / bwd_threads<TW, TH>()) k_blend_bwd_persistent(const BlendView *__restrict__ views,
                                                                 const uint32_t *__restrict__ items,
                                                                 const uint32_t *__restrict__ n_items, int *counter,
                                                                 const float *__restrict__ medium)
{
    int it;
    while (next_item(counter, n_items, it)) {
        const uint32_t code = items[it];
        blend_tile_bwd<TW, TH, NB, false>(views[code >> 24], (int)(code & 0xffffffu), medium);  // no depth loss in batches
    }
}

// dispatch over tile shape x staging batch
template <template <int, int, int> class F, class... Args>
void dispatch(int tw, int nb, Args... args)
{
    const int bi = nb <= 64 ? 0 : (nb <= 128 ? 1 : 2);
    if (tw == 8) {
        if (bi == 0) F<8, 32, 64>::run(args...);
        else if (bi == 1) F<8, 32, 128>::run(args...);
        else F<8, 32, 256>::run(args...);
    } else if (tw == 32) {
        if (bi == 0) F<32, 8, 64>::run(args...);
        else if (bi == 1) F<32, 8, 128>::run(args...);
        else F<32, 8, 256>::run(args...);
    } else {
        if (bi == 0) F<16, 16, 64>::run(args...);
        else if (bi == 1) F<16, 16, 128>::run(args...);
        else F<16, 16, 256>::run(args...);
    }
}

template <int TW, int TH, int NB>
struct FwdPlain {
    static void run(const BlendView &v, const float *medium, cudaStream_t s)
    {
        k_blend_fwd<TW, TH, NB><<<v.tg.tx * v.tg.ty, fwd_threads<TW, TH>(), 0, s>>>(v, medium);
        count_launch();
    }
};
template <int TW, int TH, int NB>
struct BwdPlain {
    static void run(const BlendView &v, const float *medium, cudaStream_t s)
    {
        if (v.dL_ddepth || v.dL_ddepth01)
            k_blend_bwd<TW, TH, NB, true><<<v.tg.tx * v.tg.ty, bwd_threads<TW, TH>(), 0, s>>>(v, medium);
        else
            k_blend_bwd<TW, TH, NB, false><<<v.tg.tx * v.tg.ty, bwd_threads<TW, TH>(), 0, s>>>(v, medium);
        count_launch();
    }
};
template <int TW, int TH, int NB>
struct FwdPersistent {
    static void run(const BlendView *v, const uint32_t *items, const uint32_t *n, int *counter, const float *medium,
                    int ctas, cudaStream_t s)
    {
        k_blend_fwd_persistent<TW, TH, NB><<<ctas, fwd_threads<TW, TH>(), 0, s>>>(v, items, n, counter, medium);
        count_launch();
    }
};
template <int TW, int TH, int NB>
struct BwdPersistent {
    static void run(const BlendView *v, const uint32_t *items, const uint32_t *n, int *counter, const float *medium,
                    int ctas, cudaStream_t s)
    {
        k_blend_bwd_persistent<TW, TH, NB><<<ctas, bwd_threads<TW, TH>(), 0, s>>>(v, items, n, counter, medium);
        count_launch();
    }
};
template <int TW, int TH, int NB>
struct Occupancy {
    static void run(bool backward, int *out)
    {
        int dev = 0, sms = 148, per = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (backward)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_blend_bwd_persistent<TW, TH, NB>, bwd_threads<TW, TH>(), 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_blend_fwd_persistent<TW, TH, NB>, fwd_threads<TW, TH>(), 0);
        *out = sms * (per > 0 ? per : 1);
    }
};

}  // namespace

void launch_blend_fwd(const BlendView &v, const float *medium, int batch, cudaStream_t s)
{
    dispatch<FwdPlain>(v.tg.tw, batch, v, medium, s);
}

void launch_blend_bwd(const BlendView &v, const float *medium, int batch, cudaStream_t s)
{
    dispatch<BwdPlain>(v.tg.tw, batch, v, medium, s);
}

void launch_blend_fwd_persistent(int tw, int th, int batch, const BlendView *views, const uint32_t *items,
                                 const uint32_t *n_items, int *counter, const float *medium, int ctas, cudaStream_t s)
{
    (void)th;
    dispatch<FwdPersistent>(tw, batch, views, items, n_items, counter, medium, ctas, s);
}

void launch_blend_bwd_persistent(int tw, int th, int batch, const BlendView *views, const uint32_t *items,
                                 const uint32_t *n_items, int *counter, const float *medium, int ctas, cudaStream_t s)
{
    (void)th;
    dispatch<BwdPersistent>(tw, batch, views, items, n_items, counter, medium, ctas, s);
}

int blend_persistent_ctas(int tw, int th, int batch, bool backward)
{
    (void)th;
    int out = 148;
    dispatch<Occupancy>(tw, batch, backward, &out);
    return out;
}

}  // namespace splash
