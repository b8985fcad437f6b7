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
// Work decomposition: one CTA per tile, 4 pixels of one row per thread in
// both passes (they share the dy terms and, backward, one warp reduction of
// the gradient fields per Gaussian). A thread's pixels run as two FP32x2 lane
// pairs (packed add / mul / fma, one lane per pixel column) through
// predicated bodies: a pixel that a Gaussian does not reach gets alpha = 0,
// which adds nothing. Gaussians are staged in shared memory in batches of NB
// (64 forward, 128 backward by default) with every per-Gaussian constant
// stored twice, so one 16-byte load yields a packed operand; the local centre
// is formed once per (tile, Gaussian) from the doubled-precision record,
// relative to the 32-pixel-aligned corner that holds the tile (the same
// corner for every tile shape, so all shapes do identical per-pixel
// arithmetic). A warp skips a Gaussian that none of its pixels reaches and a
// batch once all its pixels are done; the CTA stops when all are.
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
constexpr int kPxFwd = 4;
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

// Forward staging: every per-Gaussian constant twice, so that one 16-byte
// shared load yields the packed operand of a thread's two pixel columns
// (FP32x2 arithmetic, one lane per column). Positions are stored negated:
// pxl + (-x) rounds exactly as pxl - x. sth: the Gaussian's threshold on the
// exponent qs of a pixel, max(3-sigma cut, log2(1/255) - log2 opacity): a
// pixel takes part where qs >= it, i.e. within 3 sigma and at least 1/255
// opaque (both tests in one comparison, in the exponent's domain). The
// backward forms the same threshold from the staged log2 opacity (null sth).
__device__ __forceinline__ float exponent_threshold(float log2_opacity) { return fmaxf(kQsMin, kLog2AlphaMin - log2_opacity); }

__device__ __forceinline__ void stage_fwd(const Rec *__restrict__ rec, uint32_t gid, int ox, int oy, float4 *sx,
                                          float4 *sy, float4 *sc, float4 *sk, float4 *sb, float *sth, int slot)
{
    const Rec r = rec[gid];
    const float xl = (r.r0.x - (float)ox) + r.r0.z;
    const float yl = (r.r0.y - (float)oy) + r.r0.w;
    sx[slot] = make_float4(-xl, -xl, r.r1.x, r.r1.x);          // {-x, -x, A, A}
    sy[slot] = make_float4(-yl, -yl, r.r1.y, r.r1.y);          // {-y, -y, B, B}
    sc[slot] = make_float4(r.r1.z, r.r1.z, r.r1.w, r.r1.w);    // {C, C, lo, lo}
    sk[slot] = make_float4(r.r2.y, r.r2.y, r.r2.z, r.r2.z);    // {ct_r, ct_r, ct_g, ct_g}
    sb[slot] = make_float4(r.r2.w, r.r2.w, r.r2.x, r.r2.x);    // {ct_b, ct_b, d, d}
    if (sth) sth[slot] = exponent_threshold(r.r1.w);
}

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// Forward. The thread's PX pixels (one row, HW columns apart) run as PX/2
// FP32x2 lane pairs through one predicated body: a pair that is outside the
// pixel's 3-sigma ellipse or below 1/255 gets alpha = 0 (adds nothing,
// leaves T), a finished pixel has a NaN column (its quadratic form is NaN, so
// it fails the 3-sigma test), and only the rare stop at the transmittance
// floor branches. Per-lane arithmetic is the scalar IEEE arithmetic of the
// backward (same dx, quadratic form, exponent and tests), so both passes take
// identical decisions.
template <int TW, int TH, int NB>
__device__ __forceinline__ void blend_tile_fwd(const BlendView &v, int tile, const float *__restrict__ medium)
{
    constexpr int PX = kPxFwd, NP = PX / 2;
    constexpr int NT = Tile<TW, TH, PX>::NT, HW = Tile<TW, TH, PX>::HW;
    __shared__ float4 sx[NB], sy[NB], sc[NB], sk[NB], sb[NB];
    __shared__ float sth[NB];
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
    const float kNaN = __int_as_float(0x7fc00000);
    if (v.clear) {
        // this tile's share of the backward's accumulators: the stores drain
        // while the blend below computes
        const int64_t ntiles = (int64_t)v.tg.tx * v.tg.ty;
        const int64_t per = (v.clear_n + ntiles - 1) / ntiles;
        const int64_t b = min((int64_t)tile * per, v.clear_n), e = min(b + per, v.clear_n);
        float4 *dst = reinterpret_cast<float4 *>(v.clear + b);
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t q = tid; q < 3 * (e - b); q += NT) dst[q] = z;
    }

    // a finished pixel's column is a quiet NaN whose payload is its walked
    // count (the stop position + 1, < 2^22): it fails every 3-sigma test
    float2 pxl[NP], T[NP], cr[NP], cg[NP], cb[NP], D[NP], A[NP];
    int live = 0;
#pragma unroll
    for (int j = 0; j < NP; j++) {
        float c2[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int q = 2 * j + h;
            const bool in = gy < H && x0 + col + q * HW < W;
            c2[h] = in ? (float)(x0 - ox + col + q * HW) + 0.5f : kNaN;
            live += in;
        }
        pxl[j] = make_float2(c2[0], c2[1]);
        T[j] = make_float2(1.f, 1.f);
        cr[j] = cg[j] = cb[j] = D[j] = A[j] = make_float2(0.f, 0.f);
    }
    const float2 pyl2 = make_float2(pyl, pyl), neg1 = make_float2(-1.f, -1.f);

    for (int b0 = 0; b0 < n; b0 += NB) {
        if (__syncthreads_count(live > 0) == 0) break;
        for (int sl = tid; sl < NB && b0 + sl < n; sl += NT)
            stage_fwd(v.rec, v.gauss_ids[rg.x + b0 + sl], ox, oy, sx, sy, sc, sk, sb, sth, sl);
        __syncthreads();
        const int nb = min(NB, n - b0);
        if (!__any_sync(0xffffffffu, live > 0)) continue;
        for (int k = 0; k < nb; k++) {
            const float4 fx = sx[k], fy = sy[k], fc = sc[k];
            const float th = sth[k];
            const float2 dy = __fadd2_rn(pyl2, lo2(fy));
            const float2 Bdy = __fmul2_rn(hi2(fy), dy);
            const float2 Cdy2 = __fmul2_rn(__fmul2_rn(lo2(fc), dy), dy);
            float2 qs[NP];
            bool inside = false;
#pragma unroll
            for (int j = 0; j < NP; j++) {
                const float2 dx = __fadd2_rn(pxl[j], lo2(fx));
                qs[j] = __ffma2_rn(dx, __ffma2_rn(hi2(fx), dx, Bdy), Cdy2);
                inside |= (qs[j].x >= th) | (qs[j].y >= th);
            }
            // none of the thread's pixels within 3 sigma and 1/255 opaque:
            // nothing to add (a warp skips the rest when this holds for all
            // its lanes)
            if (!inside) continue;
            float2 w[NP], tn[NP];
            bool stop = false;
#pragma unroll
            for (int j = 0; j < NP; j++) {
                const float2 e = __fadd2_rn(qs[j], hi2(fc));
                // the same test as the backward's (qs against the threshold), then the clamp
                const float r0 = ex2_approx(e.x), r1 = ex2_approx(e.y);
                const float a0 = qs[j].x >= th ? fminf(kAlphaMax, r0) : 0.f;
                const float a1 = qs[j].y >= th ? fminf(kAlphaMax, r1) : 0.f;
                w[j] = __fmul2_rn(make_float2(a0, a1), T[j]);
                tn[j] = __ffma2_rn(w[j], neg1, T[j]);  // T - alpha T
                stop |= (tn[j].x < kTStop) | (tn[j].y < kTStop);
            }
            if (stop) {
                // stop before this Gaussian: it adds nothing, the pixel is finished
#pragma unroll
                for (int j = 0; j < NP; j++) {
                    const float done = __int_as_float(0x7fc00000 | (b0 + k + 1));
                    if (tn[j].x < kTStop) {
                        w[j].x = 0.f;
                        tn[j].x = T[j].x;
                        pxl[j].x = done;
                        live--;
                    }
                    if (tn[j].y < kTStop) {
                        w[j].y = 0.f;
                        tn[j].y = T[j].y;
                        pxl[j].y = done;
                        live--;
                    }
                }
            }
            const float4 fk = sk[k], fb = sb[k];
#pragma unroll
            for (int j = 0; j < NP; j++) {
                cr[j] = __ffma2_rn(w[j], lo2(fk), cr[j]);
                cg[j] = __ffma2_rn(w[j], hi2(fk), cg[j]);
                cb[j] = __ffma2_rn(w[j], lo2(fb), cb[j]);
                D[j] = __ffma2_rn(w[j], hi2(fb), D[j]);
                A[j] = __fadd2_rn(A[j], w[j]);
                T[j] = tn[j];
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
    uint32_t walk_max = 0;  // the tile's largest walk bound, for the backward's tile order
#pragma unroll
    for (int q = 0; q < PX; q++) {
        const int gx = x0 + col + q * HW;
        if (!(gy < H && gx < W)) continue;
        const int j = q >> 1;
        const bool h = q & 1;
        const float Tq = h ? T[j].y : T[j].x, Aq = h ? A[j].y : A[j].x, Dq = h ? D[j].y : D[j].x;
        const float rq = h ? cr[j].y : cr[j].x, gq = h ? cg[j].y : cg[j].x, bq = h ? cb[j].y : cb[j].x;
        const float pq = h ? pxl[j].y : pxl[j].x;
        const bool stopped = isnan(pq);
        const int walk = stopped ? (__float_as_int(pq) & 0x3fffff) : n;
        const int p = gy * W + gx;
        v.image[p] = rq + binf[0] * (1.f - Tq * bfar[0]);
        v.image[HWimg + p] = gq + binf[1] * (1.f - Tq * bfar[1]);
        v.image[2 * HWimg + p] = bq + binf[2] * (1.f - Tq * bfar[2]);
        const float z = Aq > 0.f ? Dq / Aq : zfar;
        if (v.depth) v.depth[p] = z;
        if (v.depth01) v.depth01[p] = 2.f / (1.f + expf(-0.1f * z)) - 1.f;
        v.final_T[p] = Tq;
        v.acc_alpha[p] = Aq;
        v.zhat[p] = z;
        // the backward's bound: every contributor lies in front of the
        // Gaussian that stopped the pixel (the entries between the last
        // contributor and it fail the 3-sigma or 1/255 test in both passes)
        const uint32_t bound = (uint32_t)(stopped ? walk - 1 : n);
        v.n_last[p] = bound;
        v.n_walk[p] = (uint32_t)walk;
        walk_max = max(walk_max, bound);
    }
    if (v.tile_walk) {
        __shared__ uint32_t s_walk[NT / 32];
        walk_max = __reduce_max_sync(0xffffffffu, walk_max);
        if ((tid & 31) == 0) s_walk[tid >> 5] = walk_max;
        __syncthreads();
        if (tid == 0) {
#pragma unroll
            for (int w = 1; w < NT / 32; w++) walk_max = max(walk_max, s_walk[w]);
            v.tile_walk[tile] = walk_max;
        }
    }
}

// ---------------------------------------------------------------------------
// Backward.

// State of the back-to-front walk for a pair of a thread's pixels (one FP32x2
// lane each).
struct PairB {
    float2 T;                 // transmittance behind the current Gaussian (starts at T_final)
    float2 S;                 // sum over Gaussians behind: w (G.ct + gD d + gA), plus the water term
    float2 G0, G1, G2, gD, gA;
    int last0, last1;         // walk bounds (list entries in front of the stop)
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

// Adjoint of a pixel pair at one Gaussian, lanes masked by on0 / on1: a lane
// that does not take part gets alpha = 0 (1 - alpha = 1, so its T, S and
// every accumulated term stay unchanged). ar: raw alpha per lane; dx: the
// lanes' column offsets; kc = {ct_r, ct_r, ct_g, ct_g}, kb = {ct_b, ct_b, d, d}.
// DG: the loss has a depth term (gD, gA non-zero). The exponent's gradient
// gqs enters the centre and conic gradients only through its moments: a0 =
// sum gqs dx, a2 = sum gqs dx^2, a5 = sum gqs over the thread's pixels (one
// row, so dy is shared); the dy moments and the conic coefficients are
// applied once per Gaussian.
template <bool DG>
__device__ __forceinline__ void pair_grad(PairB &p, float2 dx, float2 ar, bool on0, bool on1, float4 kc, float4 kb,
                                          float2 &a0, float2 &a2, float2 &a5, float2 &a6, float2 &a7, float2 &a8,
                                          float2 &a9)
{
    const float2 neg1 = make_float2(-1.f, -1.f), one = make_float2(1.f, 1.f);
    const float2 al = make_float2(on0 ? fminf(kAlphaMax, ar.x) : 0.f, on1 ? fminf(kAlphaMax, ar.y) : 0.f);
    const float2 om = __ffma2_rn(al, neg1, one);  // 1 - alpha
    const float2 inv = make_float2(rcp_approx(om.x), rcp_approx(om.y));
    const float2 Tj = __fmul2_rn(p.T, inv);       // transmittance in front of this Gaussian
    const float2 w = __fmul2_rn(al, Tj);
    const float2 u = DG ? __ffma2_rn(p.G0, lo2(kc), __ffma2_rn(p.G1, hi2(kc), __ffma2_rn(p.G2, lo2(kb),
                                                                                       __ffma2_rn(p.gD, hi2(kb), p.gA))))
                        : __ffma2_rn(p.G0, lo2(kc), __ffma2_rn(p.G1, hi2(kc), __fmul2_rn(p.G2, lo2(kb))));
    // dL/dalpha = T_j u - S / (1 - alpha)
    const float2 galpha = __ffma2_rn(__fmul2_rn(p.S, inv), neg1, __fmul2_rn(Tj, u));
    // the exponent's gradient up to its factor ln 2 (applied once per
    // Gaussian when the tile's sums are flushed)
    float2 gqs = __fmul2_rn(galpha, al);
    gqs.x = ar.x < kAlphaMax ? gqs.x : 0.f;  // zero through the alpha clamp
    gqs.y = ar.y < kAlphaMax ? gqs.y : 0.f;
    const float2 gx = __fmul2_rn(gqs, dx);
    a0 = __fadd2_rn(a0, gx);
    a2 = __ffma2_rn(gx, dx, a2);
    a5 = __fadd2_rn(a5, gqs);
    if (DG) a6 = __ffma2_rn(p.gD, w, a6);
    a7 = __ffma2_rn(p.G0, w, a7);
    a8 = __ffma2_rn(p.G1, w, a8);
    a9 = __ffma2_rn(p.G2, w, a9);
    p.S = __ffma2_rn(w, u, p.S);
    p.T = Tj;
}

template <int TW, int TH, int NB, bool DG>
__device__ __forceinline__ void blend_tile_bwd(const BlendView &v, int tile, const float *__restrict__ medium)
{
    constexpr int PX = kPxBwd, NP = PX / 2;
    constexpr int NT = Tile<TW, TH, PX>::NT, HW = Tile<TW, TH, PX>::HW;
    constexpr int NW = NT / 32;
    __shared__ float4 sx[NB], sy[NB], sc[NB], sk[NB], sb[NB];
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
    float2 pxl[NP];
    PairB P[NP];
    int mylast = 0;
#pragma unroll
    for (int jp = 0; jp < NP; jp++) {
        float T[2] = {1.f, 1.f}, S[2] = {0.f, 0.f}, G0[2] = {0.f, 0.f}, G1[2] = {0.f, 0.f}, G2[2] = {0.f, 0.f};
        float gD[2] = {0.f, 0.f}, gA[2] = {0.f, 0.f}, px[2];
        int last[2] = {0, 0};
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int q = 2 * jp + h;
            const int gx = x0 + col + q * HW;
            px[h] = (float)(x0 - ox + col + q * HW) + 0.5f;
            if (!(gy < H && gx < W)) continue;
            const int pix = gy * W + gx;
            T[h] = v.final_T[pix];
            last[h] = (int)v.n_last[pix];
            G0[h] = v.dL_dimage[pix];
            G1[h] = v.dL_dimage[HWimg + pix];
            G2[h] = v.dL_dimage[2 * HWimg + pix];
            if (DG) {
                const float A = v.acc_alpha[pix], z = v.zhat[pix];
                float gz = v.dL_ddepth ? v.dL_ddepth[pix] : 0.f;
                if (v.dL_ddepth01) {
                    const float e = expf(-0.1f * z);
                    gz += v.dL_ddepth01[pix] * 0.2f * e / ((1.f + e) * (1.f + e));
                }
                if (A > 0.f) {
                    gD[h] = gz / A;  // z = D / A
                    gA[h] = -gz * z / A;
                }
            }
            const float Gc[3] = {G0[h], G1[h], G2[h]};
#pragma unroll
            for (int ch = 0; ch < 3; ch++) {
                mB[ch] += Gc[ch] * (1.f - T[h] * bfar[ch]);
                mBB[ch] += Gc[ch] * binf[ch] * T[h] * zfar * bfar[ch];
                S[h] -= Gc[ch] * binf[ch] * bfar[ch] * T[h];  // the water behind the last Gaussian
            }
            mylast = max(mylast, last[h]);
        }
        pxl[jp] = make_float2(px[0], px[1]);
        PairB &p = P[jp];
        p.T = make_float2(T[0], T[1]);
        p.S = make_float2(S[0], S[1]);
        p.G0 = make_float2(G0[0], G0[1]);
        p.G1 = make_float2(G1[0], G1[1]);
        p.G2 = make_float2(G2[0], G2[1]);
        p.gD = make_float2(gD[0], gD[1]);
        p.gA = make_float2(gA[0], gA[1]);
        p.last0 = last[0];
        p.last1 = last[1];
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
    const float2 pyl2 = make_float2(pyl, pyl);

    for (int bend = maxlast; bend > 0; bend -= NB) {
        const int b0 = max(0, bend - NB);
        const int nb = bend - b0;
        __syncthreads();  // the previous batch's flush has read s_g / s_id
        for (int sl = tid; sl < nb; sl += NT) {
            const uint32_t gid = v.gauss_ids[rg.x + b0 + sl];
            stage_fwd(v.rec, gid, ox, oy, sx, sy, sc, sk, sb, nullptr, sl);
            s_id[sl] = gid;
        }
        for (int sl = tid; sl < NB; sl += NT)
#pragma unroll
            for (int f = 0; f < 10; f++) s_g[f][sl] = 0.f;
        __syncthreads();
        if (__any_sync(0xffffffffu, mylast > b0)) {
            for (int k = nb - 1; k >= 0; k--) {
                const int j = b0 + k;
                const float4 fx = sx[k], fy = sy[k], fc = sc[k];
                const float th = exponent_threshold(fc.z);  // as the forward staged it
                const float2 dy = __fadd2_rn(pyl2, lo2(fy));
                const float2 Bdy = __fmul2_rn(hi2(fy), dy);
                const float2 Cdy2 = __fmul2_rn(__fmul2_rn(lo2(fc), dy), dy);
                // the exponent and raw alpha of all the thread's pixels first, without
                // branches (independent chains the scheduler can overlap); a pixel
                // takes part if the Gaussian is in front of its walk bound and its
                // exponent reaches the threshold (within 3 sigma, at least 1/255
                // opaque)
                float2 dx[NP], ar[NP];
                bool on0[NP], on1[NP];
                bool any = false;
#pragma unroll
                for (int jp = 0; jp < NP; jp++) {
                    dx[jp] = __fadd2_rn(pxl[jp], lo2(fx));
                    const float2 qs = __ffma2_rn(dx[jp], __ffma2_rn(hi2(fx), dx[jp], Bdy), Cdy2);
                    const float2 e = __fadd2_rn(qs, hi2(fc));
                    ar[jp] = make_float2(ex2_approx(e.x), ex2_approx(e.y));
                    on0[jp] = (j < P[jp].last0) & (qs.x >= th);
                    on1[jp] = (j < P[jp].last1) & (qs.y >= th);
                    any |= on0[jp] | on1[jp];
                }
                if (!__any_sync(0xffffffffu, any)) continue;
                float2 a0 = make_float2(0.f, 0.f), a2 = a0, a5 = a0, a6 = a0, a7 = a0, a8 = a0, a9 = a0;
                const float4 kc = sk[k], kb = sb[k];
                // both pairs, masked, without a branch: their dependency chains overlap
#pragma unroll
                for (int jp = 0; jp < NP; jp++)
                    pair_grad<DG>(P[jp], dx[jp], ar[jp], on0[jp], on1[jp], kc, kb, a0, a2, a5, a6, a7, a8, a9);
                float acc[10];
                const float dys = dy.x;
                acc[0] = a0.x + a0.y;
                acc[2] = a2.x + a2.y;
                acc[5] = a5.x + a5.y;
                acc[6] = DG ? a6.x + a6.y : 0.f;
                acc[7] = a7.x + a7.y;
                acc[8] = a8.x + a8.y;
                acc[9] = a9.x + a9.y;
                // moments in y from the row's dy: sum gqs dy, sum gqs dx dy, sum gqs dy^2
                acc[1] = acc[5] * dys;
                acc[3] = acc[0] * dys;
                acc[4] = acc[5] * (dys * dys);
                const float r = warp_reduce10(acc, lane);
                if (my_field >= 0) atomicAdd(&s_g[my_field][k], r);
            }
        }
        __syncthreads();
        for (int sl = tid; sl < nb; sl += NT) {
            // fields 0-5 (the exponent moments) carry the factor ln 2 from here
            const float g[10] = {kLn2 * s_g[0][sl], kLn2 * s_g[1][sl], kLn2 * s_g[2][sl], kLn2 * s_g[3][sl],
                                 kLn2 * s_g[4][sl], kLn2 * s_g[5][sl], s_g[6][sl], s_g[7][sl], s_g[8][sl], s_g[9][sl]};
            bool nz = false;
#pragma unroll
            for (int f = 0; f < 10; f++) nz |= g[f] != 0.f;
            if (nz) {
                // centre gradient from the moments: dqs/dx = 2A dx + B dy, dqs/dy = B dx + 2C dy
                const float A = sx[sl].z, B = sy[sl].z, C = sc[sl].x;
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

// occupancy target: 16 blocks of 64 threads per SM (64 registers)
template <int TW, int TH, int NB>
__global__ void __launch_bounds__(fwd_threads<TW, TH>(), 1024 / fwd_threads<TW, TH>()) k_blend_fwd(BlendView v, const float *__restrict__ medium)
{
    pdl_enter();
    blend_tile_fwd<TW, TH, NB>(v, blockIdx.x, medium);
}

// occupancy target: 12 blocks of 64 threads per SM without the depth terms
// (80 registers, no spills), 11 with them
template <int TW, int TH, int NB, bool DG>
__global__ void __launch_bounds__(bwd_threads<TW, TH>(), (DG ? 704 : 768) / bwd_threads<TW, TH>()) k_blend_bwd(BlendView v, const float *__restrict__ medium)
{
    pdl_enter();
    blend_tile_bwd<TW, TH, NB, DG>(v, v.tile_order ? (int)v.tile_order[blockIdx.x] : (int)blockIdx.x, medium);
}

// The backward's tile order: tiles by descending walk bound, so that the
// longest tiles start in the first wave instead of trailing the last one (one
// CTA per tile, handed out in launch order). A counting sort over
// kOrderBuckets walk values in one CTA: histogram, exclusive scan, scatter.
// Walks past the last bucket share it; the order within a bucket is the order
// of the scatter's shared-memory atomics (any order is a valid schedule).
constexpr int kOrderThreads = 1024, kOrderBuckets = 2 * kOrderThreads;
constexpr int kOrderItems = 16;  // walk values per thread and round, all loaded before the first atomic
__device__ __forceinline__ uint32_t walk_bucket(uint32_t w)
{
    return kOrderBuckets - 1 - min(w, (uint32_t)(kOrderBuckets - 1));
}
__global__ void __launch_bounds__(kOrderThreads) k_tile_order(const uint32_t *__restrict__ walk, int ntiles,
                                                              uint32_t *__restrict__ order)
{
    __shared__ uint32_t cnt[kOrderBuckets];
    __shared__ uint32_t wsum[kOrderThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kRound = kOrderThreads * kOrderItems;
    cnt[tid] = 0;
    cnt[tid + kOrderThreads] = 0;
    __syncthreads();
    for (int base = 0; base < ntiles; base += kRound) {
        uint32_t b[kOrderItems];
#pragma unroll
        for (int j = 0; j < kOrderItems; j++) {
            const int i = base + j * kOrderThreads + tid;
            b[j] = i < ntiles ? walk_bucket(__ldg(walk + i)) : 0xffffffffu;
        }
#pragma unroll
        for (int j = 0; j < kOrderItems; j++)
            if (b[j] != 0xffffffffu) atomicAdd(&cnt[b[j]], 1u);
    }
    __syncthreads();
    // thread t owns buckets 2t and 2t + 1
    const uint32_t c0 = cnt[2 * tid], c1 = cnt[2 * tid + 1];
    uint32_t incl = c0 + c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = wsum[lane], wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        wsum[lane] = wi - w;  // exclusive over warps
    }
    __syncthreads();
    const uint32_t excl = wsum[warp] + incl - (c0 + c1);
    cnt[2 * tid] = excl;
    cnt[2 * tid + 1] = excl + c0;
    __syncthreads();
    for (int base = 0; base < ntiles; base += kRound) {
        uint32_t b[kOrderItems];
#pragma unroll
        for (int j = 0; j < kOrderItems; j++) {
            const int i = base + j * kOrderThreads + tid;
            b[j] = i < ntiles ? walk_bucket(__ldg(walk + i)) : 0xffffffffu;
        }
#pragma unroll
        for (int j = 0; j < kOrderItems; j++)
            if (b[j] != 0xffffffffu) order[atomicAdd(&cnt[b[j]], 1u)] = (uint32_t)(base + j * kOrderThreads + tid);
    }
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
__global__ void __launch_bounds__(fwd_threads<TW, TH>(), 1024 / fwd_threads<TW, TH>()) k_blend_fwd_persistent(const BlendView *__restrict__ views,
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
        // a plain launch: started early behind the binning kernels (programmatic
        // launch) the training step ran 0.17 ms slower on the B300
        k_blend_fwd<TW, TH, NB><<<v.tg.tx * v.tg.ty, fwd_threads<TW, TH>(), 0, s>>>(v, medium);
        count_launch();
    }
};
template <int TW, int TH, int NB>
struct BwdPlain {
    static void run(const BlendView &v, const float *medium, cudaStream_t s)
    {
        if (v.dL_ddepth || v.dL_ddepth01)
            launch_pdl(k_blend_bwd<TW, TH, NB, true>, v.tg.tx * v.tg.ty, bwd_threads<TW, TH>(), 0, s, v, medium);
        else
            launch_pdl(k_blend_bwd<TW, TH, NB, false>, v.tg.tx * v.tg.ty, bwd_threads<TW, TH>(), 0, s, v, medium);
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

void launch_tile_order(const uint32_t *tile_walk, int ntiles, uint32_t *order, cudaStream_t s)
{
    if (ntiles <= 0) return;
    k_tile_order<<<1, kOrderThreads, 0, s>>>(tile_walk, ntiles, order);
    count_launch();
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
