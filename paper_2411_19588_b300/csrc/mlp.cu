// Learned warm-start (the paper has no learned part; this form predicts the
// nine per-channel medium parameters of Eq. 4-5 from one rendered view so the
// fit of Sec. IV-C can start from them):
//   * featuriser: 32x32 adaptive-average downsample of the image + 8-bin
//     histogram of the Eq. 6 depth over [0, z_far], stored as one BF16 row;
//   * 3080 -> 128 -> 128 -> 9 MLP with BF16 weights and FP32 accumulation on
//     the 5th-generation tensor cores: operands staged by TMA (128-byte
//     swizzle) through an mbarrier ring, tcgen05.mma issued by one thread,
//     accumulators in tensor memory, epilogue through tcgen05.ld;
//   * fused Adam + BF16 refresh of the weights.
// Every bias rides as one more input column that multiplies a constant 1, so
// the bias gradients come out of the weight-gradient GEMMs (no atomics).
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

#include "host.h"
#include "splash.h"

namespace splash {
namespace mlp {

constexpr int kGrid = 32, kBins = 8;
constexpr int kImg = 3 * kGrid * kGrid;  // 3072
constexpr int kIn = kImg + kBins;        // 3080 features
constexpr int kK1 = 3136;                // row width: features, bias 1, zeros
constexpr int kHid = 128;
constexpr int kK2 = 192;                 // hidden width: 128 units, bias 1, zeros
constexpr int kOut = 9;
constexpr int kOutPad = 16;              // output GEMM width
constexpr int kDyPad = 64;               // dY width (K of one stage)

// GEMM tiling: one CTA computes a 128 x nt tile of D = A B^T, K in slices of 64
constexpr int kBM = 128, kBK = 64, kStages = 4, kMaxNT = 256;
constexpr int kStageA = kBM * kBK * 2;       // 16 KB
constexpr int kStageB = kMaxNT * kBK * 2;    // 32 KB
constexpr int kTileBytes = kStages * (kStageA + kStageB);
constexpr int kGemmSmem = kTileBytes + 1024 + 128;  // + alignment slack + barriers

enum Epi : int { kEpiF32 = 0, kEpiReluBf16 = 1, kEpiDReluBf16 = 2 };

struct GemmArgs {
    int nt, nk, tcols, epi;
    float *d;
    int64_t ldd;
    __nv_bfloat16 *out, *out_t;   // row-major [m][n] and transposed [n][m] (either may be null)
    int64_t ld_out, ld_t;
    const __nv_bfloat16 *ref;     // ReLU mask source for kEpiDReluBf16 ([m][n])
    int64_t ld_ref;
    uint32_t *status;
    uint32_t spin;
};

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bounded wait for the completion of the phase with the given parity: a
// non-blocking test with a short sleep after the first polls, so `limit`
// bounds the time spent (about limit x 0.1 us).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; i++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (i >= 64) __nanosleep(64);
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_alloc(uint32_t slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// D (tensor memory) (+)= A (shared) * B (shared)^T, both K-major BF16, FP32 accumulate
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// the barrier receives one arrival once every MMA this thread issued so far has completed
__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// 16 consecutive FP32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    // the registers are defined only after the wait; tie them to it
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor of a K-major tile whose rows are 128 bytes
// (64 BF16) written by TMA with the 128-byte swizzle: 8-row atoms of 1024 B,
// so the stride between row groups is 1024 B; the leading offset is unused
// for this layout. Tiles start 1024-aligned; a K step of 16 inside the row
// advances the start address by 32 B.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr)
{
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;           // leading byte offset (16 B, ignored here)
    d |= (uint64_t)(1024 >> 4) << 32; // stride byte offset
    d |= (uint64_t)1 << 46;           // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;           // 128-byte swizzle
    return d;
}
// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void store_bf16x16(__nv_bfloat16 *dst, const float (&v)[16])
{
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        w[i] = *reinterpret_cast<uint32_t *>(&p);
    }
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    d[0] = make_uint4(w[0], w[1], w[2], w[3]);
    d[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// D[m0:m0+128, n0:n0+nt] = A[m, :] . B[n, :] over K = 64 nk.
// Warp 0 (one lane) feeds the ring with TMA, warp 1 (one lane) issues the
// MMAs, warp 2 owns the tensor-memory allocation, and all four warps run the
// epilogue (warp w reads accumulator lanes 32w..32w+31 = rows of D).
__global__ void __launch_bounds__(128, 1)
k_gemm_bf16(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, const GemmArgs g)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint32_t s_tmem, s_fail, s_issued, s_consumed;
    uint8_t *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t *tiles_a = base;
    uint8_t *tiles_b = base + kStages * kStageA;
    const uint32_t bars = smem_u32(base + kTileBytes);
    const uint32_t full = bars, empty = bars + 8 * kStages, done = bars + 16 * kStages;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * g.nt;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(full + 8 * s, 1);
            mbar_init(empty + 8 * s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
    }
    if (warp == 2) tc_alloc(smem_u32(&s_tmem), (uint32_t)g.tcols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (warp == 0 && lane == 0) {
        const uint32_t bytes = (uint32_t)(kBM + g.nt) * kBK * 2;
        int k = 0;
        for (; k < g.nk; k++) {
            const int s = k % kStages;
            if (k >= kStages && !mbar_wait(empty + 8 * s, ((k / kStages) - 1) & 1, g.spin)) {
                s_fail = 1;
                break;
            }
            mbar_expect_tx(full + 8 * s, bytes);
            tma_load_2d(smem_u32(tiles_a + s * kStageA), &map_a, full + 8 * s, k * kBK, m0);
            tma_load_2d(smem_u32(tiles_b + s * kStageB), &map_b, full + 8 * s, k * kBK, n0);
        }
        s_issued = (uint32_t)k;
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = idesc_bf16(kBM, g.nt);
        int k = 0;
        for (; k < g.nk; k++) {
            const int s = k % kStages;
            if (!mbar_wait(full + 8 * s, (k / kStages) & 1, g.spin)) {
                s_fail = 1;
                break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(tiles_a + s * kStageA), b0 = smem_u32(tiles_b + s * kStageB);
#pragma unroll
            for (int kk = 0; kk < kBK / 16; kk++)
                tc_mma(tmem, sw128_desc(a0 + 32 * kk), sw128_desc(b0 + 32 * kk), idesc, (k | kk) != 0);
            tc_commit(empty + 8 * s);
        }
        s_consumed = (uint32_t)k;
        tc_commit(done);
    }
    __syncthreads();

    const bool ok = mbar_wait(done, 0, g.spin) && !s_fail;
    tc_fence_after();
    if (ok) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c = 0; c < g.nt; c += 16) {
            float v[16];
            tc_ld16(lane_addr + (uint32_t)c, v);
            const int n = n0 + c;
            if (g.epi == kEpiF32) {
                float4 *d = reinterpret_cast<float4 *>(g.d + (int64_t)row * g.ldd + n);
#pragma unroll
                for (int i = 0; i < 4; i++) d[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            } else {
                if (g.epi == kEpiReluBf16) {
#pragma unroll
                    for (int i = 0; i < 16; i++) v[i] = fmaxf(v[i], 0.f);
                } else {
                    const uint4 *r = reinterpret_cast<const uint4 *>(g.ref + (int64_t)row * g.ld_ref + n);
                    const uint4 q[2] = {r[0], r[1]};
                    const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(q);
#pragma unroll
                    for (int i = 0; i < 16; i++) v[i] = __bfloat162float(h[i]) > 0.f ? v[i] : 0.f;
                }
                if (g.out) store_bf16x16(g.out + (int64_t)row * g.ld_out + n, v);
                if (g.out_t) {
#pragma unroll
                    for (int i = 0; i < 16; i++) g.out_t[(int64_t)(n + i) * g.ld_t + row] = __float2bfloat16_rn(v[i]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && !ok) {
        atomicOr(g.status, kStatusTimeout);
        // let copies still in flight land before the shared memory is released
        for (uint32_t k = s_consumed; k < s_issued; k++) mbar_wait(full + 8 * (k % kStages), (k / kStages) & 1, g.spin);
    }
    if (warp == 2) {
        tc_fence_after();
        tc_dealloc(tmem, (uint32_t)g.tcols);
    }
}

// ------------------------------------------------------------------ featuriser
__device__ __forceinline__ int cell_lo(int i, int n) { return (i * n) / kGrid; }
__device__ __forceinline__ int cell_hi(int i, int n) { return ((i + 1) * n + kGrid - 1) / kGrid; }

// One CTA per output cell (blockIdx.x = column j, blockIdx.y = row i): the
// three channel means over the adaptive-pooling block, and the depth
// histogram of the disjoint block [floor(iH/32), floor((i+1)H/32)) x (same in x).
__global__ void __launch_bounds__(256) k_featurise_cells(const float *__restrict__ image, const float *__restrict__ depth,
                                                          int W, int H, float z_far, __nv_bfloat16 *row,
                                                          uint32_t *counts)
{
    __shared__ float s_sum[3][8];
    __shared__ uint32_t s_cnt[kBins];
    const int i = blockIdx.y, j = blockIdx.x;
    const int y0 = cell_lo(i, H), y1 = cell_hi(i, H), x0 = cell_lo(j, W), x1 = cell_hi(j, W);
    const int cw = x1 - x0, npx = (y1 - y0) * cw;
    const int64_t plane = (int64_t)W * H;
    if (threadIdx.x < kBins) s_cnt[threadIdx.x] = 0;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    for (int t = threadIdx.x; t < npx; t += blockDim.x) {
        const int64_t p = (int64_t)(y0 + t / cw) * W + x0 + t % cw;
        a0 += image[p];
        a1 += image[plane + p];
        a2 += image[2 * plane + p];
    }
    __syncthreads();
    // depth histogram of the disjoint block; the bin is decided in FP32
    const int hy0 = cell_lo(i, H), hy1 = cell_lo(i + 1, H), hx0 = cell_lo(j, W), hx1 = cell_lo(j + 1, W);
    const int hw = hx1 - hx0, nh = (hy1 - hy0) * hw;
    for (int t = threadIdx.x; t < nh; t += blockDim.x) {
        const float z = depth[(int64_t)(hy0 + t / hw) * W + hx0 + t % hw];
        const float q = floorf(__fdiv_rn(__fmul_rn(z, (float)kBins), z_far));
        const int b = (q >= 0.f) ? ((q < (float)(kBins - 1)) ? (int)q : kBins - 1) : 0;  // NaN -> last bin
        atomicAdd(&s_cnt[(q != q) ? kBins - 1 : b], 1u);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_sum[0][warp] = a0;
        s_sum[1][warp] = a1;
        s_sum[2][warp] = a2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        float s = 0.f;
        for (int w = 0; w < 8; w++) s += s_sum[threadIdx.x][w];
        row[threadIdx.x * kGrid * kGrid + i * kGrid + j] = __float2bfloat16_rn(__fdiv_rn(s, (float)npx));
    }
    if (threadIdx.x < kBins && s_cnt[threadIdx.x]) atomicAdd(&counts[threadIdx.x], s_cnt[threadIdx.x]);
}

// Histogram fractions, the bias input and the zero tail; clears the counters.
__global__ void k_featurise_finish(uint32_t *counts, float npix, __nv_bfloat16 *row)
{
    const int t = threadIdx.x;
    if (t < kBins) {
        row[kImg + t] = __float2bfloat16_rn(__fdiv_rn((float)counts[t], npix));
        counts[t] = 0;
    }
    for (int c = kIn + t; c < kK1; c += blockDim.x) row[c] = __float2bfloat16_rn(c == kIn ? 1.f : 0.f);
}

// ------------------------------------------------------------------ MLP pieces
// X[b] = bank[idx[b]] (or bank[b] without idx) for b < B, zero rows up to Bp;
// the transposed copy Xt[f][b]; targets T[b] = tbank[idx[b]].
__global__ void __launch_bounds__(256) k_mlp_gather(const __nv_bfloat16 *__restrict__ bank, const int32_t *__restrict__ idx,
                                                     int64_t n_rows, const float *__restrict__ tbank, int B, int Bp,
                                                     __nv_bfloat16 *X, __nv_bfloat16 *Xt, float *T, uint32_t *status)
{
    __shared__ uint16_t tile[64][64 + 8];
    const int b0 = blockIdx.x * 64, f0 = blockIdx.y * 64;
    const int t = threadIdx.x, r = t >> 2, q = t & 3;
    const int b = b0 + r;
    uint4 v0 = make_uint4(0, 0, 0, 0), v1 = v0;
    if (b < B) {
        int64_t src = idx ? (int64_t)idx[b] : (int64_t)b;
        if (src < 0 || src >= n_rows) {  // never read outside the bank; report it
            if (blockIdx.y == 0 && q == 0) atomicOr(status, kStatusIndex);
            src = src < 0 ? 0 : n_rows - 1;
        }
        const uint4 *p = reinterpret_cast<const uint4 *>(bank + src * kK1 + f0 + q * 16);
        v0 = p[0];
        v1 = p[1];
        if (blockIdx.y == 0 && q == 0 && tbank)
            for (int k = 0; k < kOut; k++) T[(int64_t)b * kOut + k] = tbank[src * kOut + k];
    }
    uint4 *d = reinterpret_cast<uint4 *>(X + (int64_t)b * kK1 + f0 + q * 16);
    d[0] = v0;
    d[1] = v1;
    const uint16_t *h0 = reinterpret_cast<const uint16_t *>(&v0), *h1 = reinterpret_cast<const uint16_t *>(&v1);
#pragma unroll
    for (int k = 0; k < 8; k++) {
        tile[r][q * 16 + k] = h0[k];
        tile[r][q * 16 + 8 + k] = h1[k];
    }
    __syncthreads();
    // transposed: thread (fr, q) writes samples q*16 .. q*16+15 of feature f0 + fr
    uint32_t w[8];
#pragma unroll
    for (int k = 0; k < 8; k++) w[k] = (uint32_t)tile[q * 16 + 2 * k][r] | ((uint32_t)tile[q * 16 + 2 * k + 1][r] << 16);
    uint4 *dt = reinterpret_cast<uint4 *>(Xt + (int64_t)(f0 + r) * Bp + b0 + q * 16);
    dt[0] = make_uint4(w[0], w[1], w[2], w[3]);
    dt[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

__device__ __forceinline__ float softplus_f(float y) { return y > 20.f ? y : log1pf(expf(y)); }
__device__ __forceinline__ float sigmoid_f(float y) { return 1.f / (1.f + expf(-y)); }

// Heads (softplus for beta_D, beta_B; sigmoid for B_inf), predictions, and
// with targets the loss mean|log p - log t| and dL/dY as BF16 ([b][k] and [k][b]).
__global__ void __launch_bounds__(256) k_mlp_head(const float *__restrict__ Y, const float *__restrict__ T, int B, int Bp,
                                                   float *pred, __nv_bfloat16 *dY, __nv_bfloat16 *dYt, float *loss)
{
    __shared__ float s_red[8];
    const float inv = 1.f / (float)(B * kOut);
    float acc = 0.f;
    for (int e = threadIdx.x; e < Bp * kOut; e += blockDim.x) {
        const int b = e / kOut, k = e % kOut;
        if (b >= B) {  // rows past the batch carry no gradient (they may hold an earlier batch's)
            if (T) {
                dY[(int64_t)b * kDyPad + k] = __float2bfloat16_rn(0.f);
                dYt[(int64_t)k * Bp + b] = __float2bfloat16_rn(0.f);
            }
            continue;
        }
        const float y = Y[(int64_t)b * kOutPad + k];
        const float p = k < 6 ? softplus_f(y) : sigmoid_f(y);
        if (pred) pred[e] = p;
        if (T) {
            const float u = logf(p) - logf(T[e]);
            acc += fabsf(u);
            const float dlogp = k < 6 ? sigmoid_f(y) / p : 1.f - p;
            const float sg = (u > 0.f) ? 1.f : ((u < 0.f) ? -1.f : 0.f);
            const __nv_bfloat16 gb = __float2bfloat16_rn(sg * dlogp * inv);
            dY[(int64_t)b * kDyPad + k] = gb;
            dYt[(int64_t)k * Bp + b] = gb;
        }
    }
    if (!T) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += s_red[w];
        loss[0] = s * inv;
    }
}

struct LayerRef {
    float *p, *m, *v;
    const float *g;
    __nv_bfloat16 *wb, *wt;  // BF16 copies [rows][cols] and [cols][ld_t] (wt may be null)
    int rows, cols, ld_t;
    int64_t start;           // first flat index of this layer in the launch
};
struct AdamCast {
    LayerRef L[3];
    int64_t total;
    float lr;
    AdamHyper h;
    int do_adam;
};

// One Adam step on the FP32 masters (optional) and the BF16 refresh of each
// layer's weights and transposed weights.
__global__ void __launch_bounds__(256) k_mlp_adam_cast(const AdamCast a)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.total) return;
    const int l = e < a.L[1].start ? 0 : (e < a.L[2].start ? 1 : 2);
    const LayerRef &L = a.L[l];
    const int64_t k = e - L.start;
    float p = L.p[k];
    if (a.do_adam) {
        float m = L.m[k], v = L.v[k];
        adam_update(p, L.g[k], m, v, a.lr, a.h);
        L.p[k] = p;
        L.m[k] = m;
        L.v[k] = v;
    }
    const __nv_bfloat16 pb = __float2bfloat16_rn(p);
    L.wb[k] = pb;
    if (L.wt) {
        const int r = (int)(k / L.cols), c = (int)(k % L.cols);
        L.wt[(int64_t)c * L.ld_t + r] = pb;
    }
}

// ------------------------------------------------------------------ host side
using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;

EncodeFn encoder()
{
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// [rows x cols] BF16 row-major with leading dimension ld (elements); boxes of
// 64 columns x box_rows rows with the 128-byte swizzle.
bool make_map(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows)
{
    EncodeFn enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// N tile: 256 when that still gives every SM a tile, else the largest
// multiple of 16 up to 128 that divides N (small GEMMs spread over more CTAs)
int pick_nt(int M, int N)
{
    if (N % 256 == 0 && (int64_t)(M / kBM) * (N / 256) >= 148) return 256;
    for (int nt = 128; nt >= 16; nt -= 16)
        if (N % nt == 0) return nt;
    return 0;
}
int tmem_cols(int nt)
{
    int c = 32;
    while (c < nt) c <<= 1;
    return c;
}

struct Gemm {
    CUtensorMap a, b;
    int M = 0, N = 0, K = 0;
    GemmArgs args{};
};

splash_status launch_gemm(const Gemm &g, cudaStream_t s)
{
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] { attr = cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem); });
    if (attr != cudaSuccess) return splash_host::fail(SPLASH_ERR_CUDA, "cannot raise the GEMM shared-memory limit");
    const dim3 grid(g.M / kBM, g.N / g.args.nt);
    k_gemm_bf16<<<grid, 128, kGemmSmem, s>>>(g.a, g.b, g.args);
    count_launch();
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}

// Build a GEMM D[M x N] = A[M x K] B[N x K]^T
bool setup_gemm(Gemm &g, const void *A, int64_t lda, const void *B, int64_t ldb, int M, int N, int K, uint32_t *status,
                uint32_t spin)
{
    g.M = M;
    g.N = N;
    g.K = K;
    g.args = GemmArgs{};
    g.args.nt = pick_nt(M, N);
    g.args.nk = K / kBK;
    g.args.tcols = tmem_cols(g.args.nt);
    g.args.status = status;
    g.args.spin = spin;
    return g.args.nt > 0 && make_map(&g.a, A, M, K, lda, kBM) && make_map(&g.b, B, N, K, ldb, g.args.nt);
}

}  // namespace mlp
}  // namespace splash

using namespace splash;
using namespace splash::mlp;
using splash_host::fail;

namespace {
constexpr uint32_t kMlpSpin = 1u << 22;
inline bool al16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
}  // namespace

extern "C" splash_status splash_gemm_bf16(splash_ctx *ctx, const uint16_t *A, int64_t lda, const uint16_t *B, int64_t ldb,
                                          float *D, int64_t ldd, int32_t M, int32_t N, int32_t K, void *stream)
{
    if (!ctx || !A || !B || !D) return fail(SPLASH_ERR_INVALID_ARG, "null context or matrix");
    if (M <= 0 || N <= 0 || K <= 0 || M % 128 || N % 16 || K % 64)
        return fail(SPLASH_ERR_INVALID_ARG, "need M % 128 == 0, N % 16 == 0, K % 64 == 0, all positive");
    if (lda < K || ldb < K || lda % 8 || ldb % 8 || ldd < N || ldd % 4)
        return fail(SPLASH_ERR_INVALID_ARG, "lda, ldb must be >= K and multiples of 8; ldd >= N and a multiple of 4");
    if (!al16(A) || !al16(B) || !al16(D)) return fail(SPLASH_ERR_INVALID_ARG, "A, B and D must be 16-byte aligned");
    Gemm g;
    if (!setup_gemm(g, A, lda, B, ldb, M, N, K, ctx->d_status, kMlpSpin))
        return fail(SPLASH_ERR_CUDA, "tensor map encoding failed");
    g.args.epi = kEpiF32;
    g.args.d = D;
    g.args.ldd = ldd;
    return launch_gemm(g, (cudaStream_t)stream);
}

extern "C" splash_status splash_featurise(splash_ctx *ctx, const float *image, const float *depth, int32_t width,
                                          int32_t height, float z_far, uint16_t *row, void *stream)
{
    if (!ctx || !image || !depth || !row) return fail(SPLASH_ERR_INVALID_ARG, "null context, image, depth or row");
    if (width <= 0 || height <= 0 || (int64_t)width * height >= ((int64_t)1 << 31))
        return fail(SPLASH_ERR_INVALID_ARG, "image size must be positive and below 2^31 pixels");
    if (!(z_far > 0.f)) return fail(SPLASH_ERR_INVALID_ARG, "z_far must be positive");
    cudaStream_t s = (cudaStream_t)stream;
    if (!ctx->feat_counts.p) {
        ENSURE(ctx->feat_counts, kBins * sizeof(uint32_t));
        SPLASH_CUDA_TRY(cudaMemsetAsync(ctx->feat_counts.p, 0, kBins * sizeof(uint32_t), s));
    }
    uint32_t *counts = ctx->feat_counts.as<uint32_t>();
    __nv_bfloat16 *r = reinterpret_cast<__nv_bfloat16 *>(row);
    k_featurise_cells<<<dim3(kGrid, kGrid), 256, 0, s>>>(image, depth, width, height, z_far, r, counts);
    k_featurise_finish<<<1, 64, 0, s>>>(counts, (float)((int64_t)width * height), r);
    count_launch(2);
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}

struct splash_mlp {
    splash_ctx *ctx = nullptr;
    int Bp = 0;
    int step = 0;
    // FP32 masters (augmented: bias column, zero padding), moments, gradients
    splash_host::Buf P1, P2, P3, M1, M2, M3, V1, V2, V3, G1, G2, G3;
    // BF16 weights and transposed weights
    splash_host::Buf W1, W2, W2t, W3, W3t;
    // activations and backward signals
    splash_host::Buf X, Xt, H1, H1t, H2, H2t, Y, dY, dYt, dZ2, dZ2t, dZ1t, T, loss;
    Gemm f1, f2, f3, b1, b2, b3, b4, b5;
};

namespace {
template <class T>
T *bf(splash_host::Buf &b) { return b.as<T>(); }

splash_status mlp_forward(splash_mlp *m, cudaStream_t s)
{
    splash_status st;
    if ((st = launch_gemm(m->f1, s)) != SPLASH_OK) return st;
    if ((st = launch_gemm(m->f2, s)) != SPLASH_OK) return st;
    return launch_gemm(m->f3, s);
}

splash_status mlp_gather(splash_mlp *m, const uint16_t *bank, int64_t n_rows, const int32_t *idx, const float *tbank,
                         int B, cudaStream_t s)
{
    k_mlp_gather<<<dim3(m->Bp / 64, kK1 / 64), 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16 *>(bank), idx, n_rows,
                                                            tbank, B, m->Bp, bf<__nv_bfloat16>(m->X),
                                                            bf<__nv_bfloat16>(m->Xt), m->T.as<float>(),
                                                            m->ctx->d_status);
    count_launch();
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}

splash_status mlp_adam_cast(splash_mlp *m, const splash_mlp_adam *adam, cudaStream_t s)
{
    AdamCast a{};
    auto layer = [&](int l, splash_host::Buf &P, splash_host::Buf &Mo, splash_host::Buf &Vo, splash_host::Buf &G,
                     splash_host::Buf &Wb, __nv_bfloat16 *wt, int rows, int cols, int ld_t, int64_t start) {
        a.L[l] = LayerRef{P.as<float>(), Mo.as<float>(), Vo.as<float>(), G.as<float>(), Wb.as<__nv_bfloat16>(), wt,
                          rows, cols, ld_t, start};
        return start + (int64_t)rows * cols;
    };
    int64_t e = layer(0, m->P1, m->M1, m->V1, m->G1, m->W1, nullptr, kHid, kK1, 0, 0);
    e = layer(1, m->P2, m->M2, m->V2, m->G2, m->W2, bf<__nv_bfloat16>(m->W2t), kHid, kK2, kHid, e);
    e = layer(2, m->P3, m->M3, m->V3, m->G3, m->W3, bf<__nv_bfloat16>(m->W3t), kOutPad, kK2, kDyPad, e);
    a.total = e;
    a.do_adam = adam != nullptr;
    if (adam) {
        a.lr = adam->lr;
        a.h = make_adam_hyper(adam->beta1, adam->beta2, adam->eps, m->step);
    }
    k_mlp_adam_cast<<<(unsigned)((a.total + 255) / 256), 256, 0, s>>>(a);
    count_launch();
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}

// natural <-> augmented parameter copies (strided device copies)
splash_status copy_params(splash_mlp *m, const splash_mlp_params *p, bool to_master, cudaStream_t s)
{
    struct L {
        float *W, *b;
        float *aug;
        int out, in, ld;
    } ls[3] = {{p->W1, p->b1, m->P1.as<float>(), kHid, kIn, kK1},
               {p->W2, p->b2, m->P2.as<float>(), kHid, kHid, kK2},
               {p->W3, p->b3, m->P3.as<float>(), kOut, kHid, kK2}};
    for (auto &l : ls) {
        const size_t f = sizeof(float);
        if (to_master) {
            SPLASH_CUDA_TRY(cudaMemcpy2DAsync(l.aug, l.ld * f, l.W, l.in * f, l.in * f, l.out, cudaMemcpyDeviceToDevice, s));
            SPLASH_CUDA_TRY(cudaMemcpy2DAsync(l.aug + l.in, l.ld * f, l.b, f, f, l.out, cudaMemcpyDeviceToDevice, s));
        } else {
            SPLASH_CUDA_TRY(cudaMemcpy2DAsync(l.W, l.in * f, l.aug, l.ld * f, l.in * f, l.out, cudaMemcpyDeviceToDevice, s));
            SPLASH_CUDA_TRY(cudaMemcpy2DAsync(l.b, f, l.aug + l.in, l.ld * f, f, l.out, cudaMemcpyDeviceToDevice, s));
        }
    }
    return SPLASH_OK;
}

splash_status copy_grads(splash_mlp *m, const splash_mlp_params *p, cudaStream_t s)
{
    struct L {
        float *W, *b;
        const float *g;
        int out, in, ld;
    } ls[3] = {{p->W1, p->b1, m->G1.as<float>(), kHid, kIn, kK1},
               {p->W2, p->b2, m->G2.as<float>(), kHid, kHid, kK2},
               {p->W3, p->b3, m->G3.as<float>(), kOut, kHid, kK2}};
    for (auto &l : ls) {
        const size_t f = sizeof(float);
        if (l.W) SPLASH_CUDA_TRY(cudaMemcpy2DAsync(l.W, l.in * f, l.g, l.ld * f, l.in * f, l.out, cudaMemcpyDeviceToDevice, s));
        if (l.b) SPLASH_CUDA_TRY(cudaMemcpy2DAsync(l.b, f, l.g + l.in, l.ld * f, f, l.out, cudaMemcpyDeviceToDevice, s));
    }
    return SPLASH_OK;
}
}  // namespace

extern "C" splash_status splash_mlp_create(splash_ctx *ctx, int32_t max_batch, splash_mlp **out)
{
    if (!ctx || !out) return fail(SPLASH_ERR_INVALID_ARG, "null context or output");
    if (max_batch <= 0 || max_batch > 65536) return fail(SPLASH_ERR_INVALID_ARG, "max_batch must be in 1..65536");
    if (!encoder()) return fail(SPLASH_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    splash_mlp *m = new splash_mlp;
    m->ctx = ctx;
    const int Bp = (max_batch + 127) / 128 * 128;
    m->Bp = Bp;
    const size_t f = sizeof(float), h = 2;
    struct {
        splash_host::Buf *b;
        size_t bytes;
    } all[] = {{&m->P1, (size_t)kHid * kK1 * f},  {&m->P2, (size_t)kHid * kK2 * f},  {&m->P3, (size_t)kOutPad * kK2 * f},
               {&m->M1, (size_t)kHid * kK1 * f},  {&m->M2, (size_t)kHid * kK2 * f},  {&m->M3, (size_t)kOutPad * kK2 * f},
               {&m->V1, (size_t)kHid * kK1 * f},  {&m->V2, (size_t)kHid * kK2 * f},  {&m->V3, (size_t)kOutPad * kK2 * f},
               {&m->G1, (size_t)kHid * kK1 * f},  {&m->G2, (size_t)kHid * kK2 * f},  {&m->G3, (size_t)kHid * kK2 * f},
               {&m->W1, (size_t)kHid * kK1 * h},  {&m->W2, (size_t)kHid * kK2 * h},  {&m->W2t, (size_t)kK2 * kHid * h},
               {&m->W3, (size_t)kOutPad * kK2 * h}, {&m->W3t, (size_t)kK2 * kDyPad * h},
               {&m->X, (size_t)Bp * kK1 * h},     {&m->Xt, (size_t)kK1 * Bp * h},    {&m->H1, (size_t)Bp * kK2 * h},
               {&m->H1t, (size_t)kK2 * Bp * h},   {&m->H2, (size_t)Bp * kK2 * h},    {&m->H2t, (size_t)kK2 * Bp * h},
               {&m->Y, (size_t)Bp * kOutPad * f}, {&m->dY, (size_t)Bp * kDyPad * h}, {&m->dYt, (size_t)kHid * Bp * h},
               {&m->dZ2, (size_t)Bp * kHid * h},  {&m->dZ2t, (size_t)kHid * Bp * h}, {&m->dZ1t, (size_t)kHid * Bp * h},
               {&m->T, (size_t)Bp * kOut * f},    {&m->loss, 16}};
    for (auto &a : all) {
        if (!a.b->ensure(a.bytes)) {
            delete m;
            return fail(SPLASH_ERR_OOM, "cudaMalloc failed for the MLP buffers");
        }
        if (cudaMemset(a.b->p, 0, a.b->cap) != cudaSuccess) {
            delete m;
            return fail(SPLASH_ERR_CUDA, "cudaMemset failed for the MLP buffers");
        }
    }
    // the constant-1 bias inputs: column 128 of H1, H2 and row 128 of their transposes
    {
        std::vector<uint16_t> ones((size_t)Bp, 0x3F80);
        bool ok = true;
        for (splash_host::Buf *b : {&m->H1, &m->H2})
            ok &= cudaMemcpy2D(b->as<uint16_t>() + kHid, kK2 * h, ones.data(), h, h, Bp, cudaMemcpyHostToDevice) == cudaSuccess;
        for (splash_host::Buf *b : {&m->H1t, &m->H2t})
            ok &= cudaMemcpy(b->as<uint16_t>() + (size_t)kHid * Bp, ones.data(), Bp * h, cudaMemcpyHostToDevice) == cudaSuccess;
        if (!ok) {
            delete m;
            return fail(SPLASH_ERR_CUDA, "cannot write the bias inputs");
        }
    }
    uint32_t *st = ctx->d_status;
    bool ok = true;
    // forward
    ok &= setup_gemm(m->f1, m->X.p, kK1, m->W1.p, kK1, Bp, kHid, kK1, st, kMlpSpin);
    ok &= setup_gemm(m->f2, m->H1.p, kK2, m->W2.p, kK2, Bp, kHid, kK2, st, kMlpSpin);
    ok &= setup_gemm(m->f3, m->H2.p, kK2, m->W3.p, kK2, Bp, kOutPad, kK2, st, kMlpSpin);
    // backward
    ok &= setup_gemm(m->b1, m->dYt.p, Bp, m->H2t.p, Bp, kHid, kK2, Bp, st, kMlpSpin);   // dW3 (rows 0..8 used)
    ok &= setup_gemm(m->b2, m->dY.p, kDyPad, m->W3t.p, kDyPad, Bp, kHid, kDyPad, st, kMlpSpin);  // dH2
    ok &= setup_gemm(m->b3, m->dZ2t.p, Bp, m->H1t.p, Bp, kHid, kK2, Bp, st, kMlpSpin);  // dW2
    ok &= setup_gemm(m->b4, m->dZ2.p, kHid, m->W2t.p, kHid, Bp, kHid, kHid, st, kMlpSpin);  // dH1
    ok &= setup_gemm(m->b5, m->dZ1t.p, Bp, m->Xt.p, Bp, kHid, kK1, Bp, st, kMlpSpin);   // dW1
    if (!ok) {
        delete m;
        return fail(SPLASH_ERR_CUDA, "tensor map encoding failed");
    }
    auto relu = [](Gemm &g, void *out, int64_t ld_out, void *out_t, int64_t ld_t) {
        g.args.epi = kEpiReluBf16;
        g.args.out = (__nv_bfloat16 *)out;
        g.args.ld_out = ld_out;
        g.args.out_t = (__nv_bfloat16 *)out_t;
        g.args.ld_t = ld_t;
    };
    auto f32 = [](Gemm &g, void *d, int64_t ldd) {
        g.args.epi = kEpiF32;
        g.args.d = (float *)d;
        g.args.ldd = ldd;
    };
    auto drelu = [](Gemm &g, const void *ref, int64_t ld_ref, void *out, int64_t ld_out, void *out_t, int64_t ld_t) {
        g.args.epi = kEpiDReluBf16;
        g.args.ref = (const __nv_bfloat16 *)ref;
        g.args.ld_ref = ld_ref;
        g.args.out = (__nv_bfloat16 *)out;
        g.args.ld_out = ld_out;
        g.args.out_t = (__nv_bfloat16 *)out_t;
        g.args.ld_t = ld_t;
    };
    relu(m->f1, m->H1.p, kK2, m->H1t.p, Bp);
    relu(m->f2, m->H2.p, kK2, m->H2t.p, Bp);
    f32(m->f3, m->Y.p, kOutPad);
    f32(m->b1, m->G3.p, kK2);
    drelu(m->b2, m->H2.p, kK2, m->dZ2.p, kHid, m->dZ2t.p, Bp);
    f32(m->b3, m->G2.p, kK2);
    drelu(m->b4, m->H1.p, kK2, nullptr, 0, m->dZ1t.p, Bp);
    f32(m->b5, m->G1.p, kK1);
    *out = m;
    return SPLASH_OK;
}

extern "C" splash_status splash_mlp_destroy(splash_mlp *m)
{
    if (!m) return fail(SPLASH_ERR_INVALID_ARG, "null mlp");
    delete m;
    return SPLASH_OK;
}

static bool params_ok(const splash_mlp_params *p)
{
    return p && p->W1 && p->b1 && p->W2 && p->b2 && p->W3 && p->b3;
}

extern "C" splash_status splash_mlp_set_params(splash_mlp *m, const splash_mlp_params *p, void *stream)
{
    if (!m || !params_ok(p)) return fail(SPLASH_ERR_INVALID_ARG, "null mlp or parameter buffer");
    cudaStream_t s = (cudaStream_t)stream;
    splash_status st = copy_params(m, p, true, s);
    if (st != SPLASH_OK) return st;
    for (splash_host::Buf *b : {&m->M1, &m->M2, &m->M3, &m->V1, &m->V2, &m->V3})
        SPLASH_CUDA_TRY(cudaMemsetAsync(b->p, 0, b->cap, s));
    m->step = 0;
    return mlp_adam_cast(m, nullptr, s);
}

extern "C" splash_status splash_mlp_get_params(splash_mlp *m, splash_mlp_params *p, void *stream)
{
    if (!m || !params_ok(p)) return fail(SPLASH_ERR_INVALID_ARG, "null mlp or parameter buffer");
    return copy_params(m, p, false, (cudaStream_t)stream);
}

extern "C" splash_status splash_mlp_predict(splash_mlp *m, const uint16_t *rows, int32_t batch, float *pred, void *stream)
{
    if (!m || !rows || !pred) return fail(SPLASH_ERR_INVALID_ARG, "null mlp, rows or output");
    if (batch <= 0 || batch > m->Bp) return fail(SPLASH_ERR_INVALID_ARG, "batch must be in 1..max_batch");
    if (!al16(rows)) return fail(SPLASH_ERR_INVALID_ARG, "rows must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    splash_status st;
    if ((st = mlp_gather(m, rows, batch, nullptr, nullptr, batch, s)) != SPLASH_OK) return st;
    if ((st = mlp_forward(m, s)) != SPLASH_OK) return st;
    k_mlp_head<<<1, 256, 0, s>>>(m->Y.as<float>(), nullptr, batch, m->Bp, pred, nullptr, nullptr, nullptr);
    count_launch();
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}

extern "C" splash_status splash_mlp_step(splash_mlp *m, const uint16_t *bank, int64_t n_rows, const int32_t *idx,
                                         const float *targets, int32_t batch, const splash_mlp_adam *adam, float *loss, splash_mlp_params *grads,
                                         void *stream)
{
    if (!m || !bank || !targets) return fail(SPLASH_ERR_INVALID_ARG, "null mlp, feature bank or targets");
    if (batch <= 0 || batch > m->Bp) return fail(SPLASH_ERR_INVALID_ARG, "batch must be in 1..max_batch");
    if (n_rows <= 0 || (!idx && n_rows < batch)) return fail(SPLASH_ERR_INVALID_ARG, "the feature bank is too small");
    if (!al16(bank)) return fail(SPLASH_ERR_INVALID_ARG, "the feature bank must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    splash_status st;
    if ((st = mlp_gather(m, bank, n_rows, idx, targets, batch, s)) != SPLASH_OK) return st;
    if ((st = mlp_forward(m, s)) != SPLASH_OK) return st;
    k_mlp_head<<<1, 256, 0, s>>>(m->Y.as<float>(), m->T.as<float>(), batch, m->Bp, nullptr, bf<__nv_bfloat16>(m->dY),
                                 bf<__nv_bfloat16>(m->dYt), m->loss.as<float>());
    count_launch();
    SPLASH_CUDA_TRY(cudaGetLastError());
    for (Gemm *g : {&m->b1, &m->b2, &m->b3, &m->b4, &m->b5})
        if ((st = launch_gemm(*g, s)) != SPLASH_OK) return st;
    if (loss) SPLASH_CUDA_TRY(cudaMemcpyAsync(loss, m->loss.p, sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (grads && (st = copy_grads(m, grads, s)) != SPLASH_OK) return st;
    if (adam) {
        m->step++;
        if ((st = mlp_adam_cast(m, adam, s)) != SPLASH_OK) return st;
    }
    return SPLASH_OK;
}
