// Internal declarations of libsplash: constants of the rasterizer, the
// kernel-side camera, the projected-Gaussian record, the workspace state
// and the launch wrappers each .cu file provides.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>

#include "splash.h"

namespace splash {

// ---- rasterizer constants (3DGS conventions the paper inherits, Sec. III-A)
constexpr float kAlphaMax = 0.99f;           // alpha clamp
constexpr float kAlphaMin = 1.0f / 255.0f;   // a Gaussian below this at a pixel is skipped
constexpr float kTStop = 1e-4f;              // stop before T would fall below this
constexpr float kDilate = 0.3f;              // 2D covariance dilation (px^2)
constexpr float kJClamp = 1.3f;              // projection Jacobian clamp, x half-FOV tangent
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
// q <= 9 (3 sigma) expressed on the scaled form qs = -log2(e)/2 * q
constexpr float kQsMin = -4.5f * kLog2e;
constexpr float kLog2AlphaMin = -7.99435329f;  // log2(1/255), rounded to FP32

// ---- camera as the kernels see it
struct CamK {
    float R[9];      // world -> camera rotation, row-major
    float t[3];      // world -> camera translation
    float cpos[3];   // camera centre in world coordinates
    float fx, fy, cx, cy;
    float limx, limy;  // clamp of t_x/t_z, t_y/t_z inside the Jacobian
    float znear, zfar;
    int W, H;
};

struct TileGeom {
    int tw, th;      // tile size in pixels
    int tx, ty;      // tiles across, down
};

// ---- projected Gaussian (48 B, three float4):
// r0 = {x_hi, y_hi, x_lo, y_lo}, r1 = {A, B, C, lo}, r2 = {d, ct_r, ct_g, ct_b}
//  centre x = x_hi + x_lo (doubled precision; the blend forms tile-local
//  coordinates (x_hi - tile_x0) + x_lo once per tile)
//  qs(dx, dy) = A dx^2 + B dx dy + C dy^2 = -log2(e)/2 * (d^T Sigma2^-1 d)
//  alpha = min(0.99, 2^(qs + lo)), lo = log2(sigmoid(o))
//  ct = c e^{-beta_D d} - B_inf e^{-beta_B d} (per-Gaussian effective colour)
struct __align__(16) Rec {
    float4 r0, r1, r2;
};

// per-Gaussian accumulators of the blend backward (three float4):
// a0 = {g_x, g_y, g_A, g_B}, a1 = {g_C, g_lo, g_d, 0}, a2 = {g_ct_r, g_ct_g, g_ct_b, 0}
struct __align__(16) GAcc {
    float4 a0, a1, a2;
};

// ---- one Adam step (Kingma & Ba), shared by the standalone and the fused kernels
struct AdamHyper {
    float b1, b2, eps;
    float rbc1, rsbc2;  // 1 / (1 - b1^step), 1 / sqrt(1 - b2^step): the bias corrections
};
inline AdamHyper make_adam_hyper(float b1, float b2, float eps, int step)
{
    AdamHyper h;
    h.b1 = b1;
    h.b2 = b2;
    h.eps = eps;
    double p1 = 1.0, p2 = 1.0;
    for (int k = 0; k < step; k++) {
        p1 *= b1;
        p2 *= b2;
    }
    h.rbc1 = (float)(1.0 / (1.0 - p1));
    h.rsbc2 = (float)(1.0 / sqrt(1.0 - p2));
    return h;
}
// p -= lr * m_hat / (sqrt(v_hat) + eps) with m_hat = m / bc1, sqrt(v_hat) = sqrt(v) / sqrt(bc2)
__device__ __forceinline__ void adam_update(float &p, float g, float &m, float &v, float lr, const AdamHyper &h)
{
    m = fmaf(h.b1, m, (1.f - h.b1) * g);
    v = fmaf(h.b2, v, (1.f - h.b2) * g * g);
    p -= __fdividef(lr * h.rbc1 * m, fmaf(sqrtf(v), h.rsbc2, h.eps));
}

// Everything the blend of one view needs (forward state, outputs, and for the
// backward the upstream gradients and accumulators). Plain launches take one
// by value; the persistent launches read an array of them.
struct BlendView {
    CamK cam;
    TileGeom tg;
    const uint2 *ranges;
    const uint32_t *gauss_ids;
    const Rec *rec;
    float *image, *depth, *depth01;       // outputs (depth, depth01 may be null)
    float *final_T, *acc_alpha, *zhat;    // per-pixel forward state
    uint32_t *n_last, *n_walk;
    const float *dL_dimage, *dL_ddepth, *dL_ddepth01;  // backward inputs (last two may be null)
    GAcc *gacc;                           // backward: per-Gaussian accumulators
    float *tile_medium;                   // backward: per-tile medium partials [tiles][6]
    GAcc *clear;                          // forward (plain launch): zero clear[0..clear_n) for the next backward
    int64_t clear_n;
    uint32_t *tile_walk;                  // forward (may be null): per tile, the largest walk bound n_last of its pixels
    const uint32_t *tile_order;           // backward plain launch (may be null): CTA b blends tile tile_order[b]
};

// device status word bits
enum : uint32_t { kStatusTimeout = 1u, kStatusCapacity = 2u, kStatusIndex = 4u };

// ---- two FP32 lanes in one 64-bit register pair (packed f32x2 arithmetic,
// sm_100 and later): one issue slot yields two IEEE round-to-nearest results,
// each bit-identical to the scalar operation on its lane (no flush to zero,
// like the rest of the library). The FP32 pipe's rate is unchanged; what is
// saved is issue slots, which is what bounds the windowed and blending loops.
struct F2 {
    uint64_t r;
};
__device__ __forceinline__ F2 f2(float x, float y)
{
    F2 v;
    asm("mov.b64 %0, {%1, %2};" : "=l"(v.r) : "f"(x), "f"(y));
    return v;
}
__device__ __forceinline__ void f2_split(F2 v, float &x, float &y) { asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v.r)); }
__device__ __forceinline__ F2 f2_fma(F2 a, F2 b, F2 c)
{
    F2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.r) : "l"(a.r), "l"(b.r), "l"(c.r));
    return d;
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b)
{
    F2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b)
{
    F2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}

// ---- onesweep radix sort (sort.cu)
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;                         // keys per thread (pair sorts)
constexpr int kSortTile = kSortThreads * kSortItems;   // keys per partition, the smallest used
#ifndef SPLASH_DEPTH_SORT_ITEMS
#define SPLASH_DEPTH_SORT_ITEMS 20
#endif
// keys per thread of the depth sort (keys only, one CTA wave at the bench's
// sizes: wider partitions spread the per-partition cost over more keys)
constexpr int kDepthSortItems = SPLASH_DEPTH_SORT_ITEMS;
static_assert(kDepthSortItems >= kSortItems, "the scratch is sized for kSortTile partitions");
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kRadixBitsMax = 9;                 // widest digit (a sort that saves a pass with it)
constexpr int kRadixMax = 1 << kRadixBitsMax;
constexpr int kLookbackPerPart = 3 * kRadixMax;  // the largest sum over a plan's passes of max(256, 2^width)

// Digits of a sort on `bits` key bits: 8-bit passes (the last one narrower),
// unless 9-bit digits need fewer passes (then the bits are spread evenly, at
// most 9 per pass).
struct DigitPlan {
    int passes;
    int width[4];
    int shift[4];
};
DigitPlan digit_plan(int bits);
// Significant bits of the depth keys of a camera: a key is the FP32 depth's
// bits minus those of z_near (depths lie in (z_near, z_far]; positive floats
// order like their bit patterns), so the keys span bits(z_far) - bits(z_near).
int depth_key_bits(float z_near, float z_far);

struct SortScratch {
    uint32_t *hist;      // [4][kRadixMax] per-pass digit offsets
    uint32_t *lookback;  // per pass [max_parts][max(256, 2^width)], kLookbackPerPart words per partition
    uint32_t *counters;  // [4] partition tickets
    int64_t max_parts;
};
size_t sort_scratch_bytes(int64_t n_max);
// opts the wide (depth) sort kernels in to their shared memory on the
// current device; once per device before the first depth sort
cudaError_t sort_prepare_device();
void sort_scratch_carve(void *base, int64_t n_max, SortScratch *s);
// Sorts n pairs (n read from n_dev when non-null, else n_host) on bits
// [0, bits). Ping-pongs between (k0,v0) and (k1,v1); returns which buffer
// pair holds the result (0 or 1). grid is sized from n_host, which must be
// >= the device count. items: keys per thread, kSortItems or kDepthSortItems.
int sort_pairs(const uint32_t *keys_in, const uint32_t *vals_in, uint32_t *k0, uint32_t *v0, uint32_t *k1,
               uint32_t *v1, int64_t n_host, const uint32_t *n_dev, int bits, const SortScratch &s,
               uint32_t *status, int spin_limit, int stall_part, cudaStream_t stream, int items = kSortItems);

// ---- kernels by stage (launch wrappers)
void launch_preprocess_fwd(int64_t n, const splash_gaussians &g, const float *medium, const CamK &cam,
                           const TileGeom &tg, Rec *rec, uint32_t *depth_key, uint32_t *tiles_touched,
                           uint2 *rect, cudaStream_t s);
void launch_count_scan(int64_t n, const uint32_t *order, const uint32_t *tiles_touched, uint32_t *offsets,
                       uint32_t *block_sums, uint32_t *total, cudaStream_t s);
// d_medium[j] = sum over nblocks rows of partials[b][9] (the pixel form's medium gradient)
void launch_pixel_medium_final(const float *partials, int nblocks, float *d_medium, cudaStream_t s);
// scratch of the pair-count sum (binning.cu): kPairTotalBlocksMax 16-byte
// partials and a ticket word, zero before the first launch (each launch
// leaves it zero)
constexpr int kPairTotalBlocksMax = 148 * 4;
constexpr size_t kPairTotalScratchBytes = 16 * (size_t)(kPairTotalBlocksMax + 1);
// ---- two-level tile binning (binning.cu)
constexpr int kSuperW = 8, kSuperH = 4;  // tiles per super-tile
// super-tiles per row (*nsx) and the bits of a super-tile index
int super_bits(const TileGeom &tg, int *nsx);
// chunks of the super-tile lists (an upper bound from the entry count)
int64_t chunk_bound(int64_t n_super_entries, int nsuper);
// K, K_s and the status word into host_out[0..2] (mapped host memory, device
// address; null: none); sc[g] = Gaussian g's super-tile count
void launch_pair_totals(int64_t n, const uint32_t *tt, const uint2 *rect, uint32_t *sc, void *scratch,
                        uint64_t *host_out, const uint32_t *status, cudaStream_t s);
// blocks of depth-ordered Gaussians the emit takes per CTA (block_pre holds
// emit_blocks(n) + 1 words)
int64_t emit_blocks(int64_t n);
// scs[r] = sc[order[r]]; block_pre[b] = exclusive offset of emit block b;
// *total = K_s
void launch_super_scan(int64_t n, const uint32_t *order, const uint32_t *sc, uint32_t *scs, uint32_t *block_pre,
                       uint32_t *total, cudaStream_t s);
void launch_emit_super(int64_t n, const uint32_t *order, const uint32_t *scs, const uint32_t *block_pre,
                       const uint2 *rect, int nsx, int sbits, uint32_t *keys, uint32_t *vals, uint64_t capacity,
                       uint32_t *status, cudaStream_t s);
struct BinningScratch {
    uint32_t *chunk_base;   // [nsuper + 1]
    uint32_t *chunk_count;  // [chunk_bound][32]
    uint32_t *tile_count;   // [tiles]
};
// the tile lists (gauss_ids) and their ranges from the sorted super-tile
// lists; n_super_entries bounds the entries (their count is read on the
// device); the ranges are clamped to `cap` slots of gauss_ids (a longer total
// is reported); *total (optional, device) = the pair count. sranges holds the
// super-tile list ranges, or, with digit_off (the exclusive digit offsets of
// a one-pass super-tile sort), is filled from them, the last list ending at
// *n_sorted_dev (or n_super_entries when that is null)
size_t binning_scratch_words(int64_t n_super_entries, int nsuper, int ntiles);
void launch_tile_lists(const TileGeom &tg, int nsx, int sbits, int64_t n_super_entries, const uint32_t *skeys,
                       const uint32_t *svals, uint2 *sranges, const BinningScratch &bs, uint2 *ranges,
                       uint32_t *gauss_ids, uint32_t *status, cudaStream_t s, uint32_t cap, uint32_t *total = nullptr,
                       const uint32_t *digit_off = nullptr, const uint32_t *n_sorted_dev = nullptr);
BinningScratch binning_scratch_carve(uint32_t *base, int64_t n_super_entries, int nsuper);
// tile_ids[i] = t for every i in ranges[t] (the sorted tile ids, rebuilt from the ranges)
void launch_expand_tile_ids(const uint2 *ranges, int ntiles, uint32_t *tile_ids, cudaStream_t s);

// ranges[t] = [first, end) of tile t's run in the sorted tile ids, for every
// tile (empty ones as [s, s)); nothing needs clearing first
void launch_ranges(int64_t k_host, const uint32_t *k_dev, const uint32_t *tile_ids, uint2 *ranges, int ntiles,
                   cudaStream_t s, uint32_t key_mask = 0xffffffffu);
// staging batch sizes the blend kernels are built for
constexpr int kBlendBatches[3] = {64, 128, 256};
void launch_blend_fwd(const BlendView &v, const float *medium, int batch, cudaStream_t s);
void launch_blend_bwd(const BlendView &v, const float *medium, int batch, cudaStream_t s);
// tiles ordered by descending walk bound (a counting sort in one CTA), so that
// the backward starts its longest tiles first
void launch_tile_order(const uint32_t *tile_walk, int ntiles, uint32_t *order, cudaStream_t s);
// Persistent forms: `ctas` CTAs pull work items from a queue (items[k] =
// view << 24 | tile, taken in order; *counter must be zero on entry) until
// n_items (read from the device) are done. All views share one tile shape.
void launch_blend_fwd_persistent(int tw, int th, int batch, const BlendView *views, const uint32_t *items,
                                 const uint32_t *n_items, int *counter, const float *medium, int ctas, cudaStream_t s);
void launch_blend_bwd_persistent(int tw, int th, int batch, const BlendView *views, const uint32_t *items,
                                 const uint32_t *n_items, int *counter, const float *medium, int ctas, cudaStream_t s);
int blend_persistent_ctas(int tw, int th, int batch, bool backward);
void launch_preprocess_bwd(int64_t n, const splash_gaussians &g, const float *medium, const CamK &cam,
                           const GAcc *acc, const uint32_t *depth_key, const splash_grads &out,
                           float *block_medium, int *n_blocks_out, cudaStream_t s);
// scratch: kColsumParts * 15 floats
void launch_medium_reduce(const float *tile_medium, int ntiles, const float *block_medium, int nblocks,
                          float *d_medium, float *scratch, cudaStream_t s);
void launch_preprocess_bwd_adam(int64_t n, int sh_degree, const splash_param_buffers &p, const float *medium,
                                const CamK &cam, const GAcc *acc, const uint32_t *dk, const splash_adam_config &cfg,
                                float *block_medium, int *n_blocks_out, cudaStream_t s);
void launch_medium_adam(float *medium, float *grad, const splash_adam_config &cfg, cudaStream_t s);
// launch_medium_reduce followed by launch_medium_adam, in two launches
void launch_medium_reduce_adam(const float *tile_medium, int ntiles, const float *block_medium, int nblocks,
                               float *medium, float *d_medium, float *scratch, const splash_adam_config &cfg,
                               cudaStream_t s);
int preprocess_bwd_blocks(int64_t n);
int preprocess_bwd_multi_blocks(int64_t n);
void launch_preprocess_bwd_multi(int64_t n, int V, const splash_gaussians &g, const float *medium, const BlendView *views,
                                 const GAcc *gacc, const uint32_t *depth_keys, int64_t key_stride,
                                 const splash_grads &out, float *block_medium, cudaStream_t s);

// Deterministic column sums of a row-major [rows][cols] float table (cols <=
// 16), first stage: kColsumParts CTAs each write one row of partial sums to
// part[kColsumParts][cols].
constexpr int kColsumParts = 64;
void launch_colsum_partial(const float *data, int rows, int cols, float *part, cudaStream_t s);
// the partial rows of a 6-column and a 9-column table in one launch
void launch_colsum_pair_6_9(const float *a, int rows_a, float *part_a, const float *b, int rows_b, float *part_b,
                            cudaStream_t s);

void launch_ssim_loss(const float *img, const float *tgt, int C, int H, int W, float lam, float *loss,
                      float *grad, float *scratch, cudaStream_t s);
size_t ssim_scratch_floats(int C, int H, int W);

}  // namespace splash

namespace splash {
// every kernel launch site bumps this (reported by splash_kernel_launches)
void count_launch(int n = 1);

// Programmatic dependent launch. A kernel started with launch_pdl may be
// scheduled while the kernel before it in the stream is still finishing; it
// begins with pdl_enter(), which first lets the kernel after it start
// launching, then waits until the kernel before it has completed and its
// stores are visible. Nothing of the previous kernel's output is touched
// before that wait, so the stream order of the results is unchanged; what
// overlaps is the launch latency and the previous kernel's last wave.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... P, typename... A>
inline void launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A &&...args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<A &&>(args)...);  // errors surface at cudaGetLastError
}
}  // namespace splash

// ---- error plumbing shared by the host code
void splash_set_error(const std::string &msg);

#define SPLASH_CUDA_TRY(expr)                                                                  \
    do {                                                                                       \
        cudaError_t e__ = (expr);                                                              \
        if (e__ != cudaSuccess) {                                                              \
            splash_set_error(std::string(#expr) + ": " + cudaGetErrorString(e__));             \
            return SPLASH_ERR_CUDA;                                                            \
        }                                                                                      \
    } while (0)
