/*
 * splash.h -- C ABI of libsplash.so, a B300 (sm_103a) differentiable tile
 * rasterizer for 3D Gaussians with the Gaussian Splashing underwater
 * image-formation model folded into compositing (arXiv 2411.19588).
 *
 * Conventions shared by every entry point:
 *  - Pointers named *_dev / buffers of the rasterizer are DEVICE pointers
 *    (cudaMalloc'd or torch CUDA storage) on the current device; the caller
 *    owns them. Host structs (camera, options, gradient tables) are read
 *    during the call only.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Work is
 *    asynchronous on it unless stated otherwise.
 *  - Every call returns a splash_status; on failure splash_last_error()
 *    gives a message (thread-local). Errors found by kernels (a bounded
 *    device wait that gave up, a capacity overflow) are reported by the next
 *    call that synchronises with the stream, or by splash_sync_status().
 *  - Floats are IEEE binary32; layouts are C-contiguous (row-major).
 */
#ifndef SPLASH_H
#define SPLASH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPLASH_OK = 0,
    SPLASH_ERR_INVALID_ARG = 1, /* a null pointer, a bad size, degree or tile shape */
    SPLASH_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    SPLASH_ERR_OOM = 3,         /* device allocation failed */
    SPLASH_ERR_CAPACITY = 4,    /* more tile/Gaussian pairs than the workspace holds */
    SPLASH_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    SPLASH_ERR_STATE = 6        /* backward without a matching forward */
} splash_status;

typedef struct splash_ctx splash_ctx;     /* options + device status word */
typedef struct splash_state splash_state; /* per-render workspace and forward state */

/* Pinhole camera. Pixel (ix, iy) has its centre at (ix + 0.5, iy + 0.5);
 * world_to_cam is a row-major 3x4 [R | t] with OpenCV axes (x right, y down,
 * z forward). Gaussians with camera-frame z <= z_near or z > z_far are culled;
 * the water behind the last Gaussian ends at z_far. */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float world_to_cam[12];
    float z_near, z_far;
} splash_camera;

/* Gaussian parameters theta_i = (mu, Sigma, c, opacity) of Sec. III-A, as
 * device buffers: means [n,3]; log_scales [n,3] (Sigma = R S S^T R^T with
 * S = diag(exp(log_scales))); quats [n,4] as (w, x, y, z), normalised inside;
 * opacity_logits [n] (opacity = sigmoid); sh [n, (deg+1)^2, 3] real
 * spherical-harmonic colour coefficients, colour = sum + 0.5 clamped at 0.
 * n < 2^31; sh_degree in 0..3. */
typedef struct {
    const float *means;
    const float *log_scales;
    const float *quats;
    const float *opacity_logits;
    const float *sh;
    int64_t n;
    int32_t sh_degree;
} splash_gaussians;

/* Gradient outputs (device), same layouts as the parameters; medium is [9].
 * They are OVERWRITTEN (not accumulated). A null member is not written. */
typedef struct {
    float *means;
    float *log_scales;
    float *quats;
    float *opacity_logits;
    float *sh;
    float *medium;
} splash_grads;

typedef struct {
    int32_t tile_w, tile_h; /* pixel tile: 16x16 (default), 8x32 or 32x8 */
    int32_t spin_limit;     /* iterations before a device wait gives up; 0 = default (2^22) */
    int32_t test_stall_partition; /* testing aid, 0 = off: when p > 0, partition p of every
                                     sort pass never publishes its look-back entry, so the
                                     wait of partition p + 1 runs out and the call reports
                                     SPLASH_ERR_TIMEOUT (results are then invalid) */
    int32_t gaussian_batch;       /* Gaussians staged in shared memory per blend step:
                                     64, 128 or 256 for both passes; 0 (default) = 64
                                     forward, 128 backward */
} splash_options;

/* Context: options and a device status word. Allocates only the status
 * word, on the current device, which is the device of every call made with
 * the context (it also sets the depth sort's shared-memory size there).
 * opt may be NULL (defaults). */
splash_status splash_create(const splash_options *opt, splash_ctx **out);
splash_status splash_destroy(splash_ctx *ctx);

/* A state holds the workspace of one render (projected Gaussians, sorted
 * tile lists, per-pixel final transmittance) so that splash_render_backward
 * can follow splash_render_forward. Its device buffers grow on demand
 * (cudaMalloc) and are freed by splash_state_destroy. One state serves one
 * forward/backward pair at a time; use one state per in-flight render. */
splash_status splash_state_create(splash_ctx *ctx, splash_state **out);
splash_status splash_state_destroy(splash_state *st);

/* Forward render (Sec. III-A tiles and Eq. 1-2 compositing, water model of
 * Eq. 3-5, depth of Eq. 6 and its logistic map of Sec. IV-D).
 * medium_dev: device float[9] = beta_D[3], beta_B[3], B_inf[3] (1/m, 1/m, colour).
 * Per pixel, Gaussians whose 3-sigma ellipse holds the pixel centre are
 * composited front to back; Gaussian i adds c_i e^{-beta_D d_i} alpha_i T_i,
 * the water in front of it adds B_inf (e^{-beta_B d_{i-1}} - e^{-beta_B d_i}) T_i,
 * and the water behind the last one out to z_far adds
 * B_inf (e^{-beta_B d_last} - e^{-beta_B z_far}) T_final.
 * Outputs (device, caller-owned): image [3,H,W]; depth [H,W] metres
 * (z_far where nothing is hit); depth01 [H,W] = 2/(1+e^{-0.1 depth}) - 1.
 * depth and depth01 may be NULL. Synchronises `stream` once (to size the
 * sort by the number of tile/Gaussian pairs). */
splash_status splash_render_forward(splash_ctx *ctx, splash_state *st, const splash_gaussians *g,
                                    const float *medium_dev, const splash_camera *cam, float *image,
                                    float *depth, float *depth01, void *stream);

/* Backward of the last forward on `st` (same g, medium and camera, unchanged
 * in between). Upstream gradients (device): dL_dimage [3,H,W] (required),
 * dL_ddepth and dL_ddepth01 [H,W] (NULL = zero). Writes every non-null
 * member of `grads`. Forward transmittance is recomputed back to front from
 * the stored final T; no per-pixel lists are kept. */
splash_status splash_render_backward(splash_ctx *ctx, splash_state *st, const splash_gaussians *g,
                                     const float *medium_dev, const splash_camera *cam,
                                     const float *dL_dimage, const float *dL_ddepth,
                                     const float *dL_ddepth01, const splash_grads *grads, void *stream);

/* Training step, fused: the backward of the last forward on `st` followed
 * by one Adam step (Sec. IV-C: Adam over all Gaussian and medium
 * parameters) applied in place, without writing the parameter gradients to
 * memory. params: the device buffers the forward read (same layouts as
 * splash_gaussians; medium [9]); they are updated in place. adam->m and
 * adam->v: first and second moments, same layouts, updated in place.
 * lr_*: per-group learning rates; beta1, beta2, eps: Adam constants; step:
 * 1-based step count for the bias corrections; if clamp_medium is non-zero
 * the medium parameters are clamped at >= medium_min after the step.
 * Every Gaussian steps (a zero gradient still moves its moments), as in
 * dense Adam. grad_medium (device float[9], may be NULL) receives the medium
 * gradient. Upstream gradients as in splash_render_backward. With `prior`
 * non-NULL (device float[6] = beta_B_hat[3], B_inf_hat[3], e.g. the first six
 * floats of a splash_backscatter_result), the gradient of Eq. 9's
 * lambda_est L_best term, lambda_est sign(medium[3+j] - prior[j]) (sign(0) =
 * 0), is added to medium[3..8]'s gradient before the step (and to
 * grad_medium). */
typedef struct {
    float *means;
    float *log_scales;
    float *quats;
    float *opacity_logits;
    float *sh;
    float *medium;
} splash_param_buffers;
typedef struct {
    splash_param_buffers m;
    splash_param_buffers v;
    float lr_means, lr_log_scales, lr_quats, lr_opacity_logits, lr_sh, lr_medium;
    float beta1, beta2, eps;
    int32_t step;
    int32_t clamp_medium;
    float medium_min;
    const float *prior; /* device [6] or NULL: the L_best estimate */
    float lambda_est;   /* weight of L_best (Eq. 9; 0.1 in the paper) */
    float *densify_stats; /* device [n][2] or NULL: densification statistics, += */
} splash_adam_config;
splash_status splash_render_backward_adam(splash_ctx *ctx, splash_state *st, const splash_param_buffers *params,
                                          int64_t n, int32_t sh_degree, const splash_camera *cam,
                                          const float *dL_dimage, const float *dL_ddepth, const float *dL_ddepth01,
                                          const splash_adam_config *adam, float *grad_medium, void *stream);

/* Batched form: n_views fixed cameras (uneven resolutions allowed) of one
 * scene, rendered and differentiated as one unit. After one
 * splash_batch_calibrate (which renders each view once to size the per-view
 * pair buffers and synchronises), splash_batch_forward / _backward neither
 * allocate nor synchronise, so a caller may capture them in a CUDA graph.
 * Each view keeps its own preprocess, depth sort, binning and tile sort;
 * every (view, tile) of the batch then goes through ONE persistent blend
 * launch forward and ONE backward, taken longest tile list first. A view
 * whose pair count outgrows its calibrated capacity is truncated and
 * SPLASH_ERR_CAPACITY is reported by splash_sync_status (recalibrate).
 * Tile shape and staging batch come from the context's options. */
typedef struct splash_batch splash_batch;
splash_status splash_batch_create(splash_ctx *ctx, int32_t n_views, const splash_camera *cams, splash_batch **out);
splash_status splash_batch_destroy(splash_batch *b);
/* headroom: capacity = measured pairs * headroom + 1024 per view (>= 0.01; 1.25 is a good default). */
splash_status splash_batch_calibrate(splash_batch *b, const splash_gaussians *g, const float *medium_dev,
                                     float headroom, void *stream);
/* images: host array of n_views device pointers [3,H_v,W_v]; depths, depth01s: host arrays or NULL
 * (entries may be NULL). The Gaussians must match the calibration in n and SH degree. */
splash_status splash_batch_forward(splash_batch *b, const splash_gaussians *g, const float *medium_dev,
                                   float *const *images, float *const *depths, float *const *depth01s, void *stream);
/* dL_dimages: host array of n_views device pointers [3,H_v,W_v]. grads: the gradient of the sum of
 * the views' losses, OVERWRITTEN. */
splash_status splash_batch_backward(splash_batch *b, const splash_gaussians *g, const float *medium_dev,
                                    const float *const *dL_dimages, const splash_grads *grads, void *stream);
/* Per view: pairs emitted by the last forward and the calibrated capacity (synchronises). */
splash_status splash_batch_pair_counts(const splash_batch *b, int64_t *emitted, int64_t *capacity, void *stream);

/* Read-only views of the forward state, for tests and diagnostics. Device
 * pointers stay valid until the next forward on the state. */
typedef struct {
    int64_t n_keys;              /* number of (tile, Gaussian) pairs */
    int32_t tiles_x, tiles_y, tile_w, tile_h;
    int64_t n_gaussians;
    const uint32_t *tile_ids;    /* [n_keys] sorted tile index of each pair, or NULL when the
                                    forward kept only the lists and their ranges (the two-level
                                    binning): splash_state_copy(SPLASH_FIELD_TILE_IDS) rebuilds
                                    it from the ranges */
    const uint32_t *gauss_ids;   /* [n_keys] Gaussian index of each pair, tile by tile, each
                                    tile's list in depth order */
    const uint32_t *ranges;      /* [tiles][2] half-open [start, end) into the pairs; an empty
                                    tile's is [s, s), s the pairs of the tiles before it */
    const uint32_t *depth_keys;  /* [n] FP32 depth bits minus those of z_near, 0xffffffff when culled */
    const uint32_t *tiles_touched; /* [n] */
    const float *records;        /* [n][12] projected Gaussian: x_hi, y_hi, x_lo, y_lo (centre =
                                    hi + lo), A, B, C (conic scaled by -log2(e)/2, -log2(e),
                                    -log2(e)/2), log2(opacity), depth, ct_r, ct_g, ct_b with
                                    ct = c e^{-beta_D d} - B_inf e^{-beta_B d}; valid where
                                    depth_keys != 0xffffffff */
    const float *final_T;        /* [H*W] transmittance after the last contributor */
    const float *acc_alpha;      /* [H*W] sum of alpha T */
    const uint32_t *n_last;      /* [H*W] the backward's walk bound: list entries in front of the
                                    Gaussian that stopped the pixel (the whole list if none did);
                                    every contributor lies in front of it */
    const uint32_t *n_walk;      /* [H*W] list entries the pixel walked (its blend work) */
} splash_state_info;
splash_status splash_state_get_info(const splash_state *st, splash_state_info *out);

/* Copy one forward-state buffer (sizes as in splash_state_info) into `dst`
 * (device or pinned host memory), asynchronously on `stream`. `bytes` must
 * equal the buffer's size: n_keys*4 for TILE_IDS/GAUSS_IDS, tiles*8 for
 * RANGES, n*4 for DEPTH_KEYS/TILES_TOUCHED, n*48 for RECORDS, n*8 for RECTS,
 * H*W*4 for the per-pixel fields. TILE_IDS, when the forward kept only the
 * lists and ranges, is rebuilt from the ranges on `stream` first. */
typedef enum {
    SPLASH_FIELD_TILE_IDS = 0,
    SPLASH_FIELD_GAUSS_IDS = 1,
    SPLASH_FIELD_RANGES = 2,
    SPLASH_FIELD_DEPTH_KEYS = 3,
    SPLASH_FIELD_TILES_TOUCHED = 4,
    SPLASH_FIELD_RECORDS = 5,
    SPLASH_FIELD_FINAL_T = 6,
    SPLASH_FIELD_ACC_ALPHA = 7,
    SPLASH_FIELD_N_LAST = 8,
    SPLASH_FIELD_N_WALK = 9,
    SPLASH_FIELD_RECTS = 10 /* [n][2] uint32: tile columns tx0 | tx1 << 16, rows ty0 | ty1 << 16 */
} splash_field;
splash_status splash_state_copy(const splash_state *st, int32_t field, void *dst, int64_t bytes, void *stream);

/* Photometric loss of the training step: loss = mean|x - y| + lam (1 - mean SSIM)
 * (the Eq. 7 form; SSIM with an 11x11 Gaussian window, sigma 1.5, zero
 * padding, C1 = 0.01^2, C2 = 0.03^2). image, target: device [C,H,W].
 * loss_dev: device float[1] (written). dL_dimage: device [C,H,W] (written;
 * may be NULL for loss only). Uses workspace of `st`. */
splash_status splash_loss_l1_ssim(splash_ctx *ctx, splash_state *st, const float *image, const float *target,
                                  int32_t channels, int32_t height, int32_t width, float lam,
                                  float *loss_dev, float *dL_dimage, void *stream);

/* One Adam step (Sec. IV-C) over several parameter groups in one launch.
 * Each group: param, grad, m, v device float[n]; lr; optional lower clamp.
 * Bias correction uses `step` (>= 1). */
typedef struct {
    float *param;
    const float *grad;
    float *m;
    float *v;
    int64_t n;
    float lr;
    float clamp_min;
    int32_t has_clamp;
} splash_adam_group;
#define SPLASH_ADAM_MAX_GROUPS 8
splash_status splash_adam_step(const splash_adam_group *groups, int32_t n_groups, int32_t step, float beta1,
                               float beta2, float eps, void *stream);

/* Stable LSD radix sort of (uint32 key, uint32 value) pairs on key bits
 * [0, key_bits), onesweep form. keys/vals in (device, n) are left unchanged;
 * keys_out/vals_out (device, n) receive the result. vals_in NULL means
 * values 0..n-1. Uses workspace of `st`. */
splash_status splash_sort_pairs_u32(splash_ctx *ctx, splash_state *st, const uint32_t *keys_in,
                                    const uint32_t *vals_in, uint32_t *keys_out, uint32_t *vals_out,
                                    int64_t n, int32_t key_bits, void *stream);

/* Stage timing with CUDA events recorded on the caller's stream around each
 * stage of the calls that take a context (tracing aid; off by default).
 * splash_profile_enable clears the totals; splash_profile_read waits for the
 * recorded events and returns per-stage total milliseconds and launch counts
 * (arrays of SPLASH_STAGE_COUNT entries), then clears them. */
typedef enum {
    SPLASH_STAGE_PREPROCESS = 0,
    SPLASH_STAGE_DEPTH_SORT = 1,
    SPLASH_STAGE_SCAN = 2,
    SPLASH_STAGE_EMIT = 3,
    SPLASH_STAGE_TILE_SORT = 4,
    SPLASH_STAGE_RANGES = 5,
    SPLASH_STAGE_BLEND_FWD = 6,
    SPLASH_STAGE_BLEND_BWD = 7,
    SPLASH_STAGE_PREPROCESS_BWD = 8,
    SPLASH_STAGE_MEDIUM_REDUCE = 9,
    SPLASH_STAGE_LOSS = 10,
    SPLASH_STAGE_BACKSCATTER = 11, /* cluster, select, minima and fit of the backscatter estimate */
    SPLASH_STAGE_BS_RESIZE = 12,   /* the estimate's resize */
    SPLASH_STAGE_COUNT = 13
} splash_stage;
splash_status splash_profile_enable(splash_ctx *ctx, int32_t on);
splash_status splash_profile_read(splash_ctx *ctx, double *ms, int64_t *counts);
/* Restrict the timing to the stages whose bit (1 << splash_stage) is set in
 * stage_mask (all stages by default); each timed stage costs two event
 * records on the stream. */
splash_status splash_profile_mask(splash_ctx *ctx, uint32_t stage_mask);

/* ABI self-description (no counterpart in the paper; for bindings): the
 * compiler's layout of every struct declared here, so that a binding can
 * check its mirrors field by field. Structs in this order: splash_camera,
 * splash_gaussians, splash_grads, splash_options, splash_param_buffers,
 * splash_adam_config, splash_state_info, splash_adam_group,
 * splash_mlp_params, splash_mlp_adam, splash_densify_options,
 * splash_backscatter_options, splash_backscatter_result; within a struct
 * its fields in declaration order (an array or struct member counts once).
 * sizes[s] = sizeof, n_fields[s] = its field count, offsets = every field's
 * offsetof, struct after struct. Any output may be NULL (call once with
 * only n_structs and n_offsets to size the arrays). Host only; never fails. */
splash_status splash_abi_layout(int32_t *sizes, int32_t *n_fields, int32_t *offsets, int32_t *n_structs,
                                int32_t *n_offsets);

/* Number of kernels this library has launched in this process so far. */
uint64_t splash_kernel_launches(void);

/* The pair sort above for callers that cannot allocate device memory
 * (no counterpart in the paper; it exists for library users). Some callers
 * may not call cudaMalloc at all: code embedded in a host application whose
 * device memory is owned and budgeted by that application, or latency-bound
 * code that cannot take the synchronisation an allocation may imply. This
 * entry point allocates nothing: its scratch (ping-pong pair buffers, digit
 * histograms, look-back flags, a status word) is one static device array of
 * about 10 MB that every GPU loading this library holds until the process
 * exits. Same arguments and result as splash_sort_pairs_u32, without the
 * context and state: keys_in/vals_in (device, n; vals_in NULL = 0..n-1) are
 * left unchanged, keys_out/vals_out (device, n) receive the pairs sorted
 * stably on key bits [0, key_bits). n must be at most 1,048,576 (2^20);
 * larger n returns SPLASH_ERR_INVALID_ARG. keys_in must be 16-byte aligned.
 * status_out (device uint32, may be NULL) receives 0, or SPLASH_ERR_TIMEOUT's
 * kernel bit (1) if a bounded device-side wait gave up. All calls share the
 * one array (each call clears what must start at zero), so calls that
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller. The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress with that device current);
 * make that first call before any stream capture. The address is kept for
 * the life of the process: a cudaDeviceReset on a device (which unloads the
 * module and its array) ends this entry point's use on that device. */
splash_status splash_sort_pairs_u32_noalloc(const uint32_t *keys_in, const uint32_t *vals_in, uint32_t *keys_out,
                                            uint32_t *vals_out, int64_t n, int32_t key_bits, uint32_t *status_out,
                                            void *stream);

/* ---- Learned warm-start (Sec. IV-C fit initialisation) --------------------
 * The paper has no learned part. These calls predict the nine per-channel
 * medium parameters of Eq. 4-5 (beta_D[3], beta_B[3], B_inf[3]) from one
 * rendered view, so that the fit can start from them; the plain fit stays the
 * fallback and the judge of the prediction.
 *
 * Feature row of a view (splash_featurise): SPLASH_MLP_ROW BF16 values =
 * the 32x32 adaptive-average downsample of image [3,H,W] (channel-major,
 * cell (i,j) averages rows floor(iH/32)..ceil((i+1)H/32)-1 and the same in
 * x), then an 8-bin histogram of the Eq. 6 depth over [0, z_far] (bin =
 * floor(fl32(8 z) / z_far) clamped to 0..7, NaN in bin 7, divided by H W),
 * then 1 (the bias input), then zeros. All pointers are device pointers; the
 * row must be 16-byte aligned. The call uses an 8-counter scratch owned by
 * the context, so featurise calls sharing a context must be stream-ordered. */
#define SPLASH_MLP_IN 3080
#define SPLASH_MLP_ROW 3136
#define SPLASH_MLP_HIDDEN 128
#define SPLASH_MLP_OUT 9
splash_status splash_featurise(splash_ctx *ctx, const float *image, const float *depth, int32_t width, int32_t height,
                               float z_far, uint16_t *row, void *stream);

/* D[M,N] = A[M,K] . B[N,K]^T with BF16 A and B (row-major, leading dimensions
 * lda, ldb in elements) and FP32 D (ldd): the tensor-core GEMM the MLP runs
 * on (TMA-staged operands, tcgen05.mma with the accumulator in tensor
 * memory). Needs M % 128 == 0, N % 16 == 0, K % 64 == 0; lda, ldb >= K and
 * multiples of 8; ldd >= N and a multiple of 4; A, B, D 16-byte aligned.
 * Otherwise SPLASH_ERR_INVALID_ARG and nothing is launched. */
splash_status splash_gemm_bf16(splash_ctx *ctx, const uint16_t *A, int64_t lda, const uint16_t *B, int64_t ldb,
                               float *D, int64_t ldd, int32_t M, int32_t N, int32_t K, void *stream);

/* The MLP 3080 -> 128 -> 128 -> 9: ReLU hidden layers; heads softplus
 * (beta_D, beta_B) and sigmoid (B_inf); BF16 weights and activations, FP32
 * accumulation; loss = mean over batch and outputs of |log p - log target|.
 * The handle owns FP32 master weights, Adam moments, BF16 copies and every
 * activation buffer for batches up to max_batch (rounded up to 128). */
typedef struct splash_mlp splash_mlp;
typedef struct { /* device pointers, FP32, row-major */
    float *W1; /* [128, 3080] */
    float *b1; /* [128] */
    float *W2; /* [128, 128] */
    float *b2; /* [128] */
    float *W3; /* [9, 128] */
    float *b3; /* [9] */
} splash_mlp_params;
typedef struct {
    float lr, beta1, beta2, eps;
} splash_mlp_adam;
splash_status splash_mlp_create(splash_ctx *ctx, int32_t max_batch, splash_mlp **out);
splash_status splash_mlp_destroy(splash_mlp *mlp);
/* Load weights (and reset the Adam moments and step count). */
splash_status splash_mlp_set_params(splash_mlp *mlp, const splash_mlp_params *params, void *stream);
splash_status splash_mlp_get_params(splash_mlp *mlp, splash_mlp_params *params, void *stream);
/* pred[batch, 9] for `batch` consecutive feature rows. */
splash_status splash_mlp_predict(splash_mlp *mlp, const uint16_t *rows, int32_t batch, float *pred, void *stream);
/* One training step on rows bank[idx[b]] of a bank of n_rows feature rows
 * (idx null: the first `batch` rows) with targets[idx[b]] ([n_rows, 9]
 * FP32): forward, loss (written to *loss if non-null, device), backward, and
 * with `adam` non-null one Adam step on the masters followed by the BF16
 * refresh. `grads` (nullable) receives the gradients in the natural layout.
 * An index outside [0, n_rows) is clamped and reported by splash_sync_status
 * as SPLASH_ERR_INVALID_ARG. */
splash_status splash_mlp_step(splash_mlp *mlp, const uint16_t *bank, int64_t n_rows, const int32_t *idx,
                              const float *targets, int32_t batch, const splash_mlp_adam *adam, float *loss, splash_mlp_params *grads,
                              void *stream);

/* Densification (appendix: every 100 iterations from 1,500 to 15,000;
 * gradient threshold 0.0002, minimum opacity 0.1; the 3DGS procedure).
 * Statistics: with adam->densify_stats set, each fused training step adds,
 * for every Gaussian in the view, the NDC norm of its screen-space centre
 * gradient, |(g_x W/2, g_y H/2)|, and 1 (the count) to stats[i][0..1].
 * splash_densify_plan decides per Gaussian (FP32 decisions): prune if its
 * opacity logit < logit(min_opacity); otherwise, if stats[i][0] /
 * max(stats[i][1], 1) >= grad_threshold, split if its largest log-scale >
 * log(percent_dense * extent), else clone; otherwise keep. It synchronises
 * `stream` and returns the new count in *n_new (host). The plan is kept in
 * the context for the next splash_densify_apply with the same n, which
 * writes the new arrays (caller-allocated for n_new Gaussians; same layouts;
 * the medium members are ignored): survivors and a clone's original in
 * place of order with their Adam moments, a clone's copy right after it with
 * zero moments, a split Gaussian's two samples mu + R diag(exp(log_scales))
 * noise[i][k] (noise: device [n][2][3] standard normals) with log-scales
 * lowered by log(1.6) and zero moments. */
typedef struct {
    float grad_threshold; /* 0.0002 */
    float min_opacity;    /* 0.1 */
    float percent_dense;  /* 0.01 */
    float extent;         /* scene extent (m) */
} splash_densify_options;
splash_status splash_densify_plan(splash_ctx *ctx, const float *log_scales, const float *opacity_logits,
                                  const float *stats, int64_t n, const splash_densify_options *opt, int64_t *n_new,
                                  void *stream);
splash_status splash_densify_apply(splash_ctx *ctx, const splash_param_buffers *params, const splash_param_buffers *m,
                                   const splash_param_buffers *v, int64_t n, int32_t sh_degree, const float *noise,
                                   const splash_param_buffers *new_params, const splash_param_buffers *new_m,
                                   const splash_param_buffers *new_v, int64_t n_new, void *stream);

/* Opacity reset of the training schedule (appendix: every 3,000 iterations):
 * logits[i] = min(logits[i], logit(max_opacity)) for n opacity logits
 * (device), and the opacity group's Adam moments adam_m, adam_v (device,
 * nullable) set to zero. max_opacity in (0, 1); the paper's value is 0.01. */
/* MCMC densification, the form Sec. IV-D adopts (3DGS-MCMC's sampling in
 * place of clone / split / prune; Sec. VI ablates it against the 3DGS
 * procedure above). In place, the Gaussian count unchanged (to grow the set,
 * append Gaussians with opacity 0 and relocate: they are dead).
 *
 * splash_mcmc_relocate: a Gaussian is dead when sigmoid(o) <= min_opacity
 * (0.005), decided in FP64. Each dead Gaussian d draws a live source with
 * probability proportional to opacity: the first g with C_g > u_d C_total,
 * C the FP64 running sum of sigmoid(o) over live Gaussians in index order
 * and u_d = uniforms[d], which must lie in [0, 1) (device, n floats; only
 * dead entries are read). A source drawn c times stands for N =
 * min(c + 1, 51) Gaussians: it and its copies take opacity
 * o' = 1 - (1 - o)^(1/N) and scales s' = s o / Z, Z = sum_{i=1}^{N}
 * sum_{k=0}^{i-1} C(i-1,k) (-1)^k o'^(k+1) / sqrt(k+1); each dead Gaussian
 * then takes every parameter of its source, and the Adam moments (m, v:
 * same layouts as the parameters) of sources and copies are zeroed. All
 * buffers are device, caller-owned, read and written in place; quats 16-byte
 * aligned. n_dead (host, may be NULL) receives the dead count; non-NULL
 * synchronises the stream. Scratch: about 20 B per Gaussian, owned by the
 * context (grow-only); calls sharing a context must be stream-ordered.
 *
 * splash_mcmc_noise: mu += lambda_noise * lr * sigmoid(-100 (o - 0.005)) *
 * Sigma eta per Gaussian, Sigma = R diag(exp(2 log_scales)) R^T its
 * covariance, eta (device [n,3]) standard normals given by the caller
 * (lambda_noise 5e5 in the cited method, lr the position learning rate).
 * means written in place; quats 16-byte aligned. */
splash_status splash_mcmc_relocate(splash_ctx *ctx, const splash_param_buffers *params, const splash_param_buffers *m,
                                   const splash_param_buffers *v, int64_t n, int32_t sh_degree, const float *uniforms,
                                   float min_opacity, int64_t *n_dead, void *stream);
splash_status splash_mcmc_noise(float *means, const float *log_scales, const float *quats, const float *opacity_logits,
                                const float *eta, int64_t n, float lr, float lambda_noise, void *stream);

splash_status splash_opacity_reset(float *logits, float *adam_m, float *adam_v, int64_t n, float max_opacity,
                                   void *stream);

/* ---- The pixel form of the water (Eq. 5 as printed, with the Eq. 6 depth) ----
 * C = J exp(-beta_D z) + B_inf (1 - exp(-beta_B z)) per pixel and channel, with
 * J = sum_i c_i alpha_i T_i the plain composite and z the expected depth (z_far
 * where nothing composites); the default calls above instead attenuate every
 * Gaussian at its own depth and add the backscatter of every water segment.
 * splash_render_forward_pixel takes the same arguments as
 * splash_render_forward: it renders J and z (the render with a zero medium)
 * and applies Eq. 5; depth and depth01 are the same Eq. 6 outputs. The state
 * keeps J for the backward. splash_render_backward_pixel is its adjoint with
 * the arguments of splash_render_backward: dL/dJ = G exp(-beta_D z), dL/dz
 * gains sum_ch G (B_inf beta_B exp(-beta_B z) - beta_D J exp(-beta_D z)) where
 * something composites (it reaches every contributing Gaussian through
 * alpha and d), and grads->medium receives sum over pixels of G (-z J
 * exp(-beta_D z)), G B_inf z exp(-beta_B z) and G (1 - exp(-beta_B z)).
 * SPLASH_ERR_STATE if the state's last forward was not the pixel form. */
splash_status splash_render_forward_pixel(splash_ctx *ctx, splash_state *st, const splash_gaussians *g,
                                          const float *medium_dev, const splash_camera *cam, float *image, float *depth,
                                          float *depth01, void *stream);
splash_status splash_render_backward_pixel(splash_ctx *ctx, splash_state *st, const splash_gaussians *g,
                                           const float *medium_dev, const splash_camera *cam,
                                           const float *dL_dimage, const float *dL_ddepth,
                                           const float *dL_ddepth01, const splash_grads *grads, void *stream);
/* The fused training step of the pixel form: its adjoint followed by one Adam
 * step in place, with the arguments and conventions of
 * splash_render_backward_adam (prior and densification statistics
 * included). */
splash_status splash_render_backward_adam_pixel(splash_ctx *ctx, splash_state *st, const splash_param_buffers *params,
                                                int64_t n, int32_t sh_degree, const splash_camera *cam,
                                                const float *dL_dimage, const float *dL_ddepth,
                                                const float *dL_ddepth01, const splash_adam_config *adam,
                                                float *grad_medium, void *stream);

/* ---- Backscatter estimate and the L_best prior (Sec. IV-B, Eq. 7-9;
 * appendix Alg. 1 "Estimate Backscatter" and Alg. 2) -----------------------
 * splash_backscatter_estimate turns an observed image and the expected depth
 * of the current scene at the same view (Eq. 6) into per-channel estimates
 * beta_B_hat and B_inf_hat of the backscatter B_inf (1 - exp(-beta_B z)):
 *  1. image and depth are area-averaged to resized_height rows and
 *     w = floor((2 W rh + H) / (2 H)) columns (at least 1): output row o
 *     covers source rows [o H / rh, (o+1) H / rh), each weighted by its
 *     overlap length (columns alike); the exact weighted mean (FP64
 *     accumulation) is rounded once to FP32 and negative values become 0;
 *  2. edges e_i = zmin + ((zmax - zmin) i) / (edges - 1) (FP64) over the
 *     resized depth; a pixel's cluster is the largest i <= edges - 2 with
 *     z >= e_i; of a cluster of n pixels the ceil(p_dark n) darkest are kept,
 *     ranked by fl32(fl32(R + G) + B) with ties to the smaller row-major
 *     index;
 *  3. over the kept pixels' depths, bounds f_i = lo + ((hi - lo) i) /
 *     (intervals - 1); per channel and per non-empty interval (the largest
 *     i <= intervals - 2 with z >= f_i) the kept pixel with the smallest
 *     value (ties: smaller index) gives one point (its depth, its value);
 *  4. per channel, min sum_j (m_j - B (1 - exp(-beta z_j)))^2 over
 *     B in [0, b_max], beta in [0, beta_max]: an FP32 scan of 1024 betas
 *     brackets the minimum, then the zero of the derivative of the profiled
 *     residual (B = the clipped linear least-squares value for each beta) is
 *     found in FP64.
 * image: device [3,H,W] FP32; depth: device [H,W] FP32; finite values.
 * opt: NULL = the paper's values (300, 10, 25, 0.01, 1, 5). result: device,
 * 16-byte aligned; its first six floats (beta_b, then b_inf) line up with
 * medium[3..8] and serve as the `prior` of the calls below. resized
 * (device, nullable) receives [4, h, w] FP32: the resized R, G, B and depth;
 * dark (device, nullable) receives [h w] bytes, 1 for kept pixels. The
 * scratch is owned by the context (grow-only), so estimates sharing a
 * context must be stream-ordered. SPLASH_ERR_INVALID_ARG for a null
 * pointer, a size below 1, a resized image above 2^24 pixels or options out
 * of range (edges and intervals in 2..65, p_dark in (0, 1], positive bounds,
 * resized_height in 1..4096). */
#define SPLASH_BS_MAX_POINTS 64
typedef struct {
    int32_t resized_height; /* rows after the resize (300) */
    int32_t edges;          /* depth edges of Alg. 2 (10, i.e. 9 clusters) */
    int32_t intervals;      /* interval bounds of Alg. 1 (25, i.e. 24 intervals) */
    int32_t pad;
    double p_dark;          /* fraction of each cluster kept (0.01) */
    float b_max, beta_max;  /* fit bounds (1 and 5 per metre) */
} splash_backscatter_options;
typedef struct {
    float beta_b[3];       /* beta_B_hat (1/m) */
    float b_inf[3];        /* B_inf_hat */
    float residual[3];     /* sum of squared residuals of each channel's fit */
    int32_t n_points[3];   /* fitted points per channel (0: nothing kept; then 0, 0) */
    int32_t n_dark;        /* kept pixels */
    int32_t width, height; /* resized size */
    int32_t pad;
    float point_z[3][SPLASH_BS_MAX_POINTS]; /* points in interval order */
    float point_v[3][SPLASH_BS_MAX_POINTS];
} splash_backscatter_result;
splash_status splash_backscatter_estimate(splash_ctx *ctx, const float *image, const float *depth, int32_t width,
                                          int32_t height, const splash_backscatter_options *opt,
                                          splash_backscatter_result *result, float *resized, uint8_t *dark,
                                          void *stream);
/* Eq. 9's prior term for the unfused backward: with medium (device [9]) and
 * prior (device [6] = beta_B_hat, B_inf_hat), adds lambda_est (|beta_B -
 * beta_B_hat|_1 + |B_inf - B_inf_hat|_1) to *loss (device, nullable) and
 * lambda_est sign(medium[3+j] - prior[j]) (sign(0) = 0) to grad_medium[3+j]
 * (device [9], nullable). */
splash_status splash_backscatter_prior(const float *medium, const float *prior, float lambda_est, float *grad_medium,
                                       float *loss, void *stream);

/* ---- Water removal (the application of Sec. I / Sec. V) -------------------
 * The clean render of a scene, its colour with the water taken away, is
 * splash_render_forward with a zero medium: Eq. 5 with beta_D = beta_B =
 * B_inf = 0 is the plain composite of Eq. 1. splash_restore removes the water
 * from an image instead, given a depth map (e.g. the Eq. 6 depth of the
 * reconstructed scene) and the medium: per pixel and channel,
 *   out = max(I - B_inf (1 - exp(-beta_B z)), 0) exp(beta_D z),
 * the inverse of Eq. 5 with the direct signal clipped at 0. image, out: device
 * [3,H,W] FP32 (out may equal image); depth: device [H,W]; medium: device
 * [9] (beta_D, beta_B, B_inf). Asynchronous on `stream`. */
splash_status splash_restore(const float *image, const float *depth, const float *medium, int32_t width,
                             int32_t height, float *out, void *stream);

/* Synchronise `stream` and report any error a kernel recorded since the last check. */
splash_status splash_sync_status(splash_ctx *ctx, void *stream);

/* Message for the last failing call on this thread ("" if none). */
const char *splash_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SPLASH_H */
