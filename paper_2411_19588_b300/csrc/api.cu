// C ABI of libsplash: contexts, render states (grow-only device
// workspaces), argument checks and the order of the stages.
//
// Forward (one stream, one host synchronisation to read the pair count):
//   preprocess -> depth sort (N pairs) -> scan of tile counts in depth order
//   -> [read back K] -> emit K (tile, Gaussian) pairs -> tile sort -> ranges
//   -> blend.
// Backward: blend adjoint -> preprocess adjoint -> medium reduction.
#include <cstddef>
#include <cstring>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <vector>

#include "host.h"

using namespace splash;
using namespace splash_host;

namespace {
thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};
}  // namespace

void splash_set_error(const std::string &msg) { g_last_error = msg; }

namespace splash {
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
}  // namespace splash

namespace {

BlendView backward_view(splash_state *st, const CamK &ck, const float *gi, const float *gd, const float *g01)
{
    BlendView v{};
    v.cam = ck;
    v.tg = st->tg;
    v.ranges = st->ranges.as<uint2>();
    v.gauss_ids = st->gauss_ids;
    v.rec = st->rec.as<Rec>();
    v.final_T = st->fT.as<float>();
    v.acc_alpha = st->aA.as<float>();
    v.zhat = st->zh.as<float>();
    v.n_last = st->nlast.as<uint32_t>();
    v.n_walk = st->nwalk.as<uint32_t>();
    v.dL_dimage = gi;
    v.dL_ddepth = gd;
    v.dL_ddepth01 = g01;
    v.gacc = st->gacc.as<GAcc>();
    v.tile_medium = st->tile_med.as<float>();
    v.tile_order = st->tile_order.as<uint32_t>();
    return v;
}

// The backward's per-Gaussian accumulators must be zero when its blend
// starts. Once this state holds them (a backward ran on it before), the
// forward blend clears them: each of its CTAs stores its share, which drains
// under that arithmetic-bound kernel instead of costing a memset pass. The
// backward clears them itself when the last forward did not.
void preclear_backward(splash_state *st, int64_t n, BlendView &v)
{
    st->gacc_cleared = n > 0 && st->gacc.cap >= sizeof(GAcc) * (size_t)n;
    if (!st->gacc_cleared) return;
    v.clear = st->gacc.as<GAcc>();
    v.clear_n = n;
    st->gacc_clear_ptr = st->gacc.p;
    st->gacc_clear_n = n;
}

splash_status clear_backward(splash_state *st, int64_t n, cudaStream_t s)
{
    const bool covered = st->gacc_cleared && st->gacc_clear_ptr == st->gacc.p && st->gacc_clear_n >= n;
    st->gacc_cleared = false;  // the blend below dirties them
    if (!covered && n > 0) SPLASH_CUDA_TRY(cudaMemsetAsync(st->gacc.p, 0, sizeof(GAcc) * (size_t)n, s));
    return SPLASH_OK;
}

// The two-level binning leaves no array of sorted tile ids (the blends use
// the ranges); a state query rebuilds it from the ranges, on stream s.
const uint32_t *rebuilt_tile_ids(const splash_state *st, cudaStream_t s)
{
    if (!st->tid_lazy_ok) {
        if (!st->tid_lazy.ensure(4 * (size_t)std::max<int64_t>(st->K, 1))) return nullptr;
        launch_expand_tile_ids(st->ranges.as<uint2>(), st->tg.tx * st->tg.ty, st->tid_lazy.as<uint32_t>(), s);
        st->tid_lazy_ok = true;
    }
    return st->tid_lazy.as<uint32_t>();
}

// the failure a non-zero device status word reports
splash_status status_failure(uint32_t status)
{
    if (status & kStatusTimeout) return fail(SPLASH_ERR_TIMEOUT, "a device-side wait gave up (spin limit reached)");
    if (status & kStatusCapacity) return fail(SPLASH_ERR_CAPACITY, "tile/Gaussian pairs exceeded the workspace");
    if (status & kStatusIndex) return fail(SPLASH_ERR_INVALID_ARG, "a row index was outside the feature bank");
    return SPLASH_OK;
}

}  // namespace

extern "C" {

const char *splash_last_error(void) { return g_last_error.c_str(); }

splash_status splash_create(const splash_options *opt, splash_ctx **out)
{
    if (!out) return fail(SPLASH_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    splash_options o{16, 16, 0, 0, 128};
    if (opt) o = *opt;
    if (o.tile_w == 0 && o.tile_h == 0) o.tile_w = o.tile_h = 16;
    if (!valid_tile(o.tile_w, o.tile_h)) return fail(SPLASH_ERR_INVALID_ARG, "tile shape must be 16x16, 8x32 or 32x8");
    if (o.spin_limit < 0 || o.test_stall_partition < 0)
        return fail(SPLASH_ERR_INVALID_ARG, "spin_limit and test_stall_partition must be >= 0");
    if (o.spin_limit == 0) o.spin_limit = 1 << 22;
    if (o.gaussian_batch != 0 && o.gaussian_batch != 64 && o.gaussian_batch != 128 && o.gaussian_batch != 256)
        return fail(SPLASH_ERR_INVALID_ARG, "gaussian_batch must be 0 (per-pass defaults), 64, 128 or 256");
    splash_ctx *c = new splash_ctx();
    c->opt = o;
    if (cudaMalloc(&c->d_status, sizeof(uint32_t)) != cudaSuccess || cudaMemset(c->d_status, 0, sizeof(uint32_t)) != cudaSuccess ||
        sort_prepare_device() != cudaSuccess) {
        const std::string e = cudaGetErrorString(cudaGetLastError());
        delete c;
        return fail(SPLASH_ERR_CUDA, "splash_create: " + e);
    }
    *out = c;
    return SPLASH_OK;
}

splash_status splash_destroy(splash_ctx *ctx)
{
    if (!ctx) return SPLASH_OK;
    if (ctx->d_status) cudaFree(ctx->d_status);
    delete ctx;
    return SPLASH_OK;
}

splash_status splash_state_create(splash_ctx *ctx, splash_state **out)
{
    if (!ctx || !out) return fail(SPLASH_ERR_INVALID_ARG, "null argument");
    splash_state *s = new splash_state();
    s->ctx = ctx;
    if (cudaHostAlloc(reinterpret_cast<void **>(&s->h_small), 4 * sizeof(uint64_t), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void **>(&s->h_small_dev), s->h_small, 0) != cudaSuccess ||
        !s->small.ensure(64) ||
        !s->pair_part.ensure(kPairTotalScratchBytes) ||
        cudaMemset(s->pair_part.p, 0, kPairTotalScratchBytes) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->k_ready, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return fail(SPLASH_ERR_OOM, "splash_state_create: allocation failed");
    }
    *out = s;
    return SPLASH_OK;
}

splash_status splash_state_destroy(splash_state *st)
{
    if (!st) return SPLASH_OK;
    if (st->h_small) cudaFreeHost(st->h_small);
    if (st->k_ready) cudaEventDestroy(st->k_ready);
    delete st;
    return SPLASH_OK;
}

splash_status splash_render_forward(splash_ctx *ctx, splash_state *st, const splash_gaussians *g,
                                    const float *medium, const splash_camera *cam, float *image, float *depth,
                                    float *depth01, void *stream)
{
    if (!ctx || !st || st->ctx != ctx) return fail(SPLASH_ERR_INVALID_ARG, "bad context or state");
    splash_status rc;
    if ((rc = check_gaussians(g)) != SPLASH_OK) return rc;
    if ((rc = check_camera(cam)) != SPLASH_OK) return rc;
    if (!medium || !image) return fail(SPLASH_ERR_INVALID_ARG, "null medium or image");
    cudaStream_t s = (cudaStream_t)stream;
    st->has_forward = false;
    st->pixel_forward = false;

    const int64_t n = g->n;
    TileGeom tg{ctx->opt.tile_w, ctx->opt.tile_h, 0, 0};
    tg.tx = (cam->width + tg.tw - 1) / tg.tw;
    tg.ty = (cam->height + tg.th - 1) / tg.th;
    const int ntiles = tg.tx * tg.ty;
    const int64_t npix = (int64_t)cam->width * cam->height;
    const int64_t nn = std::max<int64_t>(n, 1);
    ENSURE(st->rec, sizeof(Rec) * nn);
    ENSURE(st->depth_key, 4 * nn);
    ENSURE(st->tt, 4 * nn);
    ENSURE(st->rect, 8 * nn);
    ENSURE(st->dk0, 4 * nn);
    ENSURE(st->dv0, 4 * nn);
    ENSURE(st->dk1, 4 * nn);
    ENSURE(st->dv1, 4 * nn);
    ENSURE(st->scs, 4 * nn);
    ENSURE(st->scan_sums, 4 * (size_t)(emit_blocks(nn) + 1));
    ENSURE(st->ranges, 8 * (size_t)ntiles);
    ENSURE(st->fT, 4 * npix);
    ENSURE(st->aA, 4 * npix);
    ENSURE(st->zh, 4 * npix);
    ENSURE(st->nlast, 4 * npix);
    ENSURE(st->nwalk, 4 * npix);
    ENSURE(st->tile_walk, 4 * (size_t)ntiles);
    ENSURE(st->sort_scratch, sort_scratch_bytes(nn));
    SortScratch ss;
    sort_scratch_carve(st->sort_scratch.p, nn, &ss);

    const CamK ck = make_cam(*cam);
    uint32_t *dK = st->small.as<uint32_t>();
    {
        Stage t(ctx->prof, SPLASH_STAGE_PREPROCESS, s);
        launch_preprocess_fwd(n, *g, medium, ck, tg, st->rec.as<Rec>(), st->depth_key.as<uint32_t>(),
                              st->tt.as<uint32_t>(), st->rect.as<uint2>(), s);
    }
    // Binning (Sec. III-A), two-level (binning.cu): the Gaussians in depth
    // order are stably sorted by super-tile, then each super-tile's list is
    // split into its tiles' lists, in order
    int nsx = 0;
    const int sbits = super_bits(tg, &nsx);
    const int nsuper = nsx * ((tg.ty + kSuperH - 1) / kSuperH);
    ENSURE(st->sc, 4 * nn);
    // The pair count K and the super-tile entry count K_s are summed by a
    // kernel that stores them, with the status word, into mapped host memory;
    // the host waits for it (k_ready) while the depth sort and the scan run,
    // so that it knows both before the GPU runs out of queued work
    launch_pair_totals(n, st->tt.as<uint32_t>(), st->rect.as<uint2>(), st->sc.as<uint32_t>(), st->pair_part.p,
                       st->h_small_dev, ctx->d_status, s);
    SPLASH_CUDA_TRY(cudaEventRecord(st->k_ready, s));
    const uint32_t *order = nullptr;
    if (n > 0) {
        Stage t(ctx->prof, SPLASH_STAGE_DEPTH_SORT, s);
        const int which = sort_pairs(st->depth_key.as<uint32_t>(), nullptr, st->dk0.as<uint32_t>(), st->dv0.as<uint32_t>(),
                                     st->dk1.as<uint32_t>(), st->dv1.as<uint32_t>(), n, nullptr,
                                     depth_key_bits(ck.znear, ck.zfar), ss, ctx->d_status,
                                     ctx->opt.spin_limit, ctx->opt.test_stall_partition, s, kDepthSortItems);
        order = which ? st->dv1.as<uint32_t>() : st->dv0.as<uint32_t>();
    }
    {
        Stage t(ctx->prof, SPLASH_STAGE_SCAN, s);
        launch_super_scan(n, order, st->sc.as<uint32_t>(), st->scs.as<uint32_t>(), st->scan_sums.as<uint32_t>(),
                          dK + 2, s);  // its total equals K_s
    }
    SPLASH_CUDA_TRY(cudaGetLastError());
    SPLASH_CUDA_TRY(cudaEventSynchronize(st->k_ready));
    if (const uint32_t status = (uint32_t)st->h_small[0]) {
        SPLASH_CUDA_TRY(cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), s));
        return status_failure(status);
    }
    const uint64_t K64 = st->h_small[1];
    // every uint32 offset below is valid only under this bound: nothing that
    // uses them runs before it is checked (K_s <= K: each super-tile entry
    // stands for at least one pair)
    if (K64 >= ((uint64_t)1 << 30)) return fail(SPLASH_ERR_CAPACITY, "more than 2^30 tile/Gaussian pairs");
    const int64_t K = (int64_t)K64;
    const int64_t Ks = (int64_t)std::min<uint64_t>(st->h_small[2], K64);

    const int64_t kk = std::max<int64_t>(K, 1);
    ENSURE(st->tk0, 4 * kk);
    ENSURE(st->tv0, 4 * kk);
    ENSURE(st->tk1, 4 * kk);
    ENSURE(st->tv1, 4 * kk);
    if (kk > nn) {
        ENSURE(st->sort_scratch, sort_scratch_bytes(kk));
    }
    sort_scratch_carve(st->sort_scratch.p, std::max(nn, kk), &ss);
    ENSURE(st->sranges, 8 * (size_t)nsuper);
    ENSURE(st->bin_scratch, 4 * binning_scratch_words(Ks, nsuper, ntiles));
    const BinningScratch bs = binning_scratch_carve(st->bin_scratch.as<uint32_t>(), Ks, nsuper);
    // super-tile entries into buffer pair 1, sorted by super-tile (one pass up
    // to 512 super-tiles); the tile lists go to the value buffer the sort
    // leaves free
    {
        Stage t(ctx->prof, SPLASH_STAGE_EMIT, s);
        launch_emit_super(n, order, st->scs.as<uint32_t>(), st->scan_sums.as<uint32_t>(), st->rect.as<uint2>(), nsx, sbits,
                          st->tk1.as<uint32_t>(), st->tv1.as<uint32_t>(), (uint64_t)Ks, ctx->d_status, s);
    }
    int which = 0;
    // a one-pass super-tile sort leaves each super-tile's list start in its
    // digit offsets: the tile lists take the ranges from there
    const bool one_pass = Ks > 0 && digit_plan(sbits).passes == 1;
    {
        Stage t(ctx->prof, SPLASH_STAGE_TILE_SORT, s);
        which = sort_pairs(st->tk1.as<uint32_t>(), st->tv1.as<uint32_t>(), st->tk0.as<uint32_t>(), st->tv0.as<uint32_t>(),
                           st->tk1.as<uint32_t>(), st->tv1.as<uint32_t>(), Ks, nullptr, sbits, ss, ctx->d_status,
                           ctx->opt.spin_limit, ctx->opt.test_stall_partition, s);
        if (!one_pass)
            launch_ranges(Ks, nullptr, which ? st->tk1.as<uint32_t>() : st->tk0.as<uint32_t>(), st->sranges.as<uint2>(),
                          nsuper, s, (1u << sbits) - 1u);
    }
    const uint32_t *skeys = which ? st->tk1.as<uint32_t>() : st->tk0.as<uint32_t>();
    const uint32_t *svals = which ? st->tv1.as<uint32_t>() : st->tv0.as<uint32_t>();
    uint32_t *gids = which ? st->tv0.as<uint32_t>() : st->tv1.as<uint32_t>();
    {
        Stage t(ctx->prof, SPLASH_STAGE_RANGES, s);
        launch_tile_lists(tg, nsx, sbits, Ks, skeys, svals, st->sranges.as<uint2>(), bs, st->ranges.as<uint2>(), gids,
                          ctx->d_status, s, (uint32_t)K, nullptr, one_pass ? ss.hist : nullptr);
    }
    const uint32_t *tids = nullptr;  // rebuilt from the ranges when a query asks for them
    {
        Stage t(ctx->prof, SPLASH_STAGE_BLEND_FWD, s);
        BlendView v{};
        v.cam = ck;
        v.tg = tg;
        v.ranges = st->ranges.as<uint2>();
        v.gauss_ids = gids;
        v.rec = st->rec.as<Rec>();
        v.image = image;
        v.depth = depth;
        v.depth01 = depth01;
        v.final_T = st->fT.as<float>();
        v.acc_alpha = st->aA.as<float>();
        v.zhat = st->zh.as<float>();
        v.n_last = st->nlast.as<uint32_t>();
        v.n_walk = st->nwalk.as<uint32_t>();
        v.tile_walk = st->tile_walk.as<uint32_t>();
        preclear_backward(st, n, v);
        launch_blend_fwd(v, medium, fwd_batch(ctx->opt), s);
    }
    SPLASH_CUDA_TRY(cudaGetLastError());

    st->has_forward = true;
    st->n = n;
    st->W = cam->width;
    st->H = cam->height;
    st->tg = tg;
    st->K = K;
    st->Ks = Ks;
    st->order = order;
    st->tile_ids = tids;  // null on the two-level path: rebuilt from the ranges when asked for
    st->tid_lazy_ok = false;
    st->gauss_ids = gids;
    return SPLASH_OK;
}

}  // extern "C"

// C++ linkage: called by the C ABI entry points of this file and of pixel.cu
splash_status render_backward_impl(splash_ctx *ctx, splash_state *st, const splash_gaussians *g,
                                   const float *medium, const splash_camera *cam, const float *dL_dimage,
                                   const float *dL_ddepth, const float *dL_ddepth01, const splash_grads *grads,
                                   void *stream)
{
    if (!ctx || !st || st->ctx != ctx) return fail(SPLASH_ERR_INVALID_ARG, "bad context or state");
    splash_status rc;
    if ((rc = check_gaussians(g)) != SPLASH_OK) return rc;
    if ((rc = check_camera(cam)) != SPLASH_OK) return rc;
    if (!medium || !dL_dimage || !grads) return fail(SPLASH_ERR_INVALID_ARG, "null medium, dL_dimage or grads");
    if (grads->quats && (reinterpret_cast<uintptr_t>(grads->quats) & 15))
        return fail(SPLASH_ERR_INVALID_ARG, "grads.quats must be 16-byte aligned");
    if (!st->has_forward || st->n != g->n || st->W != cam->width || st->H != cam->height)
        return fail(SPLASH_ERR_STATE, "backward does not match the last forward on this state");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = g->n;
    const int ntiles = st->tg.tx * st->tg.ty;
    const int nblocks = preprocess_bwd_blocks(std::max<int64_t>(n, 1));
    ENSURE(st->gacc, sizeof(GAcc) * std::max<int64_t>(n, 1));
    ENSURE(st->tile_med, 4 * 6 * (size_t)ntiles);
    ENSURE(st->block_med, 4 * 9 * (size_t)nblocks);
    ENSURE(st->red_scratch, 4 * 16 * (size_t)kColsumParts);
    ENSURE(st->tile_order, 4 * (size_t)ntiles);
    // (every block of the preprocess adjoint writes its block_med row: no clear)
    if ((rc = clear_backward(st, n, s)) != SPLASH_OK) return rc;
    const CamK ck = make_cam(*cam);
    {
        Stage t(ctx->prof, SPLASH_STAGE_BLEND_BWD, s);
        launch_tile_order(st->tile_walk.as<uint32_t>(), ntiles, st->tile_order.as<uint32_t>(), s);
        launch_blend_bwd(backward_view(st, ck, dL_dimage, dL_ddepth, dL_ddepth01), medium, bwd_batch(ctx->opt), s);
    }
    int nb = 0;
    {
        Stage t(ctx->prof, SPLASH_STAGE_PREPROCESS_BWD, s);
        launch_preprocess_bwd(n, *g, medium, ck, st->gacc.as<GAcc>(), st->depth_key.as<uint32_t>(), *grads,
                              st->block_med.as<float>(), &nb, s);
    }
    if (grads->medium) {
        Stage t(ctx->prof, SPLASH_STAGE_MEDIUM_REDUCE, s);
        launch_medium_reduce(st->tile_med.as<float>(), ntiles, st->block_med.as<float>(), nb, grads->medium,
                             st->red_scratch.as<float>(), s);
    }
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}

extern "C" {

splash_status splash_render_backward(splash_ctx *ctx, splash_state *st, const splash_gaussians *g,
                                     const float *medium, const splash_camera *cam, const float *dL_dimage,
                                     const float *dL_ddepth, const float *dL_ddepth01, const splash_grads *grads,
                                     void *stream)
{
    if (st && st->pixel_forward)
        return fail(SPLASH_ERR_STATE, "the last forward on this state was the pixel form: use splash_render_backward_pixel");
    return render_backward_impl(ctx, st, g, medium, cam, dL_dimage, dL_ddepth, dL_ddepth01, grads, stream);
}

}  // extern "C"

// C++ linkage: the fused backward + Adam of both water forms
splash_status backward_adam_impl(splash_ctx *ctx, splash_state *st, const splash_param_buffers *params, int64_t n,
                                 int32_t sh_degree, const splash_camera *cam, const float *dL_dimage,
                                 const float *dL_ddepth, const float *dL_ddepth01, const splash_adam_config *adam,
                                 float *grad_medium, void *stream, const float *chain_medium,
                                 const float *pixel_partials, int pixel_blocks)
{
    if (!ctx || !st || st->ctx != ctx) return fail(SPLASH_ERR_INVALID_ARG, "bad context or state");
    if (!params || !adam || !dL_dimage) return fail(SPLASH_ERR_INVALID_ARG, "null params, adam config or dL_dimage");
    splash_gaussians g{params->means, params->log_scales, params->quats, params->opacity_logits, params->sh, n, sh_degree};
    splash_status rc;
    if ((rc = check_gaussians(&g)) != SPLASH_OK) return rc;
    if ((rc = check_camera(cam)) != SPLASH_OK) return rc;
    if (!params->medium) return fail(SPLASH_ERR_INVALID_ARG, "null medium");
    if (adam->step < 1) return fail(SPLASH_ERR_INVALID_ARG, "Adam step must be >= 1");
    const splash_param_buffers *mv[2] = {&adam->m, &adam->v};
    for (int w = 0; w < 2; w++) {
        const splash_param_buffers &b = *mv[w];
        if (!b.medium || (n > 0 && (!b.means || !b.log_scales || !b.quats || !b.opacity_logits || !b.sh)))
            return fail(SPLASH_ERR_INVALID_ARG, "null Adam moment buffer");
        if (n > 0 && (reinterpret_cast<uintptr_t>(b.quats) & 15))
            return fail(SPLASH_ERR_INVALID_ARG, "quaternion moments must be 16-byte aligned");
    }
    if (!st->has_forward || st->n != n || st->W != cam->width || st->H != cam->height)
        return fail(SPLASH_ERR_STATE, "backward does not match the last forward on this state");
    cudaStream_t s = (cudaStream_t)stream;
    const int ntiles = st->tg.tx * st->tg.ty;
    const int nblocks = preprocess_bwd_blocks(std::max<int64_t>(n, 1));
    ENSURE(st->gacc, sizeof(GAcc) * std::max<int64_t>(n, 1));
    ENSURE(st->tile_med, 4 * 6 * (size_t)ntiles);
    ENSURE(st->block_med, 4 * 9 * (size_t)nblocks);
    ENSURE(st->gmed, 4 * 16);
    ENSURE(st->red_scratch, 4 * 16 * (size_t)kColsumParts);
    ENSURE(st->tile_order, 4 * (size_t)ntiles);
    // (every block of the fused adjoint writes its block_med row: no clear)
    if ((rc = clear_backward(st, n, s)) != SPLASH_OK) return rc;
    const CamK ck = make_cam(*cam);
    {
        Stage t(ctx->prof, SPLASH_STAGE_BLEND_BWD, s);
        launch_tile_order(st->tile_walk.as<uint32_t>(), ntiles, st->tile_order.as<uint32_t>(), s);
        launch_blend_bwd(backward_view(st, ck, dL_dimage, dL_ddepth, dL_ddepth01), chain_medium,
                         bwd_batch(ctx->opt), s);
    }
    int nb = 0;
    {
        Stage t(ctx->prof, SPLASH_STAGE_PREPROCESS_BWD, s);
        launch_preprocess_bwd_adam(n, sh_degree, *params, chain_medium, ck, st->gacc.as<GAcc>(),
                                   st->depth_key.as<uint32_t>(), *adam, st->block_med.as<float>(), &nb, s);
    }
    {
        Stage t(ctx->prof, SPLASH_STAGE_MEDIUM_REDUCE, s);
        if (pixel_partials) {  // the pixel form's medium gradient (its chain ran with a zero medium)
            launch_pixel_medium_final(pixel_partials, pixel_blocks, st->gmed.as<float>(), s);
            launch_medium_adam(params->medium, st->gmed.as<float>(), *adam, s);
        } else {
            launch_medium_reduce_adam(st->tile_med.as<float>(), ntiles, st->block_med.as<float>(), nb, params->medium,
                                      st->gmed.as<float>(), st->red_scratch.as<float>(), *adam, s);
        }
    }
    if (grad_medium)
        SPLASH_CUDA_TRY(cudaMemcpyAsync(grad_medium, st->gmed.p, 9 * sizeof(float), cudaMemcpyDeviceToDevice, s));
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}

extern "C" {

splash_status splash_render_backward_adam(splash_ctx *ctx, splash_state *st, const splash_param_buffers *params,
                                          int64_t n, int32_t sh_degree, const splash_camera *cam,
                                          const float *dL_dimage, const float *dL_ddepth, const float *dL_ddepth01,
                                          const splash_adam_config *adam, float *grad_medium, void *stream)
{
    if (st && st->pixel_forward)
        return fail(SPLASH_ERR_STATE, "the last forward on this state was the pixel form: use splash_render_backward_adam_pixel");
    if (!params) return fail(SPLASH_ERR_INVALID_ARG, "null params");
    return backward_adam_impl(ctx, st, params, n, sh_degree, cam, dL_dimage, dL_ddepth, dL_ddepth01, adam, grad_medium,
                              stream, params->medium, nullptr, 0);
}

splash_status splash_state_get_info(const splash_state *st, splash_state_info *out)
{
    if (!st || !out) return fail(SPLASH_ERR_INVALID_ARG, "null argument");
    if (!st->has_forward) return fail(SPLASH_ERR_STATE, "no forward on this state");
    out->n_keys = st->K;
    out->tiles_x = st->tg.tx;
    out->tiles_y = st->tg.ty;
    out->tile_w = st->tg.tw;
    out->tile_h = st->tg.th;
    out->n_gaussians = st->n;
    out->tile_ids = st->tile_ids;  // null when the forward kept only the lists and their ranges
    out->gauss_ids = st->gauss_ids;
    out->ranges = st->ranges.as<uint32_t>();
    out->depth_keys = st->depth_key.as<uint32_t>();
    out->tiles_touched = st->tt.as<uint32_t>();
    out->records = st->rec.as<float>();
    out->final_T = st->fT.as<float>();
    out->acc_alpha = st->aA.as<float>();
    out->n_last = st->nlast.as<uint32_t>();
    out->n_walk = st->nwalk.as<uint32_t>();
    return SPLASH_OK;
}

splash_status splash_state_copy(const splash_state *st, int32_t field, void *dst, int64_t bytes, void *stream)
{
    if (!st || !dst) return fail(SPLASH_ERR_INVALID_ARG, "null argument");
    if (!st->has_forward) return fail(SPLASH_ERR_STATE, "no forward on this state");
    const int64_t npix = (int64_t)st->W * st->H, ntiles = (int64_t)st->tg.tx * st->tg.ty;
    const void *src = nullptr;
    int64_t size = 0;
    switch (field) {
    case SPLASH_FIELD_TILE_IDS:
        src = st->tile_ids ? st->tile_ids : rebuilt_tile_ids(st, (cudaStream_t)stream);
        if (!src) return fail(SPLASH_ERR_OOM, "tile id buffer");
        size = 4 * st->K;
        break;
    case SPLASH_FIELD_GAUSS_IDS: src = st->gauss_ids; size = 4 * st->K; break;
    case SPLASH_FIELD_RANGES: src = st->ranges.p; size = 8 * ntiles; break;
    case SPLASH_FIELD_DEPTH_KEYS: src = st->depth_key.p; size = 4 * st->n; break;
    case SPLASH_FIELD_TILES_TOUCHED: src = st->tt.p; size = 4 * st->n; break;
    case SPLASH_FIELD_RECORDS: src = st->rec.p; size = (int64_t)sizeof(Rec) * st->n; break;
    case SPLASH_FIELD_FINAL_T: src = st->fT.p; size = 4 * npix; break;
    case SPLASH_FIELD_ACC_ALPHA: src = st->aA.p; size = 4 * npix; break;
    case SPLASH_FIELD_N_LAST: src = st->nlast.p; size = 4 * npix; break;
    case SPLASH_FIELD_N_WALK: src = st->nwalk.p; size = 4 * npix; break;
    case SPLASH_FIELD_RECTS: src = st->rect.p; size = 8 * st->n; break;
    default: return fail(SPLASH_ERR_INVALID_ARG, "unknown field");
    }
    if (bytes != size) return fail(SPLASH_ERR_INVALID_ARG, "byte count does not match the field's size");
    if (size > 0) SPLASH_CUDA_TRY(cudaMemcpyAsync(dst, src, (size_t)size, cudaMemcpyDefault, (cudaStream_t)stream));
    return SPLASH_OK;
}

splash_status splash_loss_l1_ssim(splash_ctx *ctx, splash_state *st, const float *image, const float *target,
                                  int32_t channels, int32_t height, int32_t width, float lam, float *loss_dev,
                                  float *dL_dimage, void *stream)
{
    if (!ctx || !st || st->ctx != ctx) return fail(SPLASH_ERR_INVALID_ARG, "bad context or state");
    if (!image || !target || !loss_dev) return fail(SPLASH_ERR_INVALID_ARG, "null image, target or loss");
    if (channels <= 0 || height <= 0 || width <= 0) return fail(SPLASH_ERR_INVALID_ARG, "bad image shape");
    ENSURE(st->loss_scratch, 4 * ssim_scratch_floats(channels, height, width));
    {
        Stage t(ctx->prof, SPLASH_STAGE_LOSS, (cudaStream_t)stream);
        launch_ssim_loss(image, target, channels, height, width, lam, loss_dev, dL_dimage,
                         st->loss_scratch.as<float>(), (cudaStream_t)stream);
    }
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}

splash_status splash_sort_pairs_u32(splash_ctx *ctx, splash_state *st, const uint32_t *keys_in, const uint32_t *vals_in,
                                    uint32_t *keys_out, uint32_t *vals_out, int64_t n, int32_t key_bits, void *stream)
{
    if (!ctx || !st || st->ctx != ctx) return fail(SPLASH_ERR_INVALID_ARG, "bad context or state");
    if (n < 0 || n >= ((int64_t)1 << 30)) return fail(SPLASH_ERR_INVALID_ARG, "n must be in [0, 2^30)");
    if (key_bits < 0 || key_bits > 32) return fail(SPLASH_ERR_INVALID_ARG, "key_bits must be in 0..32");
    if (n == 0) return SPLASH_OK;
    if (!keys_in || !keys_out || !vals_out) return fail(SPLASH_ERR_INVALID_ARG, "null buffer");
    if (reinterpret_cast<uintptr_t>(keys_in) & 15) return fail(SPLASH_ERR_INVALID_ARG, "keys_in must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    ENSURE(st->tmp_k, 4 * (size_t)n);
    ENSURE(st->tmp_v, 4 * (size_t)n);
    ENSURE(st->sort_scratch, sort_scratch_bytes(n));
    SortScratch ss;
    sort_scratch_carve(st->sort_scratch.p, n, &ss);
    const int which = sort_pairs(keys_in, vals_in, keys_out, vals_out, st->tmp_k.as<uint32_t>(), st->tmp_v.as<uint32_t>(),
                                 n, nullptr, key_bits, ss, ctx->d_status, ctx->opt.spin_limit, ctx->opt.test_stall_partition, s);
    if (which) {
        SPLASH_CUDA_TRY(cudaMemcpyAsync(keys_out, st->tmp_k.p, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s));
        SPLASH_CUDA_TRY(cudaMemcpyAsync(vals_out, st->tmp_v.p, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s));
    }
    SPLASH_CUDA_TRY(cudaGetLastError());
    // the forward state's pair buffers are untouched, but the scratch is shared
    return SPLASH_OK;
}

splash_status splash_profile_enable(splash_ctx *ctx, int32_t on)
{
    if (!ctx) return fail(SPLASH_ERR_INVALID_ARG, "null context");
    double ms[SPLASH_STAGE_COUNT];
    int64_t cnt[SPLASH_STAGE_COUNT];
    splash_status rc = splash_profile_read(ctx, ms, cnt);  // drain and clear
    ctx->prof.on = on != 0;
    return rc;
}

splash_status splash_profile_mask(splash_ctx *ctx, uint32_t stage_mask)
{
    if (!ctx) return fail(SPLASH_ERR_INVALID_ARG, "null context");
    ctx->prof.mask = stage_mask;
    return SPLASH_OK;
}

splash_status splash_profile_read(splash_ctx *ctx, double *ms, int64_t *counts)
{
    if (!ctx || !ms || !counts) return fail(SPLASH_ERR_INVALID_ARG, "null argument");
    Prof &p = ctx->prof;
    splash_status rc = SPLASH_OK;
    for (auto &r : p.pending) {
        float t = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
            rc = fail(SPLASH_ERR_CUDA, std::string("profile: ") + cudaGetErrorString(cudaGetLastError()));
        } else {
            p.ms[r.stage] += t;
            p.cnt[r.stage] += 1;
        }
        p.spare.push_back(r.a);
        p.spare.push_back(r.b);
    }
    p.pending.clear();
    for (int i = 0; i < SPLASH_STAGE_COUNT; i++) {
        ms[i] = p.ms[i];
        counts[i] = p.cnt[i];
        p.ms[i] = 0.0;
        p.cnt[i] = 0;
    }
    return rc;
}

uint64_t splash_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

splash_status splash_sync_status(splash_ctx *ctx, void *stream)
{
    if (!ctx) return fail(SPLASH_ERR_INVALID_ARG, "null context");
    cudaStream_t s = (cudaStream_t)stream;
    SPLASH_CUDA_TRY(cudaStreamSynchronize(s));
    uint32_t status = 0;
    SPLASH_CUDA_TRY(cudaMemcpy(&status, ctx->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (status) {
        SPLASH_CUDA_TRY(cudaMemset(ctx->d_status, 0, sizeof(uint32_t)));
        return status_failure(status);
    }
    return SPLASH_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// ABI self-description: sizeof and offsetof of every struct in splash.h, for
// bindings to check their mirrors against the compiler's own layout.

#define SPLASH_LAYOUT_STRUCTS(X)                                                                              \
    X(splash_camera, width, height, fx, fy, cx, cy, world_to_cam, z_near, z_far)                              \
    X(splash_gaussians, means, log_scales, quats, opacity_logits, sh, n, sh_degree)                           \
    X(splash_grads, means, log_scales, quats, opacity_logits, sh, medium)                                     \
    X(splash_options, tile_w, tile_h, spin_limit, test_stall_partition, gaussian_batch)                       \
    X(splash_param_buffers, means, log_scales, quats, opacity_logits, sh, medium)                             \
    X(splash_adam_config, m, v, lr_means, lr_log_scales, lr_quats, lr_opacity_logits, lr_sh, lr_medium, beta1, \
      beta2, eps, step, clamp_medium, medium_min, prior, lambda_est, densify_stats)                           \
    X(splash_state_info, n_keys, tiles_x, tiles_y, tile_w, tile_h, n_gaussians, tile_ids, gauss_ids, ranges,  \
      depth_keys, tiles_touched, records, final_T, acc_alpha, n_last, n_walk)                                 \
    X(splash_adam_group, param, grad, m, v, n, lr, clamp_min, has_clamp)                                      \
    X(splash_mlp_params, W1, b1, W2, b2, W3, b3)                                                              \
    X(splash_mlp_adam, lr, beta1, beta2, eps)                                                                 \
    X(splash_densify_options, grad_threshold, min_opacity, percent_dense, extent)                             \
    X(splash_backscatter_options, resized_height, edges, intervals, pad, p_dark, b_max, beta_max)             \
    X(splash_backscatter_result, beta_b, b_inf, residual, n_points, n_dark, width, height, pad, point_z, point_v)

namespace {

struct LayoutSink {
    int32_t *sizes, *n_fields, *offsets;
    int32_t ns = 0, no = 0;
    void begin(size_t size)
    {
        if (sizes) sizes[ns] = (int32_t)size;
        if (n_fields) n_fields[ns] = 0;
    }
    void field(size_t off)
    {
        if (offsets) offsets[no] = (int32_t)off;
        if (n_fields) n_fields[ns]++;
        no++;
    }
    void end() { ns++; }
};

}  // namespace

#define SPLASH_LAYOUT_FIELD(T, f) sink.field(offsetof(T, f));

#define SPLASH_FE_1(M, T, x) M(T, x)
#define SPLASH_FE_2(M, T, x, ...) M(T, x) SPLASH_FE_1(M, T, __VA_ARGS__)
#define SPLASH_FE_3(M, T, x, ...) M(T, x) SPLASH_FE_2(M, T, __VA_ARGS__)
#define SPLASH_FE_4(M, T, x, ...) M(T, x) SPLASH_FE_3(M, T, __VA_ARGS__)
#define SPLASH_FE_5(M, T, x, ...) M(T, x) SPLASH_FE_4(M, T, __VA_ARGS__)
#define SPLASH_FE_6(M, T, x, ...) M(T, x) SPLASH_FE_5(M, T, __VA_ARGS__)
#define SPLASH_FE_7(M, T, x, ...) M(T, x) SPLASH_FE_6(M, T, __VA_ARGS__)
#define SPLASH_FE_8(M, T, x, ...) M(T, x) SPLASH_FE_7(M, T, __VA_ARGS__)
#define SPLASH_FE_9(M, T, x, ...) M(T, x) SPLASH_FE_8(M, T, __VA_ARGS__)
#define SPLASH_FE_10(M, T, x, ...) M(T, x) SPLASH_FE_9(M, T, __VA_ARGS__)
#define SPLASH_FE_11(M, T, x, ...) M(T, x) SPLASH_FE_10(M, T, __VA_ARGS__)
#define SPLASH_FE_12(M, T, x, ...) M(T, x) SPLASH_FE_11(M, T, __VA_ARGS__)
#define SPLASH_FE_13(M, T, x, ...) M(T, x) SPLASH_FE_12(M, T, __VA_ARGS__)
#define SPLASH_FE_14(M, T, x, ...) M(T, x) SPLASH_FE_13(M, T, __VA_ARGS__)
#define SPLASH_FE_15(M, T, x, ...) M(T, x) SPLASH_FE_14(M, T, __VA_ARGS__)
#define SPLASH_FE_16(M, T, x, ...) M(T, x) SPLASH_FE_15(M, T, __VA_ARGS__)
#define SPLASH_FE_17(M, T, x, ...) M(T, x) SPLASH_FE_16(M, T, __VA_ARGS__)
#define SPLASH_FE_PICK(_1, _2, _3, _4, _5, _6, _7, _8, _9, _10, _11, _12, _13, _14, _15, _16, _17, NAME, ...) NAME
#define SPLASH_FOR_EACH(M, T, ...)                                                                                   \
    SPLASH_FE_PICK(__VA_ARGS__, SPLASH_FE_17, SPLASH_FE_16, SPLASH_FE_15, SPLASH_FE_14, SPLASH_FE_13, SPLASH_FE_12, \
                   SPLASH_FE_11, SPLASH_FE_10, SPLASH_FE_9, SPLASH_FE_8, SPLASH_FE_7, SPLASH_FE_6, SPLASH_FE_5,     \
                   SPLASH_FE_4, SPLASH_FE_3, SPLASH_FE_2, SPLASH_FE_1)(M, T, __VA_ARGS__)
#define SPLASH_LAYOUT_STRUCT(T, ...)                       \
    sink.begin(sizeof(T));                                 \
    SPLASH_FOR_EACH(SPLASH_LAYOUT_FIELD, T, __VA_ARGS__) \
    sink.end();

extern "C" splash_status splash_abi_layout(int32_t *sizes, int32_t *n_fields, int32_t *offsets, int32_t *n_structs,
                                           int32_t *n_offsets)
{
    LayoutSink sink{sizes, n_fields, offsets};
    SPLASH_LAYOUT_STRUCTS(SPLASH_LAYOUT_STRUCT)
    if (n_structs) *n_structs = sink.ns;
    if (n_offsets) *n_offsets = sink.no;
    return SPLASH_OK;
}
