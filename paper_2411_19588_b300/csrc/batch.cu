// Batched form: many views (of uneven resolution) of one scene rendered and
// differentiated as one unit.
//
//  * No host synchronisation and no allocation in forward/backward, so the
//    pair of calls can be captured in a CUDA graph: each view's pair count
//    stays on the device, clamped to a capacity measured once by
//    splash_batch_calibrate (overflow sets SPLASH_ERR_CAPACITY, every index
//    stays in range).
//  * Per view: preprocess, depth sort, and the two-level binning (super-tile
//    entries, their sort, the tile lists: the same kernels as a single
//    render, on device-side counts).
//  * One work queue of all (view, tile) items, ordered longest list first,
//    drives ONE persistent blend launch forward and ONE backward.
//  * The adjoint of the preprocess reads every Gaussian once and sums its
//    gradient over all views before writing it.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "host.h"

using namespace splash;
using namespace splash_host;

namespace {

constexpr int kMaxViews = 256;  // view index lives in the top 8 bits of a work item

__global__ void k_clamp_count(const uint32_t *__restrict__ raw, uint32_t cap, uint32_t *__restrict__ eff,
                              uint32_t *__restrict__ status)
{
    const uint32_t k = *raw;
    if (k > cap) atomicOr(status, kStatusCapacity);
    *eff = min(k, cap);
}

// one work item per (view, tile): key = 2^24 - 1 - list length (an ascending
// sort gives the longest lists first), value = view << 24 | tile
__global__ void k_build_items(const BlendView *__restrict__ views, const int64_t *__restrict__ tiles_off, int V,
                              int64_t total, uint32_t *__restrict__ keys, uint32_t *__restrict__ vals)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int lo = 0, hi = V - 1;  // the view whose tile range holds t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tiles_off[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    const uint32_t local = (uint32_t)(t - tiles_off[lo]);
    const uint2 r = views[lo].ranges[local];
    const uint32_t len = min(r.y - r.x, 0xffffffu);
    keys[t] = 0xffffffu - len;
    vals[t] = ((uint32_t)lo << 24) | local;
}

}  // namespace

struct splash_batch {
    splash_ctx *ctx = nullptr;
    int V = 0;
    std::vector<splash_camera> cams;
    std::vector<CamK> ck;
    std::vector<TileGeom> tg;
    std::vector<int64_t> tiles_off, pix_off, cap, cap_off;
    std::vector<int64_t> scap;  // per view: capacity of the super-tile entries
    int64_t tiles_total = 0, pix_total = 0, cap_total = 0, cap_max = 0;
    int64_t n = -1;
    int64_t ns = 0;  // per-view stride of the depth keys: n rounded up to a multiple of 4 (16-byte aligned slices)
    int deg = 0;
    bool calibrated = false, has_forward = false;
    int ctas_fwd = 0, ctas_bwd = 0;
    // device
    Buf rec, depth_key, tt, rect, dk0, dv0, dk1, dv1, scs, scan_sums, sort_scratch;  // scs: super-tile counts in depth order
    Buf pair_k, pair_v, tmp_k, tmp_v;  // per-view tile lists in pair_v (cap_off); super-tile sort buffers
    Buf tmp2_v;                        // the super-tile sort's second value buffer (cap_max)
    Buf ranges, counts;                // counts[2v] = the view's pairs, counts[2v + 1] = its super-tile entries (clamped)
    Buf sc, sranges, bin_scratch, pair_part, scount;  // two-level binning; scount[v] = super-tile entries emitted
    int nsuper_max = 0;
    int64_t bin_words = 0;
    Buf fT, aA, zh, nlast, nwalk;
    Buf items_k, items_v, items_k1, items_v1, item_meta;  // item_meta: [0] = item count, [1] = ticket counter
    Buf views, tiles_off_dev;
    Buf gacc, tile_med, block_med, red_scratch;
    BlendView *views_host = nullptr;  // pinned copy of the per-view descriptors
    ~splash_batch()
    {
        if (views_host) cudaFreeHost(views_host);
    }
};

extern "C" {

splash_status splash_batch_create(splash_ctx *ctx, int32_t n_views, const splash_camera *cams, splash_batch **out)
{
    if (!ctx || !cams || !out) return fail(SPLASH_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (n_views < 1 || n_views > kMaxViews) return fail(SPLASH_ERR_INVALID_ARG, "n_views must be in 1..256");
    splash_batch *b = new splash_batch();
    b->ctx = ctx;
    b->V = n_views;
    b->tiles_off.push_back(0);
    b->pix_off.push_back(0);
    for (int v = 0; v < n_views; v++) {
        splash_status rc = check_camera(&cams[v]);
        if (rc != SPLASH_OK) {
            delete b;
            return rc;
        }
        b->cams.push_back(cams[v]);
        b->ck.push_back(make_cam(cams[v]));
        TileGeom tg{ctx->opt.tile_w, ctx->opt.tile_h, 0, 0};
        tg.tx = (cams[v].width + tg.tw - 1) / tg.tw;
        tg.ty = (cams[v].height + tg.th - 1) / tg.th;
        if ((int64_t)tg.tx * tg.ty >= (1 << 24)) {
            delete b;
            return fail(SPLASH_ERR_INVALID_ARG, "a view has more than 2^24 tiles");
        }
        b->tg.push_back(tg);
        b->tiles_off.push_back(b->tiles_off.back() + (int64_t)tg.tx * tg.ty);
        b->pix_off.push_back(b->pix_off.back() + (int64_t)cams[v].width * cams[v].height);
    }
    b->tiles_total = b->tiles_off.back();
    b->pix_total = b->pix_off.back();
    if (cudaMallocHost(&b->views_host, sizeof(BlendView) * n_views) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(SPLASH_ERR_OOM, "splash_batch_create: pinned allocation failed");
    }
    memset(b->views_host, 0, sizeof(BlendView) * n_views);
    *out = b;
    return SPLASH_OK;
}

splash_status splash_batch_destroy(splash_batch *b)
{
    delete b;
    return SPLASH_OK;
}

splash_status splash_batch_calibrate(splash_batch *b, const splash_gaussians *g, const float *medium, float headroom,
                                     void *stream)
{
    if (!b) return fail(SPLASH_ERR_INVALID_ARG, "null batch");
    splash_status rc;
    if ((rc = check_gaussians(g)) != SPLASH_OK) return rc;
    if (!medium) return fail(SPLASH_ERR_INVALID_ARG, "null medium");
    if (!(headroom >= 0.01f)) return fail(SPLASH_ERR_INVALID_ARG, "headroom must be >= 0.01");
    cudaStream_t s = (cudaStream_t)stream;
    // one eager render per view (same ctx options) measures its pair count
    splash_state *st = nullptr;
    if ((rc = splash_state_create(b->ctx, &st)) != SPLASH_OK) return rc;
    int64_t maxpix = 0;
    for (int v = 0; v < b->V; v++) maxpix = std::max<int64_t>(maxpix, (int64_t)b->cams[v].width * b->cams[v].height);
    Buf img;
    if (!img.ensure(4 * 3 * (size_t)maxpix)) {
        splash_state_destroy(st);
        return fail(SPLASH_ERR_OOM, "splash_batch_calibrate: image buffer");
    }
    b->cap.assign(b->V, 0);
    b->scap.assign(b->V, 0);
    b->cap_off.assign(b->V + 1, 0);
    for (int v = 0; v < b->V; v++) {
        rc = splash_render_forward(b->ctx, st, g, medium, &b->cams[v], img.as<float>(), nullptr, nullptr, s);
        if (rc != SPLASH_OK) {
            splash_state_destroy(st);
            return rc;
        }
        // multiples of 4 keep every view's slice of the pair buffers 16-byte aligned
        b->cap[v] = (((int64_t)((double)st->K * headroom) + 1024) + 3) & ~(int64_t)3;
        b->cap_off[v + 1] = b->cap_off[v] + b->cap[v];
        b->scap[v] = std::min(b->cap[v], (((int64_t)((double)st->Ks * headroom) + 1024) + 3) & ~(int64_t)3);
    }
    splash_state_destroy(st);
    b->cap_total = b->cap_off.back();
    b->cap_max = *std::max_element(b->cap.begin(), b->cap.end());
    if (b->cap_max >= ((int64_t)1 << 30)) return fail(SPLASH_ERR_CAPACITY, "more than 2^30 pairs in one view");
    const int64_t n = g->n, nn = std::max<int64_t>(n, 1), V = b->V;
    b->ns = (nn + 3) & ~(int64_t)3;
    ENSURE(b->rec, sizeof(Rec) * V * nn);
    ENSURE(b->depth_key, 4 * V * b->ns);
    ENSURE(b->tt, 4 * nn);
    ENSURE(b->rect, 8 * nn);
    ENSURE(b->dk0, 4 * nn);
    ENSURE(b->dv0, 4 * nn);
    ENSURE(b->dk1, 4 * nn);
    ENSURE(b->dv1, 4 * nn);
    ENSURE(b->scs, 4 * nn);
    ENSURE(b->scan_sums, 4 * (size_t)(emit_blocks(nn) + 1));
    const int64_t sort_n = std::max<int64_t>(std::max<int64_t>(nn, b->cap_max), b->tiles_total);
    ENSURE(b->sort_scratch, sort_scratch_bytes(sort_n));
    ENSURE(b->pair_k, 4 * (size_t)b->cap_total);
    ENSURE(b->pair_v, 4 * (size_t)b->cap_total);
    ENSURE(b->tmp_k, 4 * (size_t)b->cap_max);
    ENSURE(b->tmp_v, 4 * (size_t)b->cap_max);
    ENSURE(b->tmp2_v, 4 * (size_t)b->cap_max);
    // two-level binning per view (the super-tile entry capacity is at most the pair capacity)
    b->nsuper_max = 0;
    b->bin_words = 0;
    for (int v = 0; v < b->V; v++) {
        int nsx = 0;
        super_bits(b->tg[v], &nsx);
        const int nsuper = nsx * ((b->tg[v].ty + kSuperH - 1) / kSuperH);
        b->nsuper_max = std::max(b->nsuper_max, nsuper);
        b->bin_words = std::max<int64_t>(b->bin_words, (int64_t)binning_scratch_words(b->scap[v], nsuper,
                                                                                     b->tg[v].tx * b->tg[v].ty));
    }
    ENSURE(b->sc, 4 * nn);
    ENSURE(b->sranges, 8 * (size_t)b->nsuper_max);
    ENSURE(b->bin_scratch, 4 * (size_t)b->bin_words);
    ENSURE(b->scount, 4 * (size_t)V);
    if (b->pair_part.cap < kPairTotalScratchBytes) {  // its ticket is kept zero by every launch
        ENSURE(b->pair_part, kPairTotalScratchBytes);
        SPLASH_CUDA_TRY(cudaMemsetAsync(b->pair_part.p, 0, kPairTotalScratchBytes, s));
    }
    ENSURE(b->ranges, 8 * (size_t)b->tiles_total);
    ENSURE(b->counts, 8 * (size_t)V);
    ENSURE(b->fT, 4 * (size_t)b->pix_total);
    ENSURE(b->aA, 4 * (size_t)b->pix_total);
    ENSURE(b->zh, 4 * (size_t)b->pix_total);
    ENSURE(b->nlast, 4 * (size_t)b->pix_total);
    ENSURE(b->nwalk, 4 * (size_t)b->pix_total);
    ENSURE(b->items_k, 4 * (size_t)b->tiles_total);
    ENSURE(b->items_v, 4 * (size_t)b->tiles_total);
    ENSURE(b->items_k1, 4 * (size_t)b->tiles_total);
    ENSURE(b->items_v1, 4 * (size_t)b->tiles_total);
    ENSURE(b->item_meta, 16);
    ENSURE(b->views, sizeof(BlendView) * V);
    ENSURE(b->tiles_off_dev, 8 * (size_t)(V + 1));
    ENSURE(b->gacc, sizeof(GAcc) * V * nn);
    ENSURE(b->tile_med, 4 * 6 * (size_t)b->tiles_total);
    ENSURE(b->block_med, 4 * 9 * (size_t)preprocess_bwd_multi_blocks(nn));
    ENSURE(b->red_scratch, 4 * 16 * (size_t)kColsumParts);
    // pair buffers start as valid entries (tile 0, Gaussian 0): after a capacity
    // overflow a view's unwritten slots can only hold ids that are in range
    SPLASH_CUDA_TRY(cudaMemsetAsync(b->pair_k.p, 0, 4 * (size_t)b->cap_total, s));
    SPLASH_CUDA_TRY(cudaMemsetAsync(b->pair_v.p, 0, 4 * (size_t)b->cap_total, s));
    SPLASH_CUDA_TRY(cudaMemsetAsync(b->tmp_k.p, 0, 4 * (size_t)b->cap_max, s));
    SPLASH_CUDA_TRY(cudaMemsetAsync(b->tmp_v.p, 0, 4 * (size_t)b->cap_max, s));
    SPLASH_CUDA_TRY(cudaMemsetAsync(b->tmp2_v.p, 0, 4 * (size_t)b->cap_max, s));
    const uint32_t nitems = (uint32_t)b->tiles_total;
    SPLASH_CUDA_TRY(cudaMemcpyAsync(b->item_meta.p, &nitems, 4, cudaMemcpyHostToDevice, s));
    SPLASH_CUDA_TRY(cudaMemcpyAsync(b->tiles_off_dev.p, b->tiles_off.data(), 8 * (V + 1), cudaMemcpyHostToDevice, s));
    SPLASH_CUDA_TRY(cudaStreamSynchronize(s));
    const int tw = b->ctx->opt.tile_w, th = b->ctx->opt.tile_h;
    b->ctas_fwd = blend_persistent_ctas(tw, th, fwd_batch(b->ctx->opt), false);
    b->ctas_bwd = blend_persistent_ctas(tw, th, bwd_batch(b->ctx->opt), true);
    b->n = n;
    b->deg = g->sh_degree;
    b->calibrated = true;
    b->has_forward = false;
    return SPLASH_OK;
}

splash_status splash_batch_forward(splash_batch *b, const splash_gaussians *g, const float *medium,
                                   float *const *images, float *const *depths, float *const *depth01s, void *stream)
{
    if (!b || !b->calibrated) return fail(SPLASH_ERR_STATE, "batch not calibrated");
    splash_status rc;
    if ((rc = check_gaussians(g)) != SPLASH_OK) return rc;
    if (g->n != b->n || g->sh_degree != b->deg)
        return fail(SPLASH_ERR_INVALID_ARG, "Gaussian count or SH degree differs from the calibration");
    if (!medium || !images) return fail(SPLASH_ERR_INVALID_ARG, "null medium or image table");
    for (int v = 0; v < b->V; v++)
        if (!images[v]) return fail(SPLASH_ERR_INVALID_ARG, "null image for a view");
    cudaStream_t s = (cudaStream_t)stream;
    splash_ctx *ctx = b->ctx;
    const int64_t n = b->n, V = b->V;
    SortScratch ss;
    sort_scratch_carve(b->sort_scratch.p,
                       std::max<int64_t>(std::max<int64_t>(std::max<int64_t>(n, 1), b->cap_max), b->tiles_total), &ss);
    uint32_t *counts = b->counts.as<uint32_t>();
    for (int v = 0; v < V; v++) {
        BlendView &d = b->views_host[v];
        d.cam = b->ck[v];
        d.tg = b->tg[v];
        d.ranges = b->ranges.as<uint2>() + b->tiles_off[v];
        d.gauss_ids = b->pair_v.as<uint32_t>() + b->cap_off[v];
        d.rec = b->rec.as<Rec>() + v * n;
        d.image = images[v];
        d.depth = depths ? depths[v] : nullptr;
        d.depth01 = depth01s ? depth01s[v] : nullptr;
        d.final_T = b->fT.as<float>() + b->pix_off[v];
        d.acc_alpha = b->aA.as<float>() + b->pix_off[v];
        d.zhat = b->zh.as<float>() + b->pix_off[v];
        d.n_last = b->nlast.as<uint32_t>() + b->pix_off[v];
        d.n_walk = b->nwalk.as<uint32_t>() + b->pix_off[v];
        d.gacc = b->gacc.as<GAcc>() + v * n;
        d.tile_medium = b->tile_med.as<float>() + 6 * b->tiles_off[v];
    }
    SPLASH_CUDA_TRY(cudaMemcpyAsync(b->views.p, b->views_host, sizeof(BlendView) * V, cudaMemcpyHostToDevice, s));
    for (int v = 0; v < V; v++) {
        const TileGeom &tg = b->tg[v];
        const int ntiles = tg.tx * tg.ty;
        uint32_t *dk = b->depth_key.as<uint32_t>() + v * b->ns;
        {
            Stage t(ctx->prof, SPLASH_STAGE_PREPROCESS, s);
            launch_preprocess_fwd(n, *g, medium, b->ck[v], tg, b->rec.as<Rec>() + v * n, dk, b->tt.as<uint32_t>(),
                                  b->rect.as<uint2>(), s);
        }
        const uint32_t *order = nullptr;
        if (n > 0) {
            Stage t(ctx->prof, SPLASH_STAGE_DEPTH_SORT, s);
            const int which = sort_pairs(dk, nullptr, b->dk0.as<uint32_t>(), b->dv0.as<uint32_t>(), b->dk1.as<uint32_t>(),
                                         b->dv1.as<uint32_t>(), n, nullptr, depth_key_bits(b->ck[v].znear, b->ck[v].zfar),
                                         ss, ctx->d_status, ctx->opt.spin_limit,
                                         ctx->opt.test_stall_partition, s, kDepthSortItems);
            order = which ? b->dv1.as<uint32_t>() : b->dv0.as<uint32_t>();
        }
        // two-level binning, as a single render does, on device-side counts bounded by
        // the view's capacities (pairs; super-tile entries, measured alike)
        int nsx = 0;
        const int sbits = super_bits(tg, &nsx);
        const int nsuper = nsx * ((tg.ty + kSuperH - 1) / kSuperH);
        uint32_t *ents = counts + 2 * v + 1;  // super-tile entries in use (clamped)
        {
            Stage t(ctx->prof, SPLASH_STAGE_SCAN, s);
            launch_pair_totals(n, b->tt.as<uint32_t>(), b->rect.as<uint2>(), b->sc.as<uint32_t>(), b->pair_part.p,
                               nullptr, ctx->d_status, s);
            launch_super_scan(n, order, b->sc.as<uint32_t>(), b->scs.as<uint32_t>(), b->scan_sums.as<uint32_t>(),
                              b->scount.as<uint32_t>() + v, s);
            k_clamp_count<<<1, 1, 0, s>>>(b->scount.as<uint32_t>() + v, (uint32_t)b->scap[v], ents, ctx->d_status);
            count_launch();
        }
        uint32_t *pk = b->pair_k.as<uint32_t>() + b->cap_off[v], *pv = b->pair_v.as<uint32_t>() + b->cap_off[v];
        uint32_t *tk = b->tmp_k.as<uint32_t>(), *tv = b->tmp_v.as<uint32_t>(), *tv2 = b->tmp2_v.as<uint32_t>();
        {
            Stage t(ctx->prof, SPLASH_STAGE_EMIT, s);
            launch_emit_super(n, order, b->scs.as<uint32_t>(), b->scan_sums.as<uint32_t>(), b->rect.as<uint2>(), nsx, sbits,
                              tk, tv, (uint64_t)b->scap[v], ctx->d_status, s);
        }
        const uint32_t *skeys = tk, *svals = tv;
        // a one-pass super-tile sort's digit offsets are the super-tile list starts
        const bool one_pass = b->scap[v] > 0 && digit_plan(sbits).passes == 1;
        {
            Stage t(ctx->prof, SPLASH_STAGE_TILE_SORT, s);
            const int which = sort_pairs(tk, tv, pk, tv2, tk, tv, b->scap[v], ents, sbits, ss, ctx->d_status,
                                         ctx->opt.spin_limit, ctx->opt.test_stall_partition, s);
            skeys = which ? tk : pk;
            svals = which ? tv : tv2;
            if (!one_pass) launch_ranges(b->scap[v], ents, skeys, b->sranges.as<uint2>(), nsuper, s, (1u << sbits) - 1u);
        }
        {
            Stage t(ctx->prof, SPLASH_STAGE_RANGES, s);
            const BinningScratch bs = binning_scratch_carve(b->bin_scratch.as<uint32_t>(), b->scap[v], nsuper);
            launch_tile_lists(tg, nsx, sbits, b->scap[v], skeys, svals, b->sranges.as<uint2>(), bs,
                              b->ranges.as<uint2>() + b->tiles_off[v], pv, ctx->d_status, s, (uint32_t)b->cap[v],
                              counts + 2 * v, one_pass ? ss.hist : nullptr, ents);
        }
    }
    // the work queue: every (view, tile), longest list first
    uint32_t *meta = b->item_meta.as<uint32_t>();
    const uint32_t *items = nullptr;
    {
        Stage t(ctx->prof, SPLASH_STAGE_RANGES, s);
        const int blocks = (int)((b->tiles_total + 255) / 256);
        k_build_items<<<blocks, 256, 0, s>>>(b->views.as<BlendView>(), b->tiles_off_dev.as<int64_t>(), (int)V,
                                             b->tiles_total, b->items_k.as<uint32_t>(), b->items_v.as<uint32_t>());
        count_launch();
        const int which = sort_pairs(b->items_k.as<uint32_t>(), b->items_v.as<uint32_t>(), b->items_k1.as<uint32_t>(),
                                     b->items_v1.as<uint32_t>(), b->items_k.as<uint32_t>(), b->items_v.as<uint32_t>(),
                                     b->tiles_total, nullptr, 24, ss, ctx->d_status, ctx->opt.spin_limit,
                                     ctx->opt.test_stall_partition, s);
        items = which ? b->items_v.as<uint32_t>() : b->items_v1.as<uint32_t>();
    }
    {
        Stage t(ctx->prof, SPLASH_STAGE_BLEND_FWD, s);
        SPLASH_CUDA_TRY(cudaMemsetAsync(meta + 1, 0, 4, s));
        launch_blend_fwd_persistent(ctx->opt.tile_w, ctx->opt.tile_h, fwd_batch(ctx->opt), b->views.as<BlendView>(),
                                    items, meta, reinterpret_cast<int *>(meta + 1), medium, b->ctas_fwd, s);
    }
    SPLASH_CUDA_TRY(cudaGetLastError());
    b->has_forward = true;
    return SPLASH_OK;
}

splash_status splash_batch_backward(splash_batch *b, const splash_gaussians *g, const float *medium,
                                    const float *const *dL_dimages, const splash_grads *grads, void *stream)
{
    if (!b || !b->has_forward) return fail(SPLASH_ERR_STATE, "no batch forward to differentiate");
    splash_status rc;
    if ((rc = check_gaussians(g)) != SPLASH_OK) return rc;
    if (g->n != b->n || g->sh_degree != b->deg) return fail(SPLASH_ERR_INVALID_ARG, "Gaussians differ from the forward");
    if (!medium || !dL_dimages || !grads) return fail(SPLASH_ERR_INVALID_ARG, "null medium, upstream table or grads");
    if (grads->quats && (reinterpret_cast<uintptr_t>(grads->quats) & 15))
        return fail(SPLASH_ERR_INVALID_ARG, "grads.quats must be 16-byte aligned");
    for (int v = 0; v < b->V; v++)
        if (!dL_dimages[v]) return fail(SPLASH_ERR_INVALID_ARG, "null upstream gradient for a view");
    cudaStream_t s = (cudaStream_t)stream;
    splash_ctx *ctx = b->ctx;
    const int64_t n = b->n, V = b->V;
    for (int v = 0; v < V; v++) b->views_host[v].dL_dimage = dL_dimages[v];
    SPLASH_CUDA_TRY(cudaMemcpyAsync(b->views.p, b->views_host, sizeof(BlendView) * V, cudaMemcpyHostToDevice, s));
    SPLASH_CUDA_TRY(cudaMemsetAsync(b->gacc.p, 0, sizeof(GAcc) * (size_t)(V * n), s));
    uint32_t *meta = b->item_meta.as<uint32_t>();
    // the forward's queue order is still in the item buffers
    const int bits_passes = digit_plan(24).passes;
    const uint32_t *items = ((bits_passes - 1) & 1) ? b->items_v.as<uint32_t>() : b->items_v1.as<uint32_t>();
    {
        Stage t(ctx->prof, SPLASH_STAGE_BLEND_BWD, s);
        SPLASH_CUDA_TRY(cudaMemsetAsync(meta + 1, 0, 4, s));
        launch_blend_bwd_persistent(ctx->opt.tile_w, ctx->opt.tile_h, bwd_batch(ctx->opt), b->views.as<BlendView>(),
                                    items, meta, reinterpret_cast<int *>(meta + 1), medium, b->ctas_bwd, s);
    }
    const int nb = preprocess_bwd_multi_blocks(std::max<int64_t>(n, 1));
    {
        Stage t(ctx->prof, SPLASH_STAGE_PREPROCESS_BWD, s);
        SPLASH_CUDA_TRY(cudaMemsetAsync(b->block_med.p, 0, 4 * 9 * (size_t)nb, s));
        launch_preprocess_bwd_multi(n, (int)V, *g, medium, b->views.as<BlendView>(), b->gacc.as<GAcc>(),
                                    b->depth_key.as<uint32_t>(), b->ns, *grads, b->block_med.as<float>(), s);
    }
    if (grads->medium) {
        Stage t(ctx->prof, SPLASH_STAGE_MEDIUM_REDUCE, s);
        launch_medium_reduce(b->tile_med.as<float>(), (int)b->tiles_total, b->block_med.as<float>(), n > 0 ? nb : 0,
                             grads->medium, b->red_scratch.as<float>(), s);
    }
    SPLASH_CUDA_TRY(cudaGetLastError());
    return SPLASH_OK;
}

splash_status splash_batch_pair_counts(const splash_batch *b, int64_t *emitted, int64_t *capacity, void *stream)
{
    if (!b || !b->calibrated || !emitted) return fail(SPLASH_ERR_INVALID_ARG, "bad batch or output");
    std::vector<uint32_t> c(2 * (size_t)b->V);
    SPLASH_CUDA_TRY(cudaMemcpyAsync(c.data(), b->counts.p, 8 * (size_t)b->V, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    SPLASH_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    for (int v = 0; v < b->V; v++) {
        emitted[v] = c[2 * v];
        if (capacity) capacity[v] = b->cap[v];
    }
    return SPLASH_OK;
}

}  // extern "C"
