// Host-side pieces shared by the C ABI translation units: grow-only device
// buffers, stage timing, argument checks, and the context/state objects.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.cuh"

namespace splash_host {

struct Buf {
    void *p = nullptr;
    size_t cap = 0;
    Buf() = default;
    Buf(const Buf &) = delete;
    Buf &operator=(const Buf &) = delete;
    ~Buf() { release(); }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    // grow-only; contents are not preserved
    bool ensure(size_t bytes)
    {
        if (bytes <= cap) return true;
        release();
        const size_t want = std::max<size_t>(bytes + bytes / 4, 256);
        if (cudaMalloc(&p, want) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return false;
        }
        cap = want;
        return true;
    }
    template <class T>
    T *as() const { return static_cast<T *>(p); }
};

// Per-stage CUDA-event timing (tracing aid)
struct Prof {
    bool on = false;
    uint32_t mask = ~0u;  // stages timed while on
    struct Rec {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> spare;
    std::vector<Rec> pending;
    double ms[SPLASH_STAGE_COUNT] = {};
    int64_t cnt[SPLASH_STAGE_COUNT] = {};
    cudaEvent_t take()
    {
        if (!spare.empty()) {
            cudaEvent_t e = spare.back();
            spare.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return e;
    }
    ~Prof()
    {
        for (auto &r : pending) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : spare) cudaEventDestroy(e);
    }
};

// Records a start event on construction and the stop event on destruction.
struct Stage {
    Prof &p;
    int stage;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    Stage(Prof &p_, int stage_, cudaStream_t s_) : p(p_), stage(stage_), s(s_)
    {
        if (p.on && ((p.mask >> stage) & 1u) && (a = p.take())) cudaEventRecord(a, s);
    }
    ~Stage()
    {
        if (!a) return;
        cudaEvent_t b = p.take();
        if (!b) {
            p.spare.push_back(a);
            return;
        }
        cudaEventRecord(b, s);
        p.pending.push_back({stage, a, b});
    }
};

inline splash_status fail(splash_status s, const std::string &msg)
{
    splash_set_error(msg);
    return s;
}

inline bool valid_tile(int tw, int th) { return (tw == 16 && th == 16) || (tw == 8 && th == 32) || (tw == 32 && th == 8); }

inline splash::CamK make_cam(const splash_camera &c)
{
    splash::CamK k{};
    for (int r = 0; r < 3; r++) {
        for (int j = 0; j < 3; j++) k.R[3 * r + j] = c.world_to_cam[4 * r + j];
        k.t[r] = c.world_to_cam[4 * r + 3];
    }
    for (int j = 0; j < 3; j++)
        k.cpos[j] = (float)-((double)k.R[j] * k.t[0] + (double)k.R[3 + j] * k.t[1] + (double)k.R[6 + j] * k.t[2]);
    k.fx = c.fx;
    k.fy = c.fy;
    k.cx = c.cx;
    k.cy = c.cy;
    k.limx = (float)(1.3 * 0.5 * c.width / c.fx);
    k.limy = (float)(1.3 * 0.5 * c.height / c.fy);
    k.znear = c.z_near;
    k.zfar = c.z_far;
    k.W = c.width;
    k.H = c.height;
    return k;
}

inline splash_status check_camera(const splash_camera *cam)
{
    if (!cam) return fail(SPLASH_ERR_INVALID_ARG, "null camera");
    if (cam->width <= 0 || cam->height <= 0 || cam->width > 32768 || cam->height > 32768)
        return fail(SPLASH_ERR_INVALID_ARG, "image size must be in 1..32768");
    if (!(cam->fx > 0.f) || !(cam->fy > 0.f)) return fail(SPLASH_ERR_INVALID_ARG, "focal lengths must be positive");
    if (!(cam->z_near > 0.f) || !(cam->z_far > cam->z_near))
        return fail(SPLASH_ERR_INVALID_ARG, "need 0 < z_near < z_far");
    return SPLASH_OK;
}

inline splash_status check_gaussians(const splash_gaussians *g)
{
    if (!g) return fail(SPLASH_ERR_INVALID_ARG, "null gaussians");
    if (g->n < 0 || g->n >= (int64_t)1 << 31) return fail(SPLASH_ERR_INVALID_ARG, "n must be in [0, 2^31)");
    if (g->sh_degree < 0 || g->sh_degree > 3) return fail(SPLASH_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
        return fail(SPLASH_ERR_INVALID_ARG, "null gaussian buffer");
    if (g->n > 0 && (reinterpret_cast<uintptr_t>(g->quats) & 15))
        return fail(SPLASH_ERR_INVALID_ARG, "quats must be 16-byte aligned");
    return SPLASH_OK;
}

inline int bits_for(int64_t count)
{
    int b = 0;
    while (((int64_t)1 << b) < count) b++;
    return b;
}

}  // namespace splash_host

#define ENSURE(buf, bytes)                                                                                \
    do {                                                                                                  \
        if (!(buf).ensure(bytes)) return splash_host::fail(SPLASH_ERR_OOM, "cudaMalloc failed for " #buf); \
    } while (0)

// Gaussians staged in shared memory per blend step: an explicit option
// applies to both passes; 0 picks each pass's measured best on the 1.5M
// training workload (forward 64, backward 128)
inline int fwd_batch(const splash_options &o) { return o.gaussian_batch ? o.gaussian_batch : 64; }
inline int bwd_batch(const splash_options &o) { return o.gaussian_batch ? o.gaussian_batch : 128; }

struct splash_ctx {
    splash_options opt;
    uint32_t *d_status = nullptr;  // kernel-reported error bits
    splash_host::Prof prof;
    splash_host::Buf feat_counts;  // featuriser histogram counters (kept zero between calls)
    splash_host::Buf bs_scratch;   // backscatter estimate: counters, keys, clusters, kept list, resized maps
    splash_host::Buf zero16;       // 16 zeros: the medium of the pixel form's inner render
    // densification plan: output counts, actions, output offsets (for dens_n Gaussians)
    splash_host::Buf dens_count, dens_action, dens_off, dens_iota, dens_sums, dens_total;
    int64_t dens_n = -1;
    // MCMC relocation: running sum of the weights, chunk sums, sources, draw counts
    splash_host::Buf mcmc_c, mcmc_sums, mcmc_src, mcmc_cnt;
};

struct splash_state {
    splash_ctx *ctx = nullptr;
    // per Gaussian
    // (scs: the super-tile counts in depth order; scan_sums: the emit blocks' offsets)
    splash_host::Buf rec, depth_key, tt, rect, dk0, dv0, dk1, dv1, scs, scan_sums;
    // per (tile, Gaussian) pair (the two-level binning uses them for its
    // super-tile entries and the tile lists)
    splash_host::Buf tk0, tv0, tk1, tv1;
    splash_host::Buf ranges, sort_scratch;
    // two-level binning: per-Gaussian super-tile counts, super-tile list
    // ranges, chunk map / chunk counts / tile counts
    splash_host::Buf sc, sranges, bin_scratch;
    // the sorted tile ids rebuilt from the ranges on request (state queries)
    mutable splash_host::Buf tid_lazy;
    mutable bool tid_lazy_ok = false;
    // per pixel
    splash_host::Buf fT, aA, zh, nlast, nwalk;
    // per tile: the forward's largest walk bound; the backward's CTA order
    splash_host::Buf tile_walk, tile_order;
    // backward
    splash_host::Buf gacc, tile_med, block_med, gmed, red_scratch;
    // loss / standalone sort
    splash_host::Buf loss_scratch, tmp_k, tmp_v;
    // pixel form of the water (Eq. 5): J, the zero-medium upstream, per-block medium sums
    splash_host::Buf pixJ, pixG, pixgz, pixmed;
    bool pixel_forward = false;  // the last forward was splash_render_forward_pixel
    splash_host::Buf small;       // [0] = pair count K, [1..] spare
    splash_host::Buf pair_part;   // the pair-count sum's partials and ticket (kept zero between calls)
    // mapped pinned words [status, K, K_s, spare] that the pair-count kernel
    // stores (host and device addresses); k_ready follows that kernel in the stream
    uint64_t *h_small = nullptr, *h_small_dev = nullptr;
    cudaEvent_t k_ready = nullptr;
    bool gacc_cleared = false;  // the last forward blend zeroed gacc[0..gacc_clear_n)
    const void *gacc_clear_ptr = nullptr;
    int64_t gacc_clear_n = 0;
    // what the last forward produced
    bool has_forward = false;
    int64_t n = 0;
    int W = 0, H = 0;
    splash::TileGeom tg{};
    int64_t K = 0;
    int64_t Ks = 0;  // super-tile entries of the two-level binning
    const uint32_t *order = nullptr;     // depth-sorted Gaussian indices
    const uint32_t *tile_ids = nullptr;  // sorted pairs
    const uint32_t *gauss_ids = nullptr;
};

// splash_render_backward without its check that the last forward was not the
// pixel form (the pixel form's own backward runs it on the zero-medium render)
splash_status render_backward_impl(splash_ctx *ctx, splash_state *st, const splash_gaussians *g,
                                   const float *medium, const splash_camera *cam, const float *dL_dimage,
                                   const float *dL_ddepth, const float *dL_ddepth01, const splash_grads *grads,
                                   void *stream);

// splash_render_backward_adam with the medium its chain sees given explicitly
// (the pixel form passes zeros) and, when pixel_partials is set, the medium
// gradient taken from those per-block sums instead of the segment terms
splash_status backward_adam_impl(splash_ctx *ctx, splash_state *st, const splash_param_buffers *params, int64_t n,
                                 int32_t sh_degree, const splash_camera *cam, const float *dL_dimage,
                                 const float *dL_ddepth, const float *dL_ddepth01, const splash_adam_config *adam,
                                 float *grad_medium, void *stream, const float *chain_medium,
                                 const float *pixel_partials, int pixel_blocks);
