// rf_render.cu -- C-ABI entry points of the Radiant Foam renderer (arXiv
// 2502.01157): forward, backward and trace over a packed scene, and the
// kernels of rf_kernels.cuh instantiated without the sphere effect.
#include <algorithm>
#include <cstring>

#include "rf_kernels.cuh"

namespace rf {

template void launch_fwd_any<false>(int, int, int, int64_t, const RenderParams &, const FwdOut &, cudaStream_t);
template void launch_bwd_any<false, false>(int, int, bool, int64_t, const RenderParams &, const BwdIO &, cudaStream_t);

// The effects kernels run when the launch has a sphere, a fisheye camera or
// a rolling shutter.
static bool needs_fx(const RenderParams &p) {
    if (p.fx.max_bounces > 0) return true;
    for (int c = 0; c < p.lc.n_cams; ++c) {
        const rf_camera &k = p.lc.cam[c];
        if (k.model != RF_CAM_PINHOLE || k.shutter[0] != 0.f || k.shutter[1] != 0.f || k.shutter[2] != 0.f)
            return true;
    }
    return false;
}

static void launch_fwd_fx(const RenderParams &p, int dtype, int deg, int mode, int64_t tiles, const FwdOut &o,
                          cudaStream_t st) {
    if (needs_fx(p)) launch_fwd_any<true>(dtype, deg, mode, tiles, p, o, st);
    else launch_fwd_any<false>(dtype, deg, mode, tiles, p, o, st);
}

static void launch_bwd_fx(const RenderParams &p, int dtype, int deg, bool quant, bool shared, int64_t tiles,
                          const BwdIO &io, cudaStream_t st) {
    if (needs_fx(p)) {
        if (shared) launch_bwd_any<true, true>(dtype, deg, quant, tiles, p, io, st);
        else launch_bwd_any<true, false>(dtype, deg, quant, tiles, p, io, st);
    } else {
        if (shared) launch_bwd_any<false, true>(dtype, deg, quant, tiles, p, io, st);
        else launch_bwd_any<false, false>(dtype, deg, quant, tiles, p, io, st);
    }
}

__global__ void mse_grad_kernel(const float *__restrict__ rgb, const float *__restrict__ target,
                                int64_t n, float scale, float *__restrict__ d_rgb, float *loss) {
    float acc = 0.f;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const float e = rgb[k] - target[k];
        d_rgb[k] = 2.f * scale * e;
        acc += e * e;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, scale * acc);
}

// g_pos[i] += acc[i].xyz, g_density[i] += acc[i].w: the per-site sums the
// backward's vector atomics collected.
__global__ void add_site_grads_kernel(const float4 *__restrict__ acc, int64_t n, float *g_pos, float *g_density) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = acc[i];
        if (g_pos) {
            g_pos[3 * i + 0] += a.x;
            g_pos[3 * i + 1] += a.y;
            g_pos[3 * i + 2] += a.z;
        }
        if (g_density) g_density[i] += a.w;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

// Segment-record bytes of the launch holding cams[first .. first + count):
// per warp of a tile and recorded step, 32 lanes x kRecWords 4-byte words.
static size_t record_bytes_of(const rf_camera *cams, int first, int count, int32_t steps) {
    int64_t tiles = 0;
    for (int c = first; c < first + count; ++c)
        tiles += (int64_t)((cams[c].width + kTileW - 1) / kTileW) * ((cams[c].height + kTileH - 1) / kTileH);
    return (size_t)tiles * (kBlock / 32) * (size_t)steps * 32 * kRecWords * sizeof(uint32_t);
}

static rf_status check_record(const rf_camera *cams, int32_t n_cams, const void *rec, size_t bytes, int32_t steps) {
    if (!rec) return RF_OK;
    if (steps < 1 || steps > (1 << 20)) return fail(RF_ERR_INVALID_ARG, "walk_record_steps must be in [1, 2^20]");
    if ((uintptr_t)rec & 15) return fail(RF_ERR_INVALID_ARG, "walk_record must be 16-byte aligned");
    size_t need = 0;
    for (int first = 0; first < n_cams; first += kMaxCamsPerLaunch)
        need += record_bytes_of(cams, first, std::min(n_cams - first, kMaxCamsPerLaunch), steps);
    if (bytes < need) return fail(RF_ERR_INVALID_ARG, "walk_record holds %zu bytes, needs %zu", bytes, need);
    return RF_OK;
}

static rf_status common_checks(const rf_scene *s, const rf_camera *cams, int32_t n_cams,
                               const rf_render_opts *opts, float *eps, int32_t *max_steps,
                               SphereFx *fx) {
    if (!s) return fail(RF_ERR_INVALID_ARG, "scene is NULL");
    if (!cams || n_cams < 1) return fail(RF_ERR_INVALID_ARG, "need at least one camera");
    for (int c = 0; c < n_cams; ++c) {
        rf_status rc = check_camera(cams[c], c);
        if (rc != RF_OK) return rc;
    }
    int64_t rays = 0;
    for (int c = 0; c < n_cams; ++c) rays += (int64_t)cams[c].width * cams[c].height;
    if (rays >= (1ll << 40)) return fail(RF_ERR_INVALID_ARG, "too many rays");
    return check_opts(opts, eps, max_steps, fx);
}

// Forward render of n <= kMaxCamsPerLaunch cameras whose outputs start at the
// given ray offsets (the serving pool), start cells in keys[0..n).
rf_status launch_fwd_batch(const rf_scene *s, const rf_camera *cams, const int64_t *ray_offsets, int n,
                           float eps, int32_t max_steps, float *rgb, float *trans, float *depth,
                           unsigned long long *keys, cudaStream_t st) {
    if (n < 1 || n > kMaxCamsPerLaunch) return fail(RF_ERR_INVALID_ARG, "batch of %d cameras", n);
    RenderParams p;
    memset(&p, 0, sizeof p);
    p.s = scene_dev(s);
    p.start_keys = keys;
    p.eps = eps;
    p.max_steps = max_steps;
    rf_status rc = launch_nearest_sites(s, cams, n, keys, st);
    if (rc != RF_OK) return rc;
    const int64_t tiles = make_launch_cams(cams, 0, n, 0, &p.lc);
    for (int c = 0; c < n; ++c) p.lc.ray_begin[c] = ray_offsets[c];
    FwdOut out = {rgb, trans, depth, nullptr, nullptr, nullptr, 0, nullptr, nullptr};
    launch_fwd_fx(p, s->attr_dtype, s->sh_degree, kPlain, tiles, out, st);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}

}  // namespace rf

using namespace rf;

static rf_status render_fwd_impl(rf_scene *s, const rf_camera *cams, int32_t n_cams,
                                 const rf_render_opts *opts, FwdOut out, int mode, void *stream,
                                 uint8_t *rec = nullptr, size_t rec_bytes = 0, int32_t rec_steps = 0) {
    float eps;
    int32_t max_steps;
    SphereFx fx;
    rf_status rc = common_checks(s, cams, n_cams, opts, &eps, &max_steps, &fx);
    if (rc != RF_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    RenderParams p;
    memset(&p, 0, sizeof p);
    p.s = scene_dev(s);
    p.start_keys = s->start_keys;
    p.eps = eps;
    p.max_steps = max_steps;
    p.fx = fx;
    if ((rc = check_record(cams, n_cams, rec, rec_bytes, rec_steps)) != RF_OK) return rc;
    p.rec_steps = rec_steps;
    int64_t ray_begin = 0;
    size_t rec_off = 0;
    for (int first = 0; first < n_cams; first += kMaxCamsPerLaunch) {
        const int count = n_cams - first < kMaxCamsPerLaunch ? n_cams - first : kMaxCamsPerLaunch;
        rc = launch_nearest_sites(s, cams + first, count, s->start_keys, st);
        if (rc != RF_OK) return rc;
        const int64_t tiles = make_launch_cams(cams, first, count, ray_begin, &p.lc);
        if (tiles >= (1ll << 31)) return fail(RF_ERR_INVALID_ARG, "too many tiles in one launch");
        for (int c = 0; c < count; ++c) ray_begin += (int64_t)cams[first + c].width * cams[first + c].height;
        p.rec = rec ? reinterpret_cast<uint32_t *>(rec + rec_off) : nullptr;
        if (rec) rec_off += record_bytes_of(cams, first, count, rec_steps);
        launch_fwd_fx(p, s->attr_dtype, s->sh_degree, mode, tiles, out, st);
        RF_CUDA(cudaGetLastError());
    }
    return RF_OK;
}

RF_API rf_status rf_render_fwd_ex(rf_scene *s, const rf_camera *cams, int32_t n_cams,
                                  const rf_render_opts *opts, const rf_fwd_outputs *o, void *stream) {
    if (!o || !o->rgb || !o->trans || !o->depth)
        return fail(RF_ERR_INVALID_ARG, "rgb, trans and depth are required");
    if (o->quantile && !o->quantile_aux)
        return fail(RF_ERR_INVALID_ARG, "quantile_aux is required with quantile");
    FwdOut out = {o->rgb, o->trans, o->depth, o->steps, o->ray_status, nullptr, 0, o->quantile,
                  o->quantile_aux};
    return render_fwd_impl(s, cams, n_cams, opts, out, o->quantile ? kQuant : kPlain, stream, o->walk_record,
                           o->walk_record_bytes, o->walk_record_steps);
}

RF_API rf_status rf_render_fwd(rf_scene *s, const rf_camera *cams, int32_t n_cams,
                               const rf_render_opts *opts, float *rgb, float *trans, float *depth,
                               int32_t *steps, uint8_t *ray_status, void *stream) {
    const rf_fwd_outputs o = {rgb, trans, depth, steps, ray_status, nullptr, nullptr, nullptr, 0, 0};
    return rf_render_fwd_ex(s, cams, n_cams, opts, &o, stream);
}

RF_API rf_status rf_trace_cells(rf_scene *s, const rf_camera *cam, const rf_render_opts *opts,
                                int32_t max_per_ray, int32_t *cells, int32_t *counts, void *stream) {
    if (!cells || !counts || max_per_ray < 1)
        return fail(RF_ERR_INVALID_ARG, "cells, counts and max_per_ray >= 1 are required");
    FwdOut out = {nullptr, nullptr, nullptr, counts, nullptr, cells, max_per_ray, nullptr, nullptr};
    return render_fwd_impl(s, cam, 1, opts, out, kTrace, stream);
}

RF_API rf_status rf_render_bwd_ex(rf_scene *s, const rf_camera *cams, int32_t n_cams,
                                  const rf_render_opts *opts, const rf_bwd_inputs *in,
                                  const rf_grads *gr, void *stream) {
    float eps;
    int32_t max_steps;
    SphereFx fx;
    rf_status rc = common_checks(s, cams, n_cams, opts, &eps, &max_steps, &fx);
    if (rc != RF_OK) return rc;
    if (!in || !gr) return fail(RF_ERR_INVALID_ARG, "inputs and gradients must not be NULL");
    if (!in->rgb || !in->trans || !in->d_rgb) return fail(RF_ERR_INVALID_ARG, "rgb, trans and d_rgb are required");
    if (in->d_depth && !in->depth) return fail(RF_ERR_INVALID_ARG, "depth is required with d_depth");
    if (in->d_quantile && !in->quantile_aux)
        return fail(RF_ERR_INVALID_ARG, "quantile_aux is required with d_quantile");
    if (!gr->density && !gr->sh && !gr->pos) return RF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // the per-site {position, density} sums: a scene-owned workspace of 16
    // bytes per site, allocated by the first backward and zeroed by each
    if ((gr->pos || gr->density) && !s->g_acc) {
        cudaError_t e = cudaMalloc((void **)&s->g_acc, sizeof(float4) * (size_t)s->n_sites);
        if (e != cudaSuccess) {
            s->g_acc = nullptr;
            return e == cudaErrorMemoryAllocation ? fail(RF_ERR_OOM, "backward workspace (%lld bytes)",
                                                         (long long)(sizeof(float4) * s->n_sites))
                                                  : cuda_fail(e, "cudaMalloc(g_acc)");
        }
        s->bytes += sizeof(float4) * (size_t)s->n_sites;
    }
    float4 *acc = (gr->pos || gr->density) ? s->g_acc : nullptr;
    if (acc) RF_CUDA(cudaMemsetAsync(acc, 0, sizeof(float4) * (size_t)s->n_sites, st));
    BwdIO io = {in->rgb, in->trans, in->depth, in->d_rgb, in->d_trans, in->d_depth, gr->density,
                gr->sh, gr->pos, (int32_t)(((uintptr_t)gr->sh & 15) == 0), acc, in->quantile_aux,
                in->d_quantile};
    const bool quant = in->d_quantile != nullptr;
    RenderParams p;
    memset(&p, 0, sizeof p);
    p.s = scene_dev(s);
    p.start_keys = s->start_keys;
    p.eps = eps;
    p.max_steps = max_steps;
    p.fx = fx;
    if ((rc = check_record(cams, n_cams, in->walk_record, in->walk_record_bytes, in->walk_record_steps)) != RF_OK)
        return rc;
    p.rec_steps = in->walk_record_steps;
    int64_t ray_begin = 0;
    size_t rec_off = 0;
    for (int first = 0; first < n_cams; first += kMaxCamsPerLaunch) {
        const int count = n_cams - first < kMaxCamsPerLaunch ? n_cams - first : kMaxCamsPerLaunch;
        rc = launch_nearest_sites(s, cams + first, count, s->start_keys, st);
        if (rc != RF_OK) return rc;
        const int64_t tiles = make_launch_cams(cams, first, count, ray_begin, &p.lc);
        if (tiles >= (1ll << 31)) return fail(RF_ERR_INVALID_ARG, "too many tiles in one launch");
        for (int c = 0; c < count; ++c) ray_begin += (int64_t)cams[first + c].width * cams[first + c].height;
        p.rec = in->walk_record ? reinterpret_cast<uint32_t *>(const_cast<uint8_t *>(in->walk_record) + rec_off)
                                : nullptr;
        if (in->walk_record) rec_off += record_bytes_of(cams, first, count, in->walk_record_steps);
        launch_bwd_fx(p, s->attr_dtype, s->sh_degree, quant, opts && (opts->flags & RF_RENDER_SHARED_CELLS), tiles,
                      io, st);
        RF_CUDA(cudaGetLastError());
    }
    if (acc) {
        const int64_t blocks = std::min<int64_t>((s->n_sites + 255) / 256, grid_cap(8));
        add_site_grads_kernel<<<(unsigned)blocks, 256, 0, st>>>(acc, s->n_sites, gr->pos, gr->density);
        RF_CUDA(cudaGetLastError());
    }
    return RF_OK;
}

RF_API rf_status rf_render_bwd(rf_scene *s, const rf_camera *cams, int32_t n_cams,
                               const rf_render_opts *opts, const float *rgb, const float *trans,
                               const float *depth, const float *d_rgb, const float *d_trans,
                               const float *d_depth, float *g_density, float *g_sh, float *g_pos,
                               void *stream) {
    const rf_bwd_inputs in = {rgb, trans, depth, nullptr, d_rgb, d_trans, d_depth, nullptr, nullptr, 0, 0};
    const rf_grads gr = {g_density, g_sh, g_pos};
    return rf_render_bwd_ex(s, cams, n_cams, opts, &in, &gr, stream);
}

RF_API rf_status rf_mse_grad(const float *rgb, const float *target, int64_t n, float scale,
                             float *d_rgb, float *loss, void *stream) {
    if (!rgb || !target || !d_rgb || n < 0) return fail(RF_ERR_INVALID_ARG, "bad mse arguments");
    if (n == 0) return RF_OK;
    int64_t blocks = (n + 255) / 256;
    if (blocks > grid_cap(8)) blocks = grid_cap(8);
    mse_grad_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(rgb, target, n, scale, d_rgb, loss);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}

RF_API size_t rf_walk_record_bytes(const rf_camera *cams, int32_t n_cams, int32_t steps) {
    if (!cams || n_cams < 1 || steps < 1) return 0;
    size_t need = 0;
    for (int first = 0; first < n_cams; first += kMaxCamsPerLaunch)
        need += record_bytes_of(cams, first, std::min(n_cams - first, kMaxCamsPerLaunch), steps);
    return need;
}
