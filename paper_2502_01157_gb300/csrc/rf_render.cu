// rf_render.cu -- forward, backward and trace kernels of the Radiant Foam
// renderer (arXiv 2502.01157) for sm_103a, and their C-ABI entry points.
//
// One thread per ray.  A block renders a 16x8 pixel tile of one camera; each
// warp owns an 8x4 patch, so the rays of a warp enter mostly the same cells
// and their 16-byte face loads hit the same L1 lines.  Tiles of all cameras
// of a call form one grid (multi-camera batches are one launch).
#include <cstring>

#include "rf_host.h"

namespace rf {

struct FwdOut {
    float *rgb;
    float *trans;
    float *depth;
    int32_t *steps;
    uint8_t *status;
    int32_t *trace;     // [R][max_trace] or null
    int32_t max_trace;
};

// Forward: Alg. 1 per ray with Eq. (3)-(4) compositing.
template <typename AT, int DEG, bool TRACE>
__global__ void __launch_bounds__(kBlock) fwd_kernel(const RenderParams p, const FwdOut out) {
    const PixelTask px = pixel_of_thread(p.lc);
    if (!px.valid) return;
    const rf_camera &cam = p.lc.cam[px.cam];
    float3 o, d;
    camera_ray(cam, px.u, px.v, o, d);
    const int64_t r = p.lc.ray_begin[px.cam] + (int64_t)px.v * cam.width + px.u;

    float C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f, T = 1.f;
    int steps = 0;
    uint8_t st = RF_RAY_OK;
    float tmin, tmax;
    if (ray_interval(o, d, p.s, cam.t_near, cam.t_far, tmin, tmax)) {
        float Y[16];
        sh_basis<DEG>(d, Y);
        int i = (int)(p.start_keys[p.lc.cam0 + px.cam] & 0xffffffffull);
        float t0 = 0.f;
        while (T > p.eps) {
            if (steps >= p.max_steps) {
                st = RF_RAY_MAX_STEPS;
                break;
            }
            const float4 cell = ldg(p.s.cells + i);
            Segment g;
            float3 oc;
            cell_step<AT, DEG>(p.s, i, cell, o, d, t0, tmin, tmax, Y, g, oc);
            if (TRACE && steps < out.max_trace) out.trace[r * out.max_trace + steps] = i;
            const float alpha = __fsub_rn(1.f, g.e);
            const float w = __fmul_rn(T, alpha);
            C0 = __fmaf_rn(w, fmaxf(g.pre[0], 0.f), C0);
            C1 = __fmaf_rn(w, fmaxf(g.pre[1], 0.f), C1);
            C2 = __fmaf_rn(w, fmaxf(g.pre[2], 0.f), C2);
            D = __fmaf_rn(w, __fmul_rn(0.5f, __fadd_rn(g.a, g.b)), D);
            T = __fmul_rn(T, g.e);
            ++steps;
            if (g.next < 0 || !(g.t1 < tmax)) break;
            t0 = g.t1 > t0 ? g.t1 : t0;
            i = g.next;
        }
    }
    if (TRACE) {
        for (int k = steps; k < out.max_trace; ++k) out.trace[r * out.max_trace + k] = -1;
        out.steps[r] = steps;
        return;
    }
    out.rgb[3 * r + 0] = C0;
    out.rgb[3 * r + 1] = C1;
    out.rgb[3 * r + 2] = C2;
    out.trans[r] = T;
    out.depth[r] = D;
    if (out.steps) out.steps[r] = steps;
    if (out.status) out.status[r] = st;
}

struct BwdIO {
    const float *rgb, *trans, *depth;
    const float *d_rgb, *d_trans, *d_depth;
    float *g_density, *g_sh, *g_pos;
    int32_t sh_vec;  // g_sh rows may use 16-byte atomics
};

// Position gradient of one crossing of the bisector of (p_a, p_b) at t:
// dt/dp_b = (p_b - x)/den, dt/dp_a = (x - p_a)/den with x = o + t d,
// den = (p_b - p_a).d; oca = o - p_a.
__device__ __forceinline__ void scatter_crossing(float *__restrict__ g_pos, int ia, const float3 &xa,
                                                 const float3 &oca, int ib, const float3 &xb,
                                                 float t, const float3 &d, float adj) {
    if (!g_pos || adj == 0.f) return;
    const float nx = xb.x - xa.x, ny = xb.y - xa.y, nz = xb.z - xa.z;
    const float den = nx * d.x + ny * d.y + nz * d.z;
    const float px = oca.x + t * d.x, py = oca.y + t * d.y, pz = oca.z + t * d.z;  // x - p_a
    const float s = adj / den;
    atomicAdd(g_pos + 3 * (int64_t)ia + 0, s * px);
    atomicAdd(g_pos + 3 * (int64_t)ia + 1, s * py);
    atomicAdd(g_pos + 3 * (int64_t)ia + 2, s * pz);
    atomicAdd(g_pos + 3 * (int64_t)ib + 0, s * (nx - px));
    atomicAdd(g_pos + 3 * (int64_t)ib + 1, s * (ny - py));
    atomicAdd(g_pos + 3 * (int64_t)ib + 2, s * (nz - pz));
}

template <int DEG>
__device__ __forceinline__ void scatter_sh(float *__restrict__ g_sh, int i, const float *cb,
                                           const float *Y, bool vec) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int NV = 3 * K;
    float *row = g_sh + (size_t)i * NV;
    if constexpr (NV % 4 == 0) {
        if (vec) {
#pragma unroll
            for (int q = 0; q < NV / 4; ++q) {
                float4 v;
                v.x = cb[(4 * q + 0) % 3] * Y[(4 * q + 0) / 3];
                v.y = cb[(4 * q + 1) % 3] * Y[(4 * q + 1) / 3];
                v.z = cb[(4 * q + 2) % 3] * Y[(4 * q + 2) / 3];
                v.w = cb[(4 * q + 3) % 3] * Y[(4 * q + 3) / 3];
                atomicAdd(reinterpret_cast<float4 *>(row) + q, v);
            }
            return;
        }
    }
#pragma unroll
    for (int g = 0; g < NV; ++g)
        if (cb[g % 3] != 0.f) atomicAdd(row + g, cb[g % 3] * Y[g / 3]);
}

// Backward: the walk of the forward is repeated with identical arithmetic;
// per segment the adjoints follow from the stored final colour, transmittance
// and depth (C_rest = C_final - C_incl), and are scattered with atomics.
template <typename AT, int DEG>
__global__ void __launch_bounds__(kBlock) bwd_kernel(const RenderParams p, const BwdIO io) {
    const PixelTask px = pixel_of_thread(p.lc);
    if (!px.valid) return;
    const rf_camera &cam = p.lc.cam[px.cam];
    float3 o, d;
    camera_ray(cam, px.u, px.v, o, d);
    const int64_t r = p.lc.ray_begin[px.cam] + (int64_t)px.v * cam.width + px.u;
    float tmin, tmax;
    if (!ray_interval(o, d, p.s, cam.t_near, cam.t_far, tmin, tmax)) return;

    const float gC[3] = {io.d_rgb[3 * r], io.d_rgb[3 * r + 1], io.d_rgb[3 * r + 2]};
    const float gT = io.d_trans ? io.d_trans[r] : 0.f;
    const float gD = io.d_depth ? io.d_depth[r] : 0.f;
    if (gC[0] == 0.f && gC[1] == 0.f && gC[2] == 0.f && gT == 0.f && gD == 0.f) return;
    const float Cf[3] = {io.rgb[3 * r], io.rgb[3 * r + 1], io.rgb[3 * r + 2]};
    const float Tf = io.trans[r];
    const float Df = io.depth ? io.depth[r] : 0.f;

    float Y[16];
    sh_basis<DEG>(d, Y);
    int i = (int)(p.start_keys[p.lc.cam0 + px.cam] & 0xffffffffull);
    float t0 = 0.f, T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
    int steps = 0;
    // the crossing that led into the current cell (scattered one step late,
    // once the t0 adjoint of the next segment is known)
    bool pend = false, pend_defines = false;
    int pa = 0, pb = 0;
    float3 pxa = make_float3(0.f, 0.f, 0.f), poca = pxa;
    float pt = 0.f, padj = 0.f;
    // the crossing that set the current t0 (t0 <- max(t0, t1))
    int da = -1, db = -1;
    float dt = 0.f;

    while (T > p.eps) {
        if (steps >= p.max_steps) break;
        const float4 cell = ldg(p.s.cells + i);
        Segment g;
        float3 oc;
        cell_step<AT, DEG>(p.s, i, cell, o, d, t0, tmin, tmax, Y, g, oc);
        const float alpha = __fsub_rn(1.f, g.e);
        const float w = __fmul_rn(T, alpha);
        const float c[3] = {fmaxf(g.pre[0], 0.f), fmaxf(g.pre[1], 0.f), fmaxf(g.pre[2], 0.f)};
        const float z = __fmul_rn(0.5f, __fadd_rn(g.a, g.b));
        C0 = __fmaf_rn(w, c[0], C0);
        C1 = __fmaf_rn(w, c[1], C1);
        C2 = __fmaf_rn(w, c[2], C2);
        D = __fmaf_rn(w, z, D);
        const float Tn = __fmul_rn(T, g.e);
        // dL/dsigma_n = delta_n * B, dL/ddelta_n = sigma_n * B with
        // B = g_C.(T_{n+1} c_n - C_rest) - g_T T_final + g_D (T_{n+1} z_n - D_rest)
        const float B = gC[0] * (Tn * c[0] - (Cf[0] - C0)) + gC[1] * (Tn * c[1] - (Cf[1] - C1)) +
                        gC[2] * (Tn * c[2] - (Cf[2] - C2)) - gT * Tf + gD * (Tn * z - (Df - D));
        if (io.g_density) atomicAdd(io.g_density + i, g.delta * B);
        if (io.g_sh) {
            const float cb[3] = {g.pre[0] > 0.f ? gC[0] * w : 0.f, g.pre[1] > 0.f ? gC[1] * w : 0.f,
                                 g.pre[2] > 0.f ? gC[2] * w : 0.f};
            if (cb[0] != 0.f || cb[1] != 0.f || cb[2] != 0.f) scatter_sh<DEG>(io.g_sh, i, cb, Y, io.sh_vec);
        }
        // segment bounds: delta = max(b - a, 0), z = (a + b)/2,
        // a = max(t0, t_min), b = min(t1, t_max)
        const float dbar = g.sigma * B;
        float abar = 0.5f * gD * w, bbar = abar;
        if (g.b > g.a) {
            bbar += dbar;
            abar -= dbar;
        }
        const float t1bar = g.t1 < tmax ? bbar : 0.f;
        const float t0bar = t0 > tmin ? abar : 0.f;
        const float3 xi = make_float3(cell.x, cell.y, cell.z);
        if (pend) {
            if (pend_defines) {
                padj += t0bar;
            } else if (da >= 0 && t0bar != 0.f) {
                const float4 ca = ldg(p.s.cells + da), cbb = ldg(p.s.cells + db);
                const float3 xa = make_float3(ca.x, ca.y, ca.z);
                scatter_crossing(io.g_pos, da, xa,
                                 make_float3(__fsub_rn(o.x, xa.x), __fsub_rn(o.y, xa.y), __fsub_rn(o.z, xa.z)),
                                 db, make_float3(cbb.x, cbb.y, cbb.z), dt, d, t0bar);
            }
            scatter_crossing(io.g_pos, pa, pxa, poca, i, xi, pt, d, padj);
        }
        pend = g.next >= 0;
        pa = i;
        pb = g.next;
        pxa = xi;
        poca = oc;
        pt = g.t1;
        padj = t1bar;
        pend_defines = g.t1 >= t0;
        if (pend && pend_defines) {
            da = i;
            db = g.next;
            dt = g.t1;
        }
        T = Tn;
        ++steps;
        if (g.next < 0 || !(g.t1 < tmax)) {
            pend = false;
            break;
        }
        t0 = g.t1 > t0 ? g.t1 : t0;
        i = g.next;
    }
    // stopped by T <= eps or the step cap right after a crossing
    if (pend && padj != 0.f) {
        const float4 cb = ldg(p.s.cells + pb);
        scatter_crossing(io.g_pos, pa, pxa, poca, pb, make_float3(cb.x, cb.y, cb.z), pt, d, padj);
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

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <typename AT, int DEG>
static void launch_fwd(bool trace, int64_t tiles, const RenderParams &p, const FwdOut &o, cudaStream_t st) {
    if (trace) fwd_kernel<AT, DEG, true><<<(unsigned)tiles, kBlock, 0, st>>>(p, o);
    else fwd_kernel<AT, DEG, false><<<(unsigned)tiles, kBlock, 0, st>>>(p, o);
}

template <typename AT, int DEG>
static void launch_bwd(int64_t tiles, const RenderParams &p, const BwdIO &io, cudaStream_t st) {
    bwd_kernel<AT, DEG><<<(unsigned)tiles, kBlock, 0, st>>>(p, io);
}

template <typename F>
static void dispatch(int dtype, int deg, F &&f) {
    auto by_deg = [&](auto tag) {
        using AT = decltype(tag);
        switch (deg) {
            case 0: f.template operator()<AT, 0>(); break;
            case 1: f.template operator()<AT, 1>(); break;
            case 2: f.template operator()<AT, 2>(); break;
            default: f.template operator()<AT, 3>(); break;
        }
    };
    if (dtype == RF_BF16) by_deg(__nv_bfloat16());
    else if (dtype == RF_F16) by_deg(__half());
    else by_deg(float());
}

static rf_status common_checks(const rf_scene *s, const rf_camera *cams, int32_t n_cams,
                               const rf_render_opts *opts, float *eps, int32_t *max_steps) {
    if (!s) return fail(RF_ERR_INVALID_ARG, "scene is NULL");
    if (!cams || n_cams < 1) return fail(RF_ERR_INVALID_ARG, "need at least one camera");
    for (int c = 0; c < n_cams; ++c) {
        rf_status rc = check_camera(cams[c], c);
        if (rc != RF_OK) return rc;
    }
    int64_t rays = 0;
    for (int c = 0; c < n_cams; ++c) rays += (int64_t)cams[c].width * cams[c].height;
    if (rays >= (1ll << 40)) return fail(RF_ERR_INVALID_ARG, "too many rays");
    return check_opts(opts, eps, max_steps);
}

}  // namespace rf

using namespace rf;

static rf_status render_fwd_impl(rf_scene *s, const rf_camera *cams, int32_t n_cams,
                                 const rf_render_opts *opts, FwdOut out, bool trace, void *stream) {
    float eps;
    int32_t max_steps;
    rf_status rc = common_checks(s, cams, n_cams, opts, &eps, &max_steps);
    if (rc != RF_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    RenderParams p;
    memset(&p, 0, sizeof p);
    p.s = scene_dev(s);
    p.start_keys = s->start_keys;
    p.eps = eps;
    p.max_steps = max_steps;
    int64_t ray_begin = 0;
    for (int first = 0; first < n_cams; first += kMaxCamsPerLaunch) {
        const int count = n_cams - first < kMaxCamsPerLaunch ? n_cams - first : kMaxCamsPerLaunch;
        rc = launch_nearest_sites(s, cams + first, count, s->start_keys, st);
        if (rc != RF_OK) return rc;
        const int64_t tiles = make_launch_cams(cams, first, count, ray_begin, &p.lc);
        if (tiles >= (1ll << 31)) return fail(RF_ERR_INVALID_ARG, "too many tiles in one launch");
        for (int c = 0; c < count; ++c) ray_begin += (int64_t)cams[first + c].width * cams[first + c].height;
        dispatch(s->attr_dtype, s->sh_degree, [&]<typename AT, int DEG>() {
            launch_fwd<AT, DEG>(trace, tiles, p, out, st);
        });
        RF_CUDA(cudaGetLastError());
    }
    return RF_OK;
}

RF_API rf_status rf_render_fwd(rf_scene *s, const rf_camera *cams, int32_t n_cams,
                               const rf_render_opts *opts, float *rgb, float *trans, float *depth,
                               int32_t *steps, uint8_t *ray_status, void *stream) {
    if (!rgb || !trans || !depth) return fail(RF_ERR_INVALID_ARG, "rgb, trans and depth are required");
    FwdOut out = {rgb, trans, depth, steps, ray_status, nullptr, 0};
    return render_fwd_impl(s, cams, n_cams, opts, out, false, stream);
}

RF_API rf_status rf_trace_cells(rf_scene *s, const rf_camera *cam, const rf_render_opts *opts,
                                int32_t max_per_ray, int32_t *cells, int32_t *counts, void *stream) {
    if (!cells || !counts || max_per_ray < 1)
        return fail(RF_ERR_INVALID_ARG, "cells, counts and max_per_ray >= 1 are required");
    FwdOut out = {nullptr, nullptr, nullptr, counts, nullptr, cells, max_per_ray};
    return render_fwd_impl(s, cam, 1, opts, out, true, stream);
}

RF_API rf_status rf_render_bwd(rf_scene *s, const rf_camera *cams, int32_t n_cams,
                               const rf_render_opts *opts, const float *rgb, const float *trans,
                               const float *depth, const float *d_rgb, const float *d_trans,
                               const float *d_depth, float *g_density, float *g_sh, float *g_pos,
                               void *stream) {
    float eps;
    int32_t max_steps;
    rf_status rc = common_checks(s, cams, n_cams, opts, &eps, &max_steps);
    if (rc != RF_OK) return rc;
    if (!rgb || !trans || !d_rgb) return fail(RF_ERR_INVALID_ARG, "rgb, trans and d_rgb are required");
    if (d_depth && !depth) return fail(RF_ERR_INVALID_ARG, "depth is required with d_depth");
    if (!g_density && !g_sh && !g_pos) return RF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    BwdIO io = {rgb, trans, depth, d_rgb, d_trans, d_depth, g_density, g_sh, g_pos,
                (int32_t)(((uintptr_t)g_sh & 15) == 0)};
    RenderParams p;
    memset(&p, 0, sizeof p);
    p.s = scene_dev(s);
    p.start_keys = s->start_keys;
    p.eps = eps;
    p.max_steps = max_steps;
    int64_t ray_begin = 0;
    for (int first = 0; first < n_cams; first += kMaxCamsPerLaunch) {
        const int count = n_cams - first < kMaxCamsPerLaunch ? n_cams - first : kMaxCamsPerLaunch;
        rc = launch_nearest_sites(s, cams + first, count, s->start_keys, st);
        if (rc != RF_OK) return rc;
        const int64_t tiles = make_launch_cams(cams, first, count, ray_begin, &p.lc);
        if (tiles >= (1ll << 31)) return fail(RF_ERR_INVALID_ARG, "too many tiles in one launch");
        for (int c = 0; c < count; ++c) ray_begin += (int64_t)cams[first + c].width * cams[first + c].height;
        dispatch(s->attr_dtype, s->sh_degree, [&]<typename AT, int DEG>() {
            launch_bwd<AT, DEG>(tiles, p, io, st);
        });
        RF_CUDA(cudaGetLastError());
    }
    return RF_OK;
}

RF_API rf_status rf_mse_grad(const float *rgb, const float *target, int64_t n, float scale,
                             float *d_rgb, float *loss, void *stream) {
    if (!rgb || !target || !d_rgb || n < 0) return fail(RF_ERR_INVALID_ARG, "bad mse arguments");
    if (n == 0) return RF_OK;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    mse_grad_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(rgb, target, n, scale, d_rgb, loss);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}
