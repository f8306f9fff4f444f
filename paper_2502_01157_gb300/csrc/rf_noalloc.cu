// rf_noalloc.cu -- a forward render that allocates no device memory at all.
//
// Some callers cannot call cudaMalloc: code that runs where the device
// allocator belongs to someone else (an engine or runtime with its own
// memory pool that forbids outside allocations), or where allocating would
// stall or break a latency-bound loop.  rf_render_fwd needs an rf_scene,
// whose packed copy and start-cell workspace are allocated by
// rf_scene_create.  rf_render_fwd_noalloc instead reads the caller's own
// site / adjacency / attribute arrays directly (the face records are
// recomputed per test with the same FP32 operations the packer uses, so the
// result is bit-identical) and keeps its only scratch -- the per-camera
// nearest-site keys -- in a fixed file-scope device array.
//
// The paper has no counterpart of this entry point; it is an interface
// convenience of this library.
#include <cstring>
#include <mutex>

#include "rf_host.h"

namespace rf {
namespace {

// Scratch shared by every call in the process, on every device that loads
// the library: one 64-bit key per camera.  It keeps the last call's contents;
// each call re-initialises the entries it uses.
constexpr int kNoAllocMaxCams = 64;
__device__ __align__(256) unsigned long long g_noalloc_keys[kNoAllocMaxCams];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long *g_keys_addr[kMaxDevices] = {};

// Device address of g_noalloc_keys on the current device, looked up once per
// device (host code only sees a stand-in symbol, not a device address).
rf_status keys_address(unsigned long long **out) {
    int dev = 0;
    RF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(RF_ERR_INVALID_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_keys_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_keys);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_keys)");
        g_keys_addr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_keys_addr[dev];
    return RF_OK;
}

struct RawScene {
    const float *pos;
    const int32_t *off;
    const int32_t *idx;
    const void *density;
    const void *sh;
    int64_t n_sites, n_edges;
    float box_lo[3], box_hi[3];
};

struct RawParams {
    RawScene s;
    LaunchCams lc;
    const unsigned long long *keys;
    float eps;
    int32_t max_steps;
};

struct NNRaw {
    float o[kMaxCamsPerLaunch][3];
};

__global__ void raw_nearest_site_kernel(const float *__restrict__ pos, int64_t n, NNRaw prm,
                                        unsigned long long *keys) {
    const int c = blockIdx.y;
    const float ox = prm.o[c][0], oy = prm.o[c][1], oz = prm.o[c][2];
    unsigned long long best = ~0ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float dx = __fsub_rn(__ldg(pos + 3 * i), ox);
        const float dy = __fsub_rn(__ldg(pos + 3 * i + 1), oy);
        const float dz = __fsub_rn(__ldg(pos + 3 * i + 2), oz);
        const float dd = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
        const unsigned long long k = ((unsigned long long)__float_as_uint(dd) << 32) | (unsigned long long)i;
        best = k < best ? k : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long q = __shfl_xor_sync(0xffffffffu, best, o);
        best = q < best ? q : best;
    }
    if ((threadIdx.x & 31) == 0 && best != ~0ull) atomicMin(keys + c, best);
}

// Alg. 1 per ray on the caller's CSR arrays; the face record of (i, j) is
// formed on the fly exactly as the packer forms it.  An out-of-range offset
// ends the ray there and an out-of-range neighbour id is skipped, instead of
// being read; this entry point has no per-ray status output, so a malformed
// adjacency silently truncates the affected rays.
template <typename AT, int DEG>
__global__ void __launch_bounds__(kBlock) raw_fwd_kernel(const RawParams p, float *rgb, float *trans,
                                                         float *depth) {
    const PixelTask px = pixel_of_thread(p.lc);
    if (!px.valid) return;
    const rf_camera &cam = p.lc.cam[px.cam];
    float3 o, d;
    camera_ray<true>(cam, px.u, px.v, o, d);
    const int64_t r = p.lc.ray_begin[px.cam] + (int64_t)px.v * cam.width + px.u;
    SceneDev box;
    for (int a = 0; a < 3; ++a) {
        box.box_lo[a] = p.s.box_lo[a];
        box.box_hi[a] = p.s.box_hi[a];
    }
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f, T = 1.f;
    float tmin, tmax;
    if (ray_interval(o, d, box, cam.t_near, cam.t_far, tmin, tmax)) {
        float Y[16];
        sh_basis<DEG>(d, Y);
        int i = (int)(p.keys[p.lc.cam0 + px.cam] & 0xffffffffull);
        float t0 = 0.f;
        int steps = 0;
        while (T > p.eps && steps < p.max_steps) {
            const float xi = __ldg(p.s.pos + 3 * (int64_t)i), yi = __ldg(p.s.pos + 3 * (int64_t)i + 1),
                        zi = __ldg(p.s.pos + 3 * (int64_t)i + 2);
            const int begin = __ldg(p.s.off + i), end = __ldg(p.s.off + i + 1);
            if (begin < 0 || end > p.s.n_edges || begin > end) break;
            const float3 oc = make_float3(__fsub_rn(o.x, xi), __fsub_rn(o.y, yi), __fsub_rn(o.z, zi));
            float nb = 1.f, db = 0.f;
            int jb = -1;
            for (int f = begin; f < end; ++f) {
                const int j = __ldg(p.s.idx + f);
                if ((unsigned)j >= (unsigned)p.s.n_sites) continue;
                const float nx = __fsub_rn(__ldg(p.s.pos + 3 * (int64_t)j), xi);
                const float ny = __fsub_rn(__ldg(p.s.pos + 3 * (int64_t)j + 1), yi);
                const float nz = __fsub_rn(__ldg(p.s.pos + 3 * (int64_t)j + 2), zi);
                const float nn = __fmaf_rn(nx, nx, __fmaf_rn(ny, ny, __fmul_rn(nz, nz)));
                const float s = __fdiv_rn(2.f, nn);
                const float ux = __fmul_rn(nx, s), uy = __fmul_rn(ny, s), uz = __fmul_rn(nz, s);
                const float den = __fmaf_rn(ux, d.x, __fmaf_rn(uy, d.y, __fmul_rn(uz, d.z)));
                const float num = __fmaf_rn(-ux, oc.x, __fmaf_rn(-uy, oc.y, __fmaf_rn(-uz, oc.z, 1.f)));
                if (den > 0.f && __fmul_rn(num, db) < __fmul_rn(nb, den)) {
                    nb = num;
                    db = den;
                    jb = j;
                }
            }
            const float t1 = jb >= 0 ? __fdiv_rn(nb, db) : __int_as_float(0x7f800000);
            const float a = t0 > tmin ? t0 : tmin;
            const float b = t1 < tmax ? t1 : tmax;
            const float wd = __fsub_rn(b, a);
            const float delta = wd > 0.f ? wd : 0.f;
            const float sigma = to_f(__ldg(reinterpret_cast<const AT *>(p.s.density) + i));
            const float e = expf(-__fmul_rn(sigma, delta));
            float pre[3];
            sh_colour<AT, DEG>(reinterpret_cast<const AT *>(p.s.sh), i, Y, pre, false);
            const float w = __fmul_rn(T, __fsub_rn(1.f, e));
            C0 = __fmaf_rn(w, fmaxf(pre[0], 0.f), C0);
            C1 = __fmaf_rn(w, fmaxf(pre[1], 0.f), C1);
            C2 = __fmaf_rn(w, fmaxf(pre[2], 0.f), C2);
            D = __fmaf_rn(w, __fmul_rn(0.5f, __fadd_rn(a, b)), D);
            T = __fmul_rn(T, e);
            ++steps;
            if (jb < 0 || !(t1 < tmax)) break;
            t0 = t1 > t0 ? t1 : t0;
            i = jb;
        }
    }
    rgb[3 * r + 0] = C0;
    rgb[3 * r + 1] = C1;
    rgb[3 * r + 2] = C2;
    trans[r] = T;
    depth[r] = D;
}

template <typename F>
void dispatch_raw(int dtype, int deg, F &&f) {
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

}  // namespace
}  // namespace rf

using namespace rf;

RF_API rf_status rf_render_fwd_noalloc(int64_t n_sites, int64_t n_edges, const float *pos,
                                       const int32_t *adj_off, const int32_t *adj_idx,
                                       const void *density, const void *sh, int32_t sh_degree,
                                       int32_t attr_dtype, const float *aabb6,
                                       const rf_camera *cams, int32_t n_cams,
                                       const rf_render_opts *opts, float *rgb, float *trans,
                                       float *depth, void *stream) {
    if (n_sites < 1 || n_sites >= (1ll << 31) || n_edges < 0 || n_edges >= (1ll << 31))
        return fail(RF_ERR_INVALID_ARG, "n_sites must be in [1, 2^31) and n_edges in [0, 2^31)");
    if (!pos || !adj_off || (n_edges > 0 && !adj_idx) || !density || !sh || !aabb6 || !rgb ||
        !trans || !depth)
        return fail(RF_ERR_INVALID_ARG, "a required pointer is NULL");
    if (sh_degree < 0 || sh_degree > RF_MAX_SH_DEGREE)
        return fail(RF_ERR_INVALID_ARG, "sh_degree %d not in [0, 3]", sh_degree);
    if (attr_dtype != RF_F32 && attr_dtype != RF_BF16 && attr_dtype != RF_F16)
        return fail(RF_ERR_INVALID_ARG, "attr_dtype %d is not RF_F32/RF_BF16/RF_F16", attr_dtype);
    if (((uintptr_t)density & 15) || ((uintptr_t)sh & 15))
        return fail(RF_ERR_INVALID_ARG, "density and sh must be 16-byte aligned");
    if (!cams || n_cams < 1) return fail(RF_ERR_INVALID_ARG, "need at least one camera");
    if (n_cams > kNoAllocMaxCams)
        return fail(RF_ERR_INVALID_ARG,
                    "rf_render_fwd_noalloc renders at most %d cameras per call (got %d); "
                    "split the batch", kNoAllocMaxCams, n_cams);
    for (int a = 0; a < 3; ++a)
        if (!(aabb6[a] <= aabb6[3 + a]))
            return fail(RF_ERR_INVALID_ARG, "aabb6 must hold min[3] <= max[3]");
    for (int c = 0; c < n_cams; ++c) {
        rf_status rc = check_camera(cams[c], c);
        if (rc != RF_OK) return rc;
        if (cams[c].shutter[0] != 0.f || cams[c].shutter[1] != 0.f || cams[c].shutter[2] != 0.f)
            return fail(RF_ERR_INVALID_ARG, "rf_render_fwd_noalloc: camera %d has a rolling shutter, "
                        "which needs a packed scene (rf_render_fwd)", c);
    }
    float eps;
    int32_t max_steps;
    rf_status rc = check_opts(opts, &eps, &max_steps, nullptr);
    if (rc != RF_OK) return rc;
    unsigned long long *keys = nullptr;
    rc = keys_address(&keys);
    if (rc != RF_OK) return rc;

    cudaStream_t st = (cudaStream_t)stream;
    // the keys are minima: they must start at all-ones
    RF_CUDA(cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * n_cams, st));
    RawParams p;
    memset(&p, 0, sizeof p);
    p.s = {pos, adj_off, adj_idx, density, sh, n_sites, n_edges, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < 3; ++a) {
        p.s.box_lo[a] = aabb6[a];
        p.s.box_hi[a] = aabb6[3 + a];
    }
    p.keys = keys;
    p.eps = eps;
    p.max_steps = max_steps;
    int64_t ray_begin = 0;
    for (int first = 0; first < n_cams; first += kMaxCamsPerLaunch) {
        const int count = n_cams - first < kMaxCamsPerLaunch ? n_cams - first : kMaxCamsPerLaunch;
        NNRaw prm;
        memset(&prm, 0, sizeof prm);
        for (int c = 0; c < count; ++c) {
            prm.o[c][0] = cams[first + c].c2w[3];
            prm.o[c][1] = cams[first + c].c2w[7];
            prm.o[c][2] = cams[first + c].c2w[11];
        }
        int64_t blocks = (n_sites + 255) / 256;
        if (blocks > grid_cap(8)) blocks = grid_cap(8);
        raw_nearest_site_kernel<<<dim3((unsigned)blocks, count), 256, 0, st>>>(pos, n_sites, prm, keys + first);
        RF_CUDA(cudaGetLastError());
        const int64_t tiles = make_launch_cams(cams, first, count, ray_begin, &p.lc);
        if (tiles >= (1ll << 31)) return fail(RF_ERR_INVALID_ARG, "too many tiles in one launch");
        p.lc.cam0 = first;
        for (int c = 0; c < count; ++c) ray_begin += (int64_t)cams[first + c].width * cams[first + c].height;
        dispatch_raw(attr_dtype, sh_degree, [&]<typename AT, int DEG>() {
            raw_fwd_kernel<AT, DEG><<<(unsigned)tiles, kBlock, 0, st>>>(p, rgb, trans, depth);
        });
        RF_CUDA(cudaGetLastError());
    }
    return RF_OK;
}
