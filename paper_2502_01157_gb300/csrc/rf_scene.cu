// rf_scene.cu -- scene packing, validation, scene box and nn(o) for the
// Radiant Foam renderer (arXiv 2502.01157), sm_103a.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rf_host.h"

namespace rf {

static thread_local std::string g_error;

rf_status fail(rf_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return code;
}

rf_status cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? RF_ERR_OOM : RF_ERR_CUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

int grid_cap(int per_sm) {
    static std::atomic<int> cached[64] = {};
    int dev = 0;
    int sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
        sms = cached[dev].load(std::memory_order_relaxed);
        if (sms <= 0 && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            cached[dev].store(sms, std::memory_order_relaxed);
    }
    if (sms <= 0) sms = 152;  // the attribute query failed: a GB300's count
    return sms * per_sm;
}

SceneDev scene_dev(const rf_scene *s) {
    SceneDev d;
    d.cells = s->cells;
    d.faces = s->faces;
    d.nbr = s->nbr;
    d.count_bits = s->count_bits;
    d.sh_v8 = s->sh_v8;
    d.n_sites = (int32_t)s->n_sites;
    d.density = s->density;
    d.sh = s->sh;
    for (int a = 0; a < 3; ++a) {
        d.box_lo[a] = s->box[a];
        d.box_hi[a] = s->box[3 + a];
    }
    return d;
}

rf_status check_camera(const rf_camera &c, int index) {
    bool ok = c.width > 0 && c.height > 0 && (int64_t)c.width * c.height < (1ll << 31) &&
              std::isfinite(c.fx) && std::isfinite(c.fy) && c.fx != 0.f && c.fy != 0.f &&
              std::isfinite(c.cx) && std::isfinite(c.cy) && std::isfinite(c.t_near) &&
              !std::isnan(c.t_far) && (c.model == RF_CAM_PINHOLE || c.model == RF_CAM_FISHEYE);
    for (int k = 0; k < 12; ++k) ok = ok && std::isfinite(c.c2w[k]);
    for (int k = 0; k < 3; ++k) ok = ok && std::isfinite(c.shutter[k]);
    if (!ok) return fail(RF_ERR_INVALID_ARG, "camera %d is invalid (size, intrinsics or pose)", index);
    return RF_OK;
}

rf_status check_opts(const rf_render_opts *o, float *eps, int32_t *max_steps, SphereFx *fx) {
    *eps = 1e-4f;
    *max_steps = kDefaultMaxSteps;
    if (fx) memset(fx, 0, sizeof *fx);
    if (o) {
        if (!(o->eps >= 0.f) || !std::isfinite(o->eps))
            return fail(RF_ERR_INVALID_ARG, "opts.eps must be finite and >= 0");
        *eps = o->eps;
        if (o->flags & ~RF_RENDER_SHARED_CELLS) return fail(RF_ERR_INVALID_ARG, "unknown bits in opts.flags");
        if (o->max_steps > 0) *max_steps = o->max_steps;
        if (o->max_bounces < 0) return fail(RF_ERR_INVALID_ARG, "opts.max_bounces must be >= 0");
        if (o->max_bounces > 0) {
            bool ok = o->sphere[3] > 0.f && std::isfinite(o->sphere[3]) && o->sphere_ior >= 0.f &&
                      std::isfinite(o->sphere_ior);
            for (int a = 0; a < 3; ++a) ok = ok && std::isfinite(o->sphere[a]);
            if (!ok) return fail(RF_ERR_INVALID_ARG, "sphere needs a finite centre, radius > 0 and ior >= 0");
            if (!fx) return fail(RF_ERR_INVALID_ARG, "this entry point does not support the sphere");
            *fx = {o->sphere[0], o->sphere[1], o->sphere[2], o->sphere[3], o->sphere_ior, o->max_bounces};
        }
    }
    return RF_OK;
}

int64_t make_launch_cams(const rf_camera *cams, int first, int count, int64_t ray_begin,
                         LaunchCams *lc) {
    memset(lc, 0, sizeof *lc);
    lc->n_cams = count;
    lc->cam0 = 0;
    int64_t tiles = 0;
    for (int c = 0; c < count; ++c) {
        const rf_camera &cam = cams[first + c];
        lc->cam[c] = cam;
        lc->tiles_x[c] = (cam.width + kTileW - 1) / kTileW;
        const int ty = (cam.height + kTileH - 1) / kTileH;
        lc->tile_begin[c] = (int32_t)tiles;
        lc->ray_begin[c] = ray_begin;
        tiles += (int64_t)lc->tiles_x[c] * ty;
        ray_begin += (int64_t)cam.width * cam.height;
    }
    lc->tile_begin[count] = (int32_t)tiles;
    return tiles;
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// flags[0]: bad offsets (non-monotone / out of range / wrong ends)
__global__ void validate_offsets_kernel(const int32_t *__restrict__ off, int64_t n, int64_t e,
                                        int32_t *flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && (off[0] != 0 || off[n] != e)) atomicAdd(flags + 0, 1);
    if (i < n) {
        const int32_t a = off[i], b = off[i + 1];
        if (a > b || a < 0 || b > e) atomicAdd(flags + 0, 1);
    }
}

// flags[1]: out-of-range / self neighbours, flags[2]: asymmetric edges,
// flags[3]: zero-length edges (coincident sites).  Offsets already valid.
__global__ void validate_edges_kernel(const int32_t *__restrict__ off,
                                      const int32_t *__restrict__ idx,
                                      const float *__restrict__ pos, int64_t n, int32_t *flags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
    for (int32_t f = off[i]; f < off[i + 1]; ++f) {
        const int32_t j = idx[f];
        if (j < 0 || j >= n || j == i) {
            atomicAdd(flags + 1, 1);
            continue;
        }
        if (pos[3 * (int64_t)j] == xi && pos[3 * (int64_t)j + 1] == yi && pos[3 * (int64_t)j + 2] == zi)
            atomicAdd(flags + 3, 1);
        bool found = false;
        for (int32_t g = off[j]; g < off[j + 1] && !found; ++g) found = idx[g] == (int32_t)i;
        if (!found) atomicAdd(flags + 2, 1);
    }
}

__device__ __forceinline__ float4 face_record(const float *__restrict__ pos, int64_t i, int32_t j) {
    const float nx = __fsub_rn(pos[3 * (int64_t)j], pos[3 * i]);
    const float ny = __fsub_rn(pos[3 * (int64_t)j + 1], pos[3 * i + 1]);
    const float nz = __fsub_rn(pos[3 * (int64_t)j + 2], pos[3 * i + 2]);
    const float nn = __fmaf_rn(nx, nx, __fmaf_rn(ny, ny, __fmul_rn(nz, nz)));
    const float s = __fdiv_rn(2.f, nn);
    return make_float4(__fmul_rn(nx, s), __fmul_rn(ny, s), __fmul_rn(nz, s), __int_as_float(j));
}

// Largest i with off[i] <= f (off monotone, off[0] = 0 <= f).
__device__ __forceinline__ int64_t owner_of(const int32_t *__restrict__ off, int64_t n, int64_t f) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= f) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void store_face(float4 *__restrict__ faces, int32_t *__restrict__ nbr,
                                           int64_t g, int l, const float4 &rec) {
    float *fl = reinterpret_cast<float *>(faces) + 12 * g;
    fl[l] = rec.x;
    fl[4 + l] = rec.y;
    fl[8 + l] = rec.z;
    nbr[4 * g + l] = __float_as_int(rec.w);
}

// One thread per caller edge f of cell i (the k-th neighbour): its u goes to
// lane k % 4 of group goff[i] + k / 4.
__global__ void pack_faces_kernel(const int32_t *__restrict__ off, const int32_t *__restrict__ goff,
                                  const int32_t *__restrict__ idx, const float *__restrict__ pos,
                                  int64_t n, int64_t e, float4 *__restrict__ faces,
                                  int32_t *__restrict__ nbr) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= e) return;
    const int64_t i = owner_of(off, n, f);
    const int64_t k = f - off[i];
    store_face(faces, nbr, (int64_t)goff[i] + k / 4, (int)(k % 4), face_record(pos, i, idx[f]));
}

// Re-pack after the sites moved: one thread per face slot; the neighbour ids
// stay, the geometry is recomputed.
__global__ void repack_faces_kernel(const int32_t *__restrict__ goff, const float *__restrict__ pos,
                                    int64_t n, int64_t groups, float4 *__restrict__ faces,
                                    int32_t *__restrict__ nbr) {
    const int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= 4 * groups) return;
    const int32_t j = nbr[sl];
    if (j < 0) return;  // padding
    const int64_t g = sl / 4;
    store_face(faces, nbr, g, (int)(sl % 4), face_record(pos, owner_of(goff, n, g), j));
}

// Headers and group padding: cell i owns groups [goff[i], goff[i+1]); its
// caller count is off[i+1] - off[i]; the remaining lanes are padding (u = 0).
__global__ void pack_cells_kernel(const int32_t *__restrict__ off, const int32_t *__restrict__ goff,
                                  const float *__restrict__ pos, int64_t n, int count_bits,
                                  float4 *__restrict__ cells, float4 *__restrict__ faces,
                                  int32_t *__restrict__ nbr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t gb = goff[i], ge = goff[i + 1];
    const uint32_t w = ((uint32_t)gb << count_bits) | (uint32_t)(ge - gb);
    cells[i] = make_float4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], __uint_as_float(w));
    for (int64_t k = off[i + 1] - off[i]; k < 4 * (int64_t)(ge - gb); ++k)
        store_face(faces, nbr, gb + k / 4, (int)(k % 4), make_float4(0.f, 0.f, 0.f, __int_as_float(-1)));
}

__global__ void update_cells_kernel(const float *__restrict__ pos, int64_t n, float4 *__restrict__ cells) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 h = cells[i];
    cells[i] = make_float4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], h.w);
}

// Order-preserving map of floats to signed ints for atomic min / max.
__device__ __forceinline__ int float_key(float v) {
    const int b = __float_as_int(v);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__host__ __device__ inline float key_float(int k) {
    const int b = k >= 0 ? k : k ^ 0x7fffffff;
    float v;
    memcpy(&v, &b, sizeof v);
    return v;
}

__global__ void box_kernel(const float *__restrict__ pos, int64_t n, int32_t *keys) {
    int lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int k = float_key(pos[3 * i + a]);
            lo[a] = min(lo[a], k);
            hi[a] = max(hi[a], k);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(keys + a, lo[a]);
            atomicMax(keys + 3 + a, hi[a]);
        }
    }
}

// nn(o) (Alg. 1, initial cell): per camera the minimum over sites of the key
// (bits of |o - p_i|^2 << 32 | i); squared distances are non-negative floats,
// so their bit patterns order like the values, and ties go to the lower index.
struct NNParams {
    float o[kMaxCamsPerLaunch][3];
};

__global__ void nearest_site_kernel(const float4 *__restrict__ cells, int64_t n, NNParams prm,
                                    unsigned long long *keys) {
    const int c = blockIdx.y;
    const float ox = prm.o[c][0], oy = prm.o[c][1], oz = prm.o[c][2];
    unsigned long long best = ~0ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = __ldg(cells + i);
        const float dx = __fsub_rn(p.x, ox), dy = __fsub_rn(p.y, oy), dz = __fsub_rn(p.z, oz);
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

rf_status launch_nearest_sites(const rf_scene *s, const rf_camera *cams, int n,
                               unsigned long long *keys, cudaStream_t st) {
    NNParams prm;
    memset(&prm, 0, sizeof prm);
    for (int c = 0; c < n; ++c) {
        prm.o[c][0] = cams[c].c2w[3];
        prm.o[c][1] = cams[c].c2w[7];
        prm.o[c][2] = cams[c].c2w[11];
    }
    RF_CUDA(cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * n, st));
    const int threads = 256;
    int64_t blocks = (s->n_sites + threads - 1) / threads;
    if (blocks > grid_cap(8)) blocks = grid_cap(8);
    nearest_site_kernel<<<dim3((unsigned)blocks, n), threads, 0, st>>>(s->cells, s->n_sites, prm, keys);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}

}  // namespace rf

using namespace rf;

RF_API int32_t rf_version(void) { return RF_VERSION; }

RF_API const char *rf_last_error(void) { return g_error.c_str(); }

static void free_scene(rf_scene *s) {
    if (!s) return;
    cudaFree(s->cells);
    cudaFree(s->off);
    cudaFree(s->faces);
    cudaFree(s->nbr);
    cudaFree(s->start_keys);
    cudaFree(s->flags);
    cudaFree(s->g_acc);
    delete s;
}

static rf_status check_attr_ptrs(const void *density, const void *sh, int32_t dtype) {
    if (dtype != RF_F32 && dtype != RF_BF16 && dtype != RF_F16)
        return fail(RF_ERR_INVALID_ARG, "attr_dtype %d is not RF_F32/RF_BF16/RF_F16", dtype);
    if (!density || !sh) return fail(RF_ERR_INVALID_ARG, "density and sh must be device pointers");
    if (((uintptr_t)density & 15) || ((uintptr_t)sh & 15))
        return fail(RF_ERR_INVALID_ARG, "density and sh must be 16-byte aligned");
    return RF_OK;
}

RF_API rf_status rf_scene_create(const rf_scene_desc *desc, void *stream, rf_scene **out) {
    if (!desc || !out) return fail(RF_ERR_INVALID_ARG, "desc and out must not be NULL");
    *out = nullptr;
    const int64_t n = desc->n_sites, e = desc->n_edges;
    if (n < 1 || n >= (1ll << 30) || e < 0 || e >= (1ll << 30))
        return fail(RF_ERR_INVALID_ARG, "n_sites must be in [1, 2^30) and n_edges in [0, 2^30)");
    if (!desc->pos || !desc->adj_off || (e > 0 && !desc->adj_idx))
        return fail(RF_ERR_INVALID_ARG, "pos, adj_off and adj_idx must be device pointers");
    if (desc->sh_degree < 0 || desc->sh_degree > RF_MAX_SH_DEGREE)
        return fail(RF_ERR_INVALID_ARG, "sh_degree %d not in [0, 3]", desc->sh_degree);
    rf_status rc = check_attr_ptrs(desc->density, desc->sh, desc->attr_dtype);
    if (rc != RF_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    rf_scene *s = new rf_scene();
    s->n_sites = n;
    s->n_edges = e;
    s->density = desc->density;
    s->sh = desc->sh;
    s->sh_degree = desc->sh_degree;
    s->attr_dtype = desc->attr_dtype;
    s->sh_v8 = ((uintptr_t)desc->sh & 31) == 0;
    cudaGetDevice(&s->device);
#define RF_TRY_ALLOC(ptr, nbytes_)                                 \
    do {                                                           \
        cudaError_t e_ = cudaMalloc((void **)&(ptr), (nbytes_));   \
        if (e_ != cudaSuccess) {                                   \
            free_scene(s);                                         \
            return cuda_fail(e_, "cudaMalloc(" #ptr ")");          \
        }                                                          \
        s->bytes += (nbytes_);                                     \
    } while (0)
    RF_TRY_ALLOC(s->off, sizeof(int32_t) * (n + 1));
    RF_TRY_ALLOC(s->start_keys, sizeof(unsigned long long) * kMaxCamsPerLaunch);
    RF_TRY_ALLOC(s->flags, sizeof(int32_t) * 8);

    auto bail = [&](rf_status r) {
        free_scene(s);
        return r;
    };
    cudaError_t ce;
    if ((ce = cudaMemcpyAsync(s->off, desc->adj_off, sizeof(int32_t) * (n + 1),
                              cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return bail(cuda_fail(ce, "copy adj_off"));
    if ((ce = cudaMemsetAsync(s->flags, 0, sizeof(int32_t) * 8, st)) != cudaSuccess)
        return bail(cuda_fail(ce, "memset flags"));
    const int threads = 256;
    validate_offsets_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(s->off, n, e, s->flags);
    int32_t flags[8];
    if ((ce = cudaMemcpyAsync(flags, s->flags, sizeof flags, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (ce = cudaStreamSynchronize(st)) != cudaSuccess)
        return bail(cuda_fail(ce, "validate offsets"));
    if (flags[0]) return bail(fail(RF_ERR_BAD_SCENE, "adjacency offsets invalid (%d bad entries)", flags[0]));
    validate_edges_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(
        s->off, desc->adj_idx, desc->pos, n, s->flags);
    if ((ce = cudaMemcpyAsync(flags, s->flags, sizeof flags, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (ce = cudaStreamSynchronize(st)) != cudaSuccess)
        return bail(cuda_fail(ce, "validate edges"));
    if (flags[1] || flags[2] || flags[3])
        return bail(fail(RF_ERR_BAD_SCENE,
                         "adjacency invalid: %d out-of-range/self, %d asymmetric, %d zero-length edges",
                         flags[1], flags[2], flags[3]));

    // face groups of four: cell i owns ceil(count / 4) groups; the header
    // packs its first group and group count into 32 bits
    std::vector<int32_t> off_h(n + 1), goff_h(n + 1);
    if ((ce = cudaMemcpyAsync(off_h.data(), s->off, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost,
                              st)) != cudaSuccess ||
        (ce = cudaStreamSynchronize(st)) != cudaSuccess)
        return bail(cuda_fail(ce, "read offsets"));
    int64_t acc = 0, max_g = 0;
    goff_h[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t g = (off_h[i + 1] - off_h[i] + 3) / 4;
        max_g = g > max_g ? g : max_g;
        acc += g;
        goff_h[i + 1] = (int32_t)acc;
    }
    int cb = 4;
    while ((1ll << cb) <= max_g) ++cb;
    if (acc >= (1ll << (32 - cb)))
        return bail(fail(RF_ERR_INVALID_ARG, "adjacency too large for the packed header (%lld groups)",
                         (long long)acc));
    s->count_bits = cb;
    s->n_groups = acc;
    RF_TRY_ALLOC(s->faces, sizeof(float4) * 3 * (acc > 0 ? acc : 1));
    RF_TRY_ALLOC(s->nbr, sizeof(int32_t) * 4 * (acc > 0 ? acc : 1));
    RF_TRY_ALLOC(s->cells, sizeof(float4) * n);
#undef RF_TRY_ALLOC
    if ((ce = cudaMemcpyAsync(s->off, goff_h.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice,
                              st)) != cudaSuccess)
        return bail(cuda_fail(ce, "upload group offsets"));
    if (e > 0) {
        pack_faces_kernel<<<(unsigned)((e + threads - 1) / threads), threads, 0, st>>>(
            desc->adj_off, s->off, desc->adj_idx, desc->pos, n, e, s->faces, s->nbr);
        if ((ce = cudaGetLastError()) != cudaSuccess) return bail(cuda_fail(ce, "pack faces"));
    }
    pack_cells_kernel<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(
        desc->adj_off, s->off, desc->pos, n, cb, s->cells, s->faces, s->nbr);
    if ((ce = cudaGetLastError()) != cudaSuccess) return bail(cuda_fail(ce, "pack cells"));

    bool box_ok = true;
    for (int a = 0; a < 3; ++a) box_ok = box_ok && desc->aabb_min[a] <= desc->aabb_max[a];
    if (box_ok) {
        for (int a = 0; a < 3; ++a) {
            s->box[a] = desc->aabb_min[a];
            s->box[3 + a] = desc->aabb_max[a];
        }
    } else {
        int32_t init[6] = {INT32_MAX, INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN, INT32_MIN};
        int32_t keys[6];
        if ((ce = cudaMemcpyAsync(s->flags, init, sizeof init, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return bail(cuda_fail(ce, "box init"));
        int64_t blocks = (n + threads - 1) / threads;
        if (blocks > grid_cap(4)) blocks = grid_cap(4);
        box_kernel<<<(unsigned)blocks, threads, 0, st>>>(desc->pos, n, s->flags);
        if ((ce = cudaMemcpyAsync(keys, s->flags, sizeof keys, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (ce = cudaStreamSynchronize(st)) != cudaSuccess)
            return bail(cuda_fail(ce, "box"));
        for (int a = 0; a < 6; ++a) s->box[a] = key_float(keys[a]);
    }
    if ((ce = cudaStreamSynchronize(st)) != cudaSuccess) return bail(cuda_fail(ce, "scene create"));
    *out = s;
    return RF_OK;
}

RF_API rf_status rf_scene_set_attributes(rf_scene *s, const void *density, const void *sh,
                                         int32_t attr_dtype) {
    if (!s) return fail(RF_ERR_INVALID_ARG, "scene is NULL");
    rf_status rc = check_attr_ptrs(density, sh, attr_dtype);
    if (rc != RF_OK) return rc;
    s->density = density;
    s->sh = sh;
    s->attr_dtype = attr_dtype;
    s->sh_v8 = ((uintptr_t)sh & 31) == 0;
    return RF_OK;
}

RF_API rf_status rf_scene_update_positions(rf_scene *s, const float *pos, void *stream) {
    if (!s || !pos) return fail(RF_ERR_INVALID_ARG, "scene and pos must not be NULL");
    // the face records hold the neighbour ids; only the geometry is recomputed
    const int threads = 256;
    cudaStream_t st = (cudaStream_t)stream;
    if (s->n_groups > 0) {
        repack_faces_kernel<<<(unsigned)((4 * s->n_groups + threads - 1) / threads), threads, 0, st>>>(
            s->off, pos, s->n_sites, s->n_groups, s->faces, s->nbr);
        RF_CUDA(cudaGetLastError());
    }
    update_cells_kernel<<<(unsigned)((s->n_sites + threads - 1) / threads), threads, 0, st>>>(
        pos, s->n_sites, s->cells);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}

RF_API rf_status rf_scene_info(const rf_scene *s, int64_t *n_sites, int64_t *n_edges, float *aabb6,
                               size_t *device_bytes) {
    if (!s) return fail(RF_ERR_INVALID_ARG, "scene is NULL");
    if (n_sites) *n_sites = s->n_sites;
    if (n_edges) *n_edges = s->n_edges;
    if (aabb6) memcpy(aabb6, s->box, sizeof s->box);
    if (device_bytes) *device_bytes = s->bytes;
    return RF_OK;
}

RF_API rf_status rf_scene_destroy(rf_scene *s) {
    if (!s) return RF_OK;
    free_scene(s);
    return RF_OK;
}
