// rf_internal.cuh -- device-side building blocks of the Radiant Foam renderer
// (arXiv 2502.01157) for sm_103a.
//
// Every piece of arithmetic that decides which cells a ray visits (ray
// generation, the scene-box clip, the exit-face search of Alg. 1, the segment
// bounds and the transmittance update) is written with explicit
// round-to-nearest intrinsics and the library is compiled with -fmad=false, so
// the compiler cannot contract it differently in the forward and backward
// kernels: the backward re-walk reproduces the forward walk bit for bit.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rf.h"

namespace rf {

constexpr int kMaxCamsPerLaunch = 16;  // cameras per kernel launch (more: several launches)
constexpr int kTileW = 16;             // pixels per tile (x)
constexpr int kTileH = 8;              // pixels per tile (y)
constexpr int kBlock = kTileW * kTileH;  // one thread per pixel of a tile
constexpr int kDefaultMaxSteps = 1 << 16;

// ---------------------------------------------------------------------------
// Packed scene (device memory owned by rf_scene)
//   cells[i] = {x_i, y_i, z_i, bits(first_group << count_bits | n_groups)}
//   faces: the neighbours of cell i in groups of four, three float4 per group
//       {u_x of faces 0..3}, {u_y 0..3}, {u_z 0..3} (12 bytes per face),
//       u = 2 (p_j - p_i) / |p_j - p_i|^2; nbr[4 g + k] = j (-1: padding, u = 0)
// The forward is bound by the bytes the L1 delivers to the lanes per cell
// step, so a step reads a 16-byte header, 12 bytes per face and one 4-byte
// neighbour id (of the exit face only).
// With o~ = o - p_i the bisector of (p_i, p_j) is crossed at
//   t = (1 - u . o~) / (u . d),
// front-facing (an exit, Fig. 3) iff u . d > 0.
// ---------------------------------------------------------------------------
struct SceneDev {
    const float4 *cells;
    const float4 *faces;
    const int32_t *nbr;
    const void *density;
    const void *sh;
    float box_lo[3];
    float box_hi[3];
    int32_t count_bits;  // low bits of a header's w that hold its group count
    int32_t sh_v8;       // SH rows are 32-byte aligned (base and row size)
    int32_t n_sites;
};

// Cameras of one launch and the tile partition of their images.
struct LaunchCams {
    rf_camera cam[kMaxCamsPerLaunch];
    int32_t tile_begin[kMaxCamsPerLaunch + 1];  // prefix over cameras of tile counts
    int32_t tiles_x[kMaxCamsPerLaunch];
    int64_t ray_begin[kMaxCamsPerLaunch];       // output offset of each camera
    int32_t n_cams;
    int32_t cam0;                               // index of cam[0] in the start-cell table
};

// Optional analytic sphere of the walk (mirror: ior = 0; glass: ior > 0).
struct SphereFx {
    float cx, cy, cz, r;
    float ior;
    int32_t max_bounces;  // 0: no sphere
};

struct RenderParams {
    SceneDev s;
    LaunchCams lc;
    const unsigned long long *start_keys;  // [cam0 + c] low 32 bits: start cell
    float eps;
    int32_t max_steps;
    SphereFx fx;
    uint32_t *rec;                         // segment record of this launch (warp-major) or null
    int32_t rec_steps;                     // recorded steps per ray
};

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

// 256-bit read-only load (sm_100+); p must be 32-byte aligned.
__device__ __forceinline__ void ldg256(const void *p, uint32_t (&v)[8]) {
    asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7])
        : "l"(p));
}

struct CellHdr {
    float x, y, z;
    int gbeg, gcnt;  // first face group, number of groups
};

__device__ __forceinline__ CellHdr load_cell(const SceneDev &s, int i) {
    const float4 h = __ldg(s.cells + i);
    const uint32_t w = __float_as_uint(h.w);
    return {h.x, h.y, h.z, (int)(w >> s.count_bits), (int)(w & ((1u << s.count_bits) - 1u))};
}

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

// Map a block to (camera, tile) and a thread to a pixel: warp w of the block
// covers an 8x4 patch of the 16x8 tile, so the 32 rays of a warp are
// neighbours on the image and walk through mostly the same cells.  Lanes are
// laid out in Z-order inside the patch (lanes 4q..4q+3 form a 2x2 quad, 8q..8q+7
// a 4x2 block): the L1 serves a load in units of consecutive lanes, and compact
// units meet fewer distinct cells than an 8x1 row.
struct PixelTask {
    int cam, u, v;
    bool valid;
};

__device__ __forceinline__ PixelTask pixel_of_thread(const LaunchCams &lc) {
    PixelTask t;
    const int tile = blockIdx.x;
    int c = 0;
#pragma unroll 1
    while (c + 1 < lc.n_cams && lc.tile_begin[c + 1] <= tile) ++c;
    const int lt = tile - lc.tile_begin[c];
    const int tx = lt % lc.tiles_x[c];
    const int ty = lt / lc.tiles_x[c];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    t.cam = c;
    const int lx = (l & 1) | ((l >> 1) & 2) | ((l >> 2) & 4);  // bits 0, 2, 4 of the lane
    const int ly = ((l >> 1) & 1) | ((l >> 2) & 2);            // bits 1, 3
    t.u = tx * kTileW + (w & 1) * 8 + lx;
    t.v = ty * kTileH + (w >> 1) * 4 + ly;
    t.valid = t.u < lc.cam[c].width && t.v < lc.cam[c].height;
    return t;
}

__device__ __forceinline__ bool has_shutter(const rf_camera &c) {
    return c.shutter[0] != 0.f || c.shutter[1] != 0.f || c.shutter[2] != 0.f;
}

// Ray through the centre of pixel (u, v): pinhole, or equidistant fisheye
// (the angle to the optical axis equals the normalised image radius); with a
// rolling shutter the origin of row v moves by ((v + 1/2)/H - 1/2) shutter.
// EXT = false compiles the pinhole, global-shutter case only (the launch has
// no other camera); its arithmetic is the same as EXT's pinhole branch.
template <bool EXT>
__device__ __forceinline__ void camera_ray(const rf_camera &c, int u, int v, float3 &o, float3 &d) {
    float xc = __fdiv_rn(__fsub_rn(__fadd_rn((float)u, 0.5f), c.cx), c.fx);
    float yc = __fdiv_rn(__fsub_rn(__fadd_rn((float)v, 0.5f), c.cy), c.fy);
    float wx, wy, wz;
    if (EXT && c.model == RF_CAM_FISHEYE) {
        const float th = __fsqrt_rn(__fmaf_rn(xc, xc, __fmul_rn(yc, yc)));
        float sn, cs;
        sincospif(__fmul_rn(th, 0.318309886183790672f), &sn, &cs);  // th / pi: no wide range reduction
        const float sc = th > 0.f ? __fdiv_rn(sn, th) : 1.f;
        xc = __fmul_rn(xc, sc);
        yc = __fmul_rn(yc, sc);
        wx = __fmaf_rn(c.c2w[0], xc, __fmaf_rn(c.c2w[1], yc, __fmul_rn(c.c2w[2], cs)));
        wy = __fmaf_rn(c.c2w[4], xc, __fmaf_rn(c.c2w[5], yc, __fmul_rn(c.c2w[6], cs)));
        wz = __fmaf_rn(c.c2w[8], xc, __fmaf_rn(c.c2w[9], yc, __fmul_rn(c.c2w[10], cs)));
    } else {
        wx = __fmaf_rn(c.c2w[0], xc, __fmaf_rn(c.c2w[1], yc, c.c2w[2]));
        wy = __fmaf_rn(c.c2w[4], xc, __fmaf_rn(c.c2w[5], yc, c.c2w[6]));
        wz = __fmaf_rn(c.c2w[8], xc, __fmaf_rn(c.c2w[9], yc, c.c2w[10]));
    }
    const float len = __fsqrt_rn(__fmaf_rn(wx, wx, __fmaf_rn(wy, wy, __fmul_rn(wz, wz))));
    d = make_float3(__fdiv_rn(wx, len), __fdiv_rn(wy, len), __fdiv_rn(wz, len));
    o = make_float3(c.c2w[3], c.c2w[7], c.c2w[11]);
    if (EXT && has_shutter(c)) {
        const float row = __fsub_rn(__fdiv_rn(__fadd_rn((float)v, 0.5f), (float)c.height), 0.5f);
        o.x = __fmaf_rn(row, c.shutter[0], o.x);
        o.y = __fmaf_rn(row, c.shutter[1], o.y);
        o.z = __fmaf_rn(row, c.shutter[2], o.z);
    }
}

// Clip the ray to [t_near, t_far] and the scene box (slab test).
__device__ __forceinline__ bool ray_interval(const float3 &o, const float3 &d, const SceneDev &s,
                                             float t_near, float t_far, float &tmin, float &tmax) {
    float lo = t_near > 0.f ? t_near : 0.f;
    float hi = t_far > 0.f ? t_far : __int_as_float(0x7f800000);
    const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (dd[a] != 0.f) {
            float t1 = __fdiv_rn(__fsub_rn(s.box_lo[a], oo[a]), dd[a]);
            float t2 = __fdiv_rn(__fsub_rn(s.box_hi[a], oo[a]), dd[a]);
            if (t1 > t2) { const float q = t1; t1 = t2; t2 = q; }
            lo = t1 > lo ? t1 : lo;
            hi = t2 < hi ? t2 : hi;
        } else if (oo[a] < s.box_lo[a] || oo[a] > s.box_hi[a]) {
            return false;
        }
    }
    tmin = lo;
    tmax = hi;
    return lo < hi;
}

// Real orthonormal spherical harmonics of degree <= DEG at the unit
// direction d (no Condon-Shortley phase), index l*l + l + m.
template <int DEG>
__device__ __forceinline__ void sh_basis(const float3 &d, float *Y) {
    const float x = d.x, y = d.y, z = d.z;
    Y[0] = 0.28209479177387814f;                      // 1/(2 sqrt(pi))
    if (DEG >= 1) {
        const float c1 = 0.4886025119029199f;         // sqrt(3/(4 pi))
        Y[1] = c1 * y;
        Y[2] = c1 * z;
        Y[3] = c1 * x;
    }
    if (DEG >= 2) {
        const float a = 1.0925484305920792f;          // sqrt(15/pi)/2
        Y[4] = a * x * y;
        Y[5] = a * y * z;
        Y[6] = 0.31539156525252005f * (3.f * z * z - 1.f);   // sqrt(5/pi)/4
        Y[7] = a * x * z;
        Y[8] = 0.5462742152960396f * (x * x - y * y);        // sqrt(15/pi)/4
    }
    if (DEG >= 3) {
        const float b = 0.5900435899266435f;          // sqrt(35/(2 pi))/4
        const float c = 0.4570457994644658f;          // sqrt(21/(2 pi))/4
        Y[9] = b * y * (3.f * x * x - y * y);
        Y[10] = 2.890611442640554f * x * y * z;       // sqrt(105/pi)/2
        Y[11] = c * y * (5.f * z * z - 1.f);
        Y[12] = 0.3731763325901154f * z * (5.f * z * z - 3.f);  // sqrt(7/pi)/4
        Y[13] = c * x * (5.f * z * z - 1.f);
        Y[14] = 1.445305721320277f * z * (x * x - y * y);       // sqrt(105/pi)/4
        Y[15] = b * x * (x * x - 3.f * y * y);
    }
}

// Unpack 16 bytes of attribute storage into floats.
template <typename AT>
__device__ __forceinline__ void unpack16(const uint4 &q, float *out);
template <>
__device__ __forceinline__ void unpack16<float>(const uint4 &q, float *out) {
    out[0] = __uint_as_float(q.x); out[1] = __uint_as_float(q.y);
    out[2] = __uint_as_float(q.z); out[3] = __uint_as_float(q.w);
}
template <typename H2, typename F>
__device__ __forceinline__ void unpack_half2x4(const uint4 &q, float *out, F cvt) {
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        H2 h = *reinterpret_cast<const H2 *>(&w[k]);
        const float2 f = cvt(h);
        out[2 * k] = f.x;
        out[2 * k + 1] = f.y;
    }
}
template <>
__device__ __forceinline__ void unpack16<__nv_bfloat16>(const uint4 &q, float *out) {
    unpack_half2x4<__nv_bfloat162>(q, out, [](__nv_bfloat162 h) { return __bfloat1622float2(h); });
}
template <>
__device__ __forceinline__ void unpack16<__half>(const uint4 &q, float *out) {
    unpack_half2x4<__half2>(q, out, [](__half2 h) { return __half22float2(h); });
}

// Colour before the clamp: pre[ch] = sum_k sh[i][k][ch] Y_k + 0.5, summed in
// increasing k (Sec. 3.4).  Rows whose size is a multiple of 32 bytes are read
// with 256-bit loads when the base is 32-byte aligned (v8), else with 128-bit
// loads when possible, else element by element; the sum order is the same.
template <typename AT, int DEG>
__device__ __forceinline__ void sh_colour(const AT *__restrict__ sh, int i, const float *Y,
                                          float *pre, bool v8) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int NV = 3 * K;
    constexpr int RB = NV * (int)sizeof(AT);
    float acc[3] = {0.f, 0.f, 0.f};
    bool done = false;
    if constexpr (RB % 32 == 0) {
        if (v8) {
            constexpr int EPV = 16 / sizeof(AT);
            const char *row = reinterpret_cast<const char *>(sh) + (size_t)i * RB;
#pragma unroll
            for (int q = 0; q < RB / 32; ++q) {
                uint32_t w[8];
                ldg256(row + 32 * q, w);
                float v[2 * EPV];
                unpack16<AT>(make_uint4(w[0], w[1], w[2], w[3]), v);
                unpack16<AT>(make_uint4(w[4], w[5], w[6], w[7]), v + EPV);
#pragma unroll
                for (int e = 0; e < 2 * EPV; ++e) {
                    const int g = q * 2 * EPV + e;
                    acc[g % 3] = __fmaf_rn(v[e], Y[g / 3], acc[g % 3]);
                }
            }
            done = true;
        }
    }
    if (!done) {
        if constexpr (RB % 16 == 0) {
            constexpr int EPV = 16 / sizeof(AT);
            const uint4 *row = reinterpret_cast<const uint4 *>(sh + (size_t)i * NV);
#pragma unroll
            for (int q = 0; q < RB / 16; ++q) {
                float v[EPV];
                unpack16<AT>(ldg(row + q), v);
#pragma unroll
                for (int e = 0; e < EPV; ++e) {
                    const int g = q * EPV + e;
                    acc[g % 3] = __fmaf_rn(v[e], Y[g / 3], acc[g % 3]);
                }
            }
        } else {
            const AT *row = sh + (size_t)i * NV;
#pragma unroll
            for (int g = 0; g < NV; ++g) acc[g % 3] = __fmaf_rn(to_f(ldg(row + g)), Y[g / 3], acc[g % 3]);
        }
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) pre[ch] = __fadd_rn(acc[ch], 0.5f);
}

// Exit face of cell i (Alg. 1 inner loop): the front-facing bisector with the
// smallest crossing parameter, first in adjacency order on ties.  The
// comparison t_j < t_best is done by cross-multiplication (both denominators
// are positive), so no division is needed per face.  Padding faces have
// u = 0 and are never exits.  Returns j or -1.
__device__ __forceinline__ void face_test(float x, float y, float z, int slot, const float3 &d,
                                          const float3 &oc, float &nb, float &db, int &fb) {
    const float den = __fmaf_rn(x, d.x, __fmaf_rn(y, d.y, __fmul_rn(z, d.z)));
    const float num = __fmaf_rn(-x, oc.x, __fmaf_rn(-y, oc.y, __fmaf_rn(-z, oc.z, 1.f)));
    if (den > 0.f && __fmul_rn(num, db) < __fmul_rn(nb, den)) {
        nb = num;
        db = den;
        fb = slot;
    }
}

__device__ __forceinline__ int find_exit(const SceneDev &s, const CellHdr &c, const float3 &d,
                                         const float3 &oc, float &num_best, float &den_best, int &slot) {
    float nb = 1.f, db = 0.f;
    int fb = -1;
    const float4 *f = s.faces + 3 * (size_t)c.gbeg;
#pragma unroll 2
    for (int g = 0; g < c.gcnt; ++g) {
        const float4 X = ldg(f + 3 * g), Y = ldg(f + 3 * g + 1), Z = ldg(f + 3 * g + 2);
        face_test(X.x, Y.x, Z.x, 4 * g + 0, d, oc, nb, db, fb);
        face_test(X.y, Y.y, Z.y, 4 * g + 1, d, oc, nb, db, fb);
        face_test(X.z, Y.z, Z.z, 4 * g + 2, d, oc, nb, db, fb);
        face_test(X.w, Y.w, Z.w, 4 * g + 3, d, oc, nb, db, fb);
    }
    num_best = nb;
    den_best = db;
    slot = fb;
    return fb >= 0 ? ldg(s.nbr + 4 * (size_t)c.gbeg + fb) : -1;
}

// One segment's bounds, width, density and colour (shared by all kernels).
struct Segment {
    float t1;      // raw exit parameter (inf: no exit)
    float a, b;    // composited part
    float delta;
    float sigma;
    float e;       // exp(-sigma delta)
    float pre[3];  // colour before the clamp
    int next;
    bool hit;      // the segment ends on the sphere at ts (FX kernels)
};

// Composited part [a, b) of the segment [t0, t1) clipped to [t_min, t_max)
// and, with FX, ended early by a sphere crossing at ts in [t0, t1) before
// t_max; its width delta = max(b - a, 0) and transmittance factor e.
template <bool FX>
__device__ __forceinline__ void segment_bounds(Segment &g, float t0, float tmin, float tmax, float ts) {
    g.a = t0 > tmin ? t0 : tmin;
    float tend = g.t1;
    g.hit = false;
    if constexpr (FX) {
        g.hit = ts >= t0 && ts < g.t1 && ts < tmax;
        if (g.hit) tend = ts;
    }
    g.b = tend < tmax ? tend : tmax;
    const float w = __fsub_rn(g.b, g.a);
    g.delta = w > 0.f ? w : 0.f;
    g.e = expf(-__fmul_rn(g.sigma, g.delta));
}

// With FX, ts is the current ray's next sphere crossing (+inf: none): when it
// falls in [t0, t1) and before t_max the segment ends there instead of at the
// face.
template <typename AT, int DEG, bool FX = false>
__device__ __forceinline__ void cell_step(const SceneDev &s, int i, const CellHdr &cell,
                                          const float3 &o, const float3 &d, float t0, float tmin,
                                          float tmax, const float *Y, Segment &g, float3 &oc,
                                          float ts = 0.f) {
    oc = make_float3(__fsub_rn(o.x, cell.x), __fsub_rn(o.y, cell.y), __fsub_rn(o.z, cell.z));
    float nb = 1.f, db = 0.f;
    int slot;
    g.next = find_exit(s, cell, d, oc, nb, db, slot);
    g.t1 = g.next >= 0 ? __fdiv_rn(nb, db) : __int_as_float(0x7f800000);
    g.sigma = to_f(ldg(reinterpret_cast<const AT *>(s.density) + i));
    segment_bounds<FX>(g, t0, tmin, tmax, ts);
    sh_colour<AT, DEG>(reinterpret_cast<const AT *>(s.sh), i, Y, g.pre, s.sh_v8 != 0);
}

// Segment record.  In a training step the forward keeps, for each of the
// first rec_steps steps of a ray, what the backward needs of the segment:
// the exit neighbour, the raw exit parameter t1, the density and the colour
// before the clamp (24 bytes).  Warp-major: per warp and step one row of six
// 32-lane columns, so a warp stores and loads each field as one coalesced
// 128-byte line, with streaming cache hints (the record is read once, by the
// backward, and must not evict the scene from L2).  The backward rebuilds the
// segment from it with the arithmetic of cell_step (segment_bounds), so it
// meets the same bits without reading the faces or the attributes again.
constexpr int kRecWords = 6;

// This lane's column of its warp's record (null without a record).
__device__ __forceinline__ uint32_t *record_column(const RenderParams &p) {
    if (!p.rec) return nullptr;
    return p.rec + ((int64_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5)) * p.rec_steps * (32 * kRecWords) +
           (threadIdx.x & 31);
}

// The backward brings its warp's record rows into L2 kRecAhead steps ahead
// of their loads, kRecAhead rows (contiguous, 768 bytes each) per bulk
// prefetch issued by one lane: the record was written long before, so
// without it every step's loads wait for DRAM.
constexpr int kRecAhead = 8;

// Prefetch the rows of steps [k, min(k + n, p.rec_steps)) of this warp's record.
__device__ __forceinline__ void record_prefetch(const RenderParams &p, int k, int n) {
    if (!p.rec || k >= p.rec_steps) return;
    if (k + n > p.rec_steps) n = p.rec_steps - k;
    const uint32_t *row = p.rec + ((int64_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5)) * p.rec_steps *
                                      (32 * kRecWords) +
                          (int64_t)k * (32 * kRecWords);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(row), "r"(n * 32 * kRecWords * 4) : "memory");
}

__device__ __forceinline__ void record_store(uint32_t *col, int k, const Segment &g) {
    uint32_t *r = col + (int64_t)k * (32 * kRecWords);
    __stcs(reinterpret_cast<int *>(r), g.next);
    __stcs(reinterpret_cast<float *>(r + 32), g.t1);
    __stcs(reinterpret_cast<float *>(r + 64), g.sigma);
    __stcs(reinterpret_cast<float *>(r + 96), g.pre[0]);
    __stcs(reinterpret_cast<float *>(r + 128), g.pre[1]);
    __stcs(reinterpret_cast<float *>(r + 160), g.pre[2]);
}

// The recorded segment of step k in the current cell (position `cell`).  An
// exit id outside the scene (a record of another scene) ends the walk there.
template <bool FX>
__device__ __forceinline__ void record_step(const SceneDev &s, const uint32_t *col, int k, const CellHdr &cell,
                                            const float3 &o, float t0, float tmin, float tmax, Segment &g,
                                            float3 &oc, float ts = 0.f) {
    const uint32_t *r = col + (int64_t)k * (32 * kRecWords);
    oc = make_float3(__fsub_rn(o.x, cell.x), __fsub_rn(o.y, cell.y), __fsub_rn(o.z, cell.z));
    const int next = __ldcs(reinterpret_cast<const int *>(r));
    g.t1 = __ldcs(reinterpret_cast<const float *>(r + 32));
    g.sigma = __ldcs(reinterpret_cast<const float *>(r + 64));
    g.pre[0] = __ldcs(reinterpret_cast<const float *>(r + 96));
    g.pre[1] = __ldcs(reinterpret_cast<const float *>(r + 128));
    g.pre[2] = __ldcs(reinterpret_cast<const float *>(r + 160));
    g.next = next >= 0 && next < s.n_sites ? next : -1;
    if (g.next < 0) g.t1 = __int_as_float(0x7f800000);
    segment_bounds<FX>(g, t0, tmin, tmax, ts);
}

// ---------------------------------------------------------------------------
// Sphere bounces (reflection / refraction met in the walk, Fig. 2)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dot3(const float3 &a, const float3 &b) {
    return __fmaf_rn(a.x, b.x, __fmaf_rn(a.y, b.y, __fmul_rn(a.z, b.z)));
}

// Parameter of the ray's next crossing of the sphere (the entry from
// outside, the exit from inside), +inf if none lies ahead.  The
// discriminant is r^2 - h^2 with h the distance of the centre from the ray
// (no cancellation when the origin lies on the sphere after a bounce).
__device__ __forceinline__ float sphere_next(const SphereFx &fx, const float3 &o, const float3 &d,
                                             bool inside) {
    const float3 oc = make_float3(__fsub_rn(o.x, fx.cx), __fsub_rn(o.y, fx.cy), __fsub_rn(o.z, fx.cz));
    const float b = dot3(d, oc);
    const float3 q = make_float3(__fmaf_rn(-b, d.x, oc.x), __fmaf_rn(-b, d.y, oc.y), __fmaf_rn(-b, d.z, oc.z));
    const float disc = __fsub_rn(__fmul_rn(fx.r, fx.r), dot3(q, q));
    if (!(disc >= 0.f)) return __int_as_float(0x7f800000);
    const float w = __fsqrt_rn(disc);
    const float t = inside ? __fadd_rn(-b, w) : __fsub_rn(-b, w);
    return t > 0.f ? t : __int_as_float(0x7f800000);
}

// Bend the ray at the hit point p: mirror reflection, or Snell refraction
// with relative index 1/n entering and n leaving (total internal reflection
// when no refracted ray exists).  Updates d (unit) and the inside flag.
__device__ __forceinline__ void sphere_bend(const SphereFx &fx, const float3 &p, float3 &d, bool &inside) {
    const float ir = __fdiv_rn(1.f, fx.r);
    const float3 n = make_float3(__fmul_rn(__fsub_rn(p.x, fx.cx), ir), __fmul_rn(__fsub_rn(p.y, fx.cy), ir),
                                 __fmul_rn(__fsub_rn(p.z, fx.cz), ir));
    const float dn = dot3(d, n);
    bool crossed = false;
    float3 r;
    if (fx.ior > 0.f) {
        const float sg = inside ? -1.f : 1.f;              // normal on the incoming side: sg n
        const float eta = inside ? fx.ior : __fdiv_rn(1.f, fx.ior);
        const float ci = __fmul_rn(-dn, sg);
        const float k = __fsub_rn(1.f, __fmul_rn(__fmul_rn(eta, eta), __fsub_rn(1.f, __fmul_rn(ci, ci))));
        if (k >= 0.f) {
            const float f = __fmul_rn(__fsub_rn(__fmul_rn(eta, ci), __fsqrt_rn(k)), sg);
            r = make_float3(__fmaf_rn(eta, d.x, __fmul_rn(f, n.x)), __fmaf_rn(eta, d.y, __fmul_rn(f, n.y)),
                            __fmaf_rn(eta, d.z, __fmul_rn(f, n.z)));
            crossed = true;
        }
    }
    if (!crossed) {
        const float m = __fmul_rn(-2.f, dn);
        r = make_float3(__fmaf_rn(m, n.x, d.x), __fmaf_rn(m, n.y, d.y), __fmaf_rn(m, n.z, d.z));
    } else {
        inside = !inside;
    }
    const float len = __fsqrt_rn(dot3(r, r));
    d = make_float3(__fdiv_rn(r.x, len), __fdiv_rn(r.y, len), __fdiv_rn(r.z, len));
}

// State of a ray that may bounce off the sphere.
struct FxRay {
    float ts;      // next sphere crossing on the current leg (+inf: none)
    float soff;    // path length before the current leg's origin
    int bounces;
    bool inside;
};

__device__ __forceinline__ void fx_begin(const SphereFx &fx, const float3 &o, const float3 &d, FxRay &f) {
    const float3 oc = make_float3(__fsub_rn(o.x, fx.cx), __fsub_rn(o.y, fx.cy), __fsub_rn(o.z, fx.cz));
    f.inside = dot3(oc, oc) < __fmul_rn(fx.r, fx.r);
    f.soff = 0.f;
    f.bounces = 0;
    f.ts = fx.max_bounces > 0 ? sphere_next(fx, o, d, f.inside) : __int_as_float(0x7f800000);
}

// After a segment that ended on the sphere: move the origin to the hit
// point, bend the direction, clip the new leg to the scene box.  Returns
// false when the new leg has no part inside the box.
__device__ __forceinline__ bool fx_bounce(const SphereFx &fx, const SceneDev &s, FxRay &f, float3 &o,
                                          float3 &d, float &tmin, float &tmax) {
    const float3 p = make_float3(__fmaf_rn(f.ts, d.x, o.x), __fmaf_rn(f.ts, d.y, o.y), __fmaf_rn(f.ts, d.z, o.z));
    sphere_bend(fx, p, d, f.inside);
    o = p;
    f.soff = __fadd_rn(f.soff, f.ts);
    ++f.bounces;
    if (!ray_interval(o, d, s, 0.f, 0.f, tmin, tmax)) return false;
    f.ts = f.bounces < fx.max_bounces ? sphere_next(fx, o, d, f.inside) : __int_as_float(0x7f800000);
    return true;
}

// Start cell of a rolling-shutter row: the cell containing the row's origin
// q, reached by walking the segment from the centre c (in cell i) to q
// through the foam with the same exit search as the ray walk.
__device__ __forceinline__ int locate_from(const SceneDev &s, int i, const float3 &c, const float3 &q,
                                           int max_steps) {
    const float3 v = make_float3(__fsub_rn(q.x, c.x), __fsub_rn(q.y, c.y), __fsub_rn(q.z, c.z));
    const float L = __fsqrt_rn(dot3(v, v));
    if (!(L > 0.f)) return i;
    const float3 d = make_float3(__fdiv_rn(v.x, L), __fdiv_rn(v.y, L), __fdiv_rn(v.z, L));
    for (int k = 0; k < max_steps; ++k) {
        const CellHdr cell = load_cell(s, i);
        const float3 oc = make_float3(__fsub_rn(c.x, cell.x), __fsub_rn(c.y, cell.y), __fsub_rn(c.z, cell.z));
        float nb, db;
        int slot;
        const int nx = find_exit(s, cell, d, oc, nb, db, slot);
        if (nx < 0 || !(__fdiv_rn(nb, db) < L)) break;
        i = nx;
    }
    return i;
}

// Start cell of a ray: nn(camera centre) from the per-camera table, moved to
// the row's origin for a rolling shutter.
template <bool EXT>
__device__ __forceinline__ int start_cell(const RenderParams &p, int cam, const float3 &o) {
    int i = (int)(p.start_keys[p.lc.cam0 + cam] & 0xffffffffull);
    const rf_camera &c = p.lc.cam[cam];
    if (EXT && has_shutter(c))
        i = locate_from(p.s, i, make_float3(c.c2w[3], c.c2w[7], c.c2w[11]), o, p.max_steps);
    return i;
}

// ---------------------------------------------------------------------------
// Quantile loss (Eq. 6) pieces.  For a segment of width delta and density
// sigma entered with transmittance T_n and accumulated weight W_n = 1 - T_n,
// with x = sigma delta, g(x) = (1 - e^-x)/x and u(s) = 1 - e^{-sigma s}:
//   A = int T/T_n = delta g,   C = int u (1 - u) = delta x g^2 / 2,
//   int u = delta f1,  f1 = 1 - g,   int u^2 = delta f2,  f2 = f1 - x g^2 / 2.
// With W(t) = 1 - T(t) = W_n + T_n u:
//   Q = int W dt  (sum of W_n delta + T_n delta f1),
//   Q2 = int W^2 dt (sum of W_n^2 delta + 2 W_n T_n delta f1 + T_n^2 delta f2),
// and the loss is 2 int W (W_tot - W) dt / W_tot^2 = 2 (W_tot Q - Q2) / W_tot^2:
// both terms are of the same order, so nearly transparent rays (small W_tot)
// do not cancel.  f1, f2 use their series for small x.
// ---------------------------------------------------------------------------
struct QuantSeg {
    float A, C, f1d, f2d;   // A, C, delta f1, delta f2
    float dA_ds, dC_ds;     // d/dsigma at fixed delta
    float alpha;            // 1 - e^-x, accurate for small x
};

__device__ __forceinline__ QuantSeg quant_seg(float sigma, float delta, float e) {
    QuantSeg q;
    const float x = sigma * delta;
    if (x < 0.1f) {
        // series in x, truncation error < 2e-8 relative at x = 0.1
        const float f1 = x * (0.5f - x * (1.f / 6.f - x * (1.f / 24.f - x * (1.f / 120.f - x * (1.f / 720.f)))));
        const float g = 1.f - f1;
        const float f2 = x * x * (1.f / 3.f - x * (0.25f - x * (7.f / 60.f - x * (1.f / 24.f - x * (31.f / 2520.f)))));
        q.A = delta * g;
        q.f1d = delta * f1;
        q.f2d = delta * f2;
        q.alpha = x * g;
        q.C = 0.5f * delta * x * g * g;
        q.dA_ds = -delta * delta * (0.5f - x * (1.f / 3.f - x * (0.125f - x * (1.f / 30.f))));
        q.dC_ds = 0.5f * delta * delta * (1.f - x * (2.f - x * (1.75f - x)));
    } else {
        const float alpha = -expm1f(-x);
        const float g = alpha / x;
        const float f1 = 1.f - g;
        q.alpha = alpha;
        q.A = delta * g;
        q.f1d = delta * f1;
        q.f2d = delta * (f1 - 0.5f * x * g * g);
        q.C = 0.5f * delta * x * g * g;
        const float s2 = sigma * sigma;
        q.dA_ds = (x * e - alpha) / s2;
        q.dC_ds = alpha * (2.f * x * e - alpha) / (2.f * s2);
    }
    return q;
}

}  // namespace rf
