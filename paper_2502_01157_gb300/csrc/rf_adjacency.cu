// rf_adjacency.cu -- GPU construction of the Voronoi adjacency N(i) that the
// walk of Alg. 1 traverses (the Delaunay neighbour lists, rebuilt whenever the
// sites move: the "Voronoi optimization" paragraph of Sec. 4).
//
// The method is the per-cell clipping of Ray, Sokolov, Lefebvre and Levy,
// "Meshless Voronoi on the GPU" (ACM TOG 2018), written here from that
// description.  Each site's cell is built directly, one warp per site, as a
// convex polytope:
// the domain box cut by the bisector half-spaces of nearby sites,
//   (p_k - p_i) . x <= |p_k - p_i|^2 / 2   (x relative to p_i).
// The polytope is kept in shared memory in dual form: every vertex is a
// triangle of three plane slots (oriented consistently), so a cut removes the
// vertices outside the new plane and closes the hole with a fan of triangles
// along its boundary cycle.  Candidates come from a uniform grid, shell by
// shell around the site's grid cell, nearest first inside each batch of 32.
// A site k can cut the cell only if |p_k - p_i| < 2 R, R the cell's largest
// vertex distance (rows of the grid beyond that are skipped), and only if it
// lies in the ball about some vertex v of radius |v|; the search stops once
// all those balls lie in the scanned block of grid cells.  The neighbours are
// the sites whose planes still hold a vertex at the end.
//
// The inside/outside test of a vertex is made in FP32 with an error bound;
// when the FP32 value lies within the bound, the vertex and the test are
// recomputed in FP64 from the sites' coordinates, so every decision is the
// FP64 one.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "rf_host.h"

namespace rf {
namespace {

constexpr int kWarps = 4;             // sites (warps) per block, normal pass
constexpr int kMaxPlanes = 64;        // normal pass: 6 box planes + up to 58 sites
constexpr int kWideWarps = 2;
constexpr int kWideMaxPlanes = 192;   // second pass for the cells that overflowed
constexpr int32_t kFreeSlot = INT32_MIN;
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanItems;

enum : int32_t { kCellOk = 0, kCellOverflow = 1, kCellBroken = 2 };

// The (dz, dy) rows of the blocks of shells 0..3 sorted by dz^2 + dy^2 (then
// dz, dy): nearer rows first, so the first cuts come from nearer sites.
__constant__ int8_t kRowOrder[84][2] = {
    // shell 0: the 1 rows of its 1x1 block
    {0, 0},
    // shell 1: the 9 rows of its 3x3 block
    {0, 0}, {-1, 0}, {0, -1}, {0, 1}, {1, 0}, {-1, -1}, {-1, 1}, {1, -1}, {1, 1},
    // shell 2: the 25 rows of its 5x5 block
    {0, 0}, {-1, 0}, {0, -1}, {0, 1}, {1, 0}, {-1, -1}, {-1, 1}, {1, -1}, {1, 1}, {-2, 0},
    {0, -2}, {0, 2}, {2, 0}, {-2, -1}, {-2, 1}, {-1, -2}, {-1, 2}, {1, -2}, {1, 2}, {2, -1},
    {2, 1}, {-2, -2}, {-2, 2}, {2, -2}, {2, 2},
    // shell 3: the 49 rows of its 7x7 block
    {0, 0}, {-1, 0}, {0, -1}, {0, 1}, {1, 0}, {-1, -1}, {-1, 1}, {1, -1}, {1, 1}, {-2, 0},
    {0, -2}, {0, 2}, {2, 0}, {-2, -1}, {-2, 1}, {-1, -2}, {-1, 2}, {1, -2}, {1, 2}, {2, -1},
    {2, 1}, {-2, -2}, {-2, 2}, {2, -2}, {2, 2}, {-3, 0}, {0, -3}, {0, 3}, {3, 0}, {-3, -1},
    {-3, 1}, {-1, -3}, {-1, 3}, {1, -3}, {1, 3}, {3, -1}, {3, 1}, {-3, -2}, {-3, 2}, {-2, -3},
    {-2, 3}, {2, -3}, {2, 3}, {3, -2}, {3, 2}, {-3, -3}, {-3, 3}, {3, -3}, {3, 3}
};
__constant__ int16_t kRowStart[5] = {0, 1, 10, 35, 84};

struct GridDev {
    const float4 *sorted;      // sites sorted by grid cell: x, y, z, bits(id)
    const int32_t *cell_start; // [ncell + 1]
    int dims[3];
    float lo[3];
    float h, inv_h;
};

struct CellParams {
    const float *pos;          // [N][3] the caller's sites
    int64_t n;
    GridDev g;
    float dom[6];              // domain box: min xyz, max xyz
    const int32_t *seed_off;   // previous adjacency (incremental) or null
    const int32_t *seed_idx;
    const int32_t *site_list;  // sites to build (wide pass) or null: all
    const int32_t *n_list;     // device count of site_list
    int32_t *row_base;         // [N] start of the site's row in edge_buf
    int32_t *row_cnt;          // [N]
    int32_t *edge_buf;
    int32_t edge_cap;
    int32_t *counters;         // [0] edges used, [1] wide sites, [2] broken sites, [3] fp64 tests
    int32_t *wide_list;        // sites that overflowed (normal pass)
};

template <int MAXP>
struct CellSmem {
    float4 pl[MAXP];                     // plane: n.xyz, b (site-relative)
    int32_t pid[MAXP];                   // site id, -1 - side for box planes, kFreeSlot
    uint32_t tri[2 * MAXP];              // vertex = plane slots a | b << 8 | c << 16
    float4 vtx[2 * MAXP];                // vertex x, y, z and its FP32 error bound
    uint32_t ebits[MAXP * (MAXP / 32)];  // directed edges of the removed triangles
    uint32_t src_seen[MAXP / 32];        // boundary-edge sources seen in this cut
    float vlen[2 * MAXP];                // |vertex|
    float box[6];                        // bounding box of the vertices (with their error bounds)
    uint8_t nxt[MAXP];                   // boundary cycle: a -> nxt[a]
    uint8_t cyc[MAXP];
};

__device__ __forceinline__ float3 cross3(const float3 &a, const float3 &b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float dot3f(const float3 &a, const float3 &b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float len3(const float3 &a) { return sqrtf(dot3f(a, a)); }

// Vertex of three planes by Cramer's rule, with a bound on its FP32 error.
__device__ __forceinline__ float4 vertex_of(const float4 &A, const float4 &B, const float4 &C) {
    const float3 na = make_float3(A.x, A.y, A.z), nb = make_float3(B.x, B.y, B.z), nc = make_float3(C.x, C.y, C.z);
    const float3 bc = cross3(nb, nc), ca = cross3(nc, na), ab = cross3(na, nb);
    const float det = dot3f(na, bc);
    const float id = 1.f / det;
    float4 v;
    v.x = (A.w * bc.x + B.w * ca.x + C.w * ab.x) * id;
    v.y = (A.w * bc.y + B.w * ca.y + C.w * ab.y) * id;
    v.z = (A.w * bc.z + B.w * ca.z + C.w * ab.z) * id;
    // each term carries a few roundings of its own size; the planes
    // themselves are rounded to a relative 2^-24
    const float mag = (fabsf(A.w) * len3(bc) + fabsf(B.w) * len3(ca) + fabsf(C.w) * len3(ab)) * fabsf(id);
    v.w = isfinite(mag) ? 64.f * 5.96e-8f * mag : __int_as_float(0x7f800000);
    return v;
}

// Plane of slot s in FP64 from the sites' coordinates (box planes from the domain).
__device__ __forceinline__ void plane64(const CellParams &P, int32_t id, const double *pi, double *n, double &b) {
    if (id >= 0) {
        double nn = 0.0;
        for (int a = 0; a < 3; ++a) {
            n[a] = (double)P.pos[3 * (int64_t)id + a] - pi[a];
            nn += n[a] * n[a];
        }
        b = 0.5 * nn;
    } else {
        const int side = -1 - id, ax = side >> 1;
        n[0] = n[1] = n[2] = 0.0;
        if (side & 1) {
            n[ax] = -1.0;
            b = pi[ax] - (double)P.dom[ax];
        } else {
            n[ax] = 1.0;
            b = (double)P.dom[3 + ax] - pi[ax];
        }
    }
}

// Side of the vertex (planes a, b, c) with respect to plane q, in FP64.
__device__ __noinline__ double side64(const CellParams &P, const double *pi, int32_t ia, int32_t ib, int32_t ic,
                                      int32_t iq) {
    double na[3], nb[3], nc[3], nq[3], ba, bb, bc, bq;
    plane64(P, ia, pi, na, ba);
    plane64(P, ib, pi, nb, bb);
    plane64(P, ic, pi, nc, bc);
    plane64(P, iq, pi, nq, bq);
    const double xbc[3] = {nb[1] * nc[2] - nb[2] * nc[1], nb[2] * nc[0] - nb[0] * nc[2], nb[0] * nc[1] - nb[1] * nc[0]};
    const double xca[3] = {nc[1] * na[2] - nc[2] * na[1], nc[2] * na[0] - nc[0] * na[2], nc[0] * na[1] - nc[1] * na[0]};
    const double xab[3] = {na[1] * nb[2] - na[2] * nb[1], na[2] * nb[0] - na[0] * nb[2], na[0] * nb[1] - na[1] * nb[0]};
    const double det = na[0] * xbc[0] + na[1] * xbc[1] + na[2] * xbc[2];
    // s = nq . v - bq with v = (ba xbc + bb xca + bc xab) / det, scaled by det
    // (sign-corrected) so that no division rounds
    double num = 0.0;
    for (int a = 0; a < 3; ++a) num += nq[a] * (ba * xbc[a] + bb * xca[a] + bc * xab[a]);
    const double s = num - bq * det;
    return det > 0.0 ? s : -s;
}

template <int MAXP>
struct Cell {
    static constexpr int MAXT = 2 * MAXP;
    static constexpr int PW = MAXP / 32;  // plane words
    CellSmem<MAXP> &m;
    const CellParams &P;
    const int lane;
    const double *pi;  // the site in FP64 (per lane copy)
    int n_tri = 0;
    float R2 = 0.f;    // squared radius bound of the cell about the site
    int32_t status = kCellOk;

    __device__ Cell(CellSmem<MAXP> &sm, const CellParams &p, int l, const double *pi64)
        : m(sm), P(p), lane(l), pi(pi64) {}

    // signed floats as ints of the same order, for the warp min / max reductions
    static __device__ __forceinline__ int okey(float f) {
        const int b = __float_as_int(f);
        return b >= 0 ? b : b ^ 0x7fffffff;
    }
    static __device__ __forceinline__ float okey_inv(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

    // radius and bounding box of the current vertices
    __device__ void update_bounds() {
        float r = 0.f;
        int lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
        for (int t = lane; t < n_tri; t += 32) {
            const float4 v = m.vtx[t];
            r = fmaxf(r, m.vlen[t] + v.w);
            lo[0] = min(lo[0], okey(v.x - v.w));
            lo[1] = min(lo[1], okey(v.y - v.w));
            lo[2] = min(lo[2], okey(v.z - v.w));
            hi[0] = max(hi[0], okey(v.x + v.w));
            hi[1] = max(hi[1], okey(v.y + v.w));
            hi[2] = max(hi[2], okey(v.z + v.w));
        }
        r = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(r)));  // r >= 0
        R2 = r * r * (1.f + 1e-5f);
        for (int a = 0; a < 3; ++a) {
            const float l = okey_inv(__reduce_min_sync(0xffffffffu, lo[a]));
            const float h = okey_inv(__reduce_max_sync(0xffffffffu, hi[a]));
            if (lane == 0) {
                m.box[a] = l;
                m.box[3 + a] = h;
            }
        }
        __syncwarp();
    }

    // Can the bisector of a site at d reach the cell?  Its half-space n . x <=
    // |n|^2 / 2 (n = d) holds the whole bounding box when the box's support in
    // direction n is below |n|^2 / 2; with a margin for the FP32 rounding, a
    // "no" is certain.
    __device__ __forceinline__ bool may_cut(const float3 &d, float d2) const {
        const float sx = d.x * m.box[d.x > 0.f ? 3 : 0];
        const float sy = d.y * m.box[d.y > 0.f ? 4 : 1];
        const float sz = d.z * m.box[d.z > 0.f ? 5 : 2];
        const float mag = fabsf(sx) + fabsf(sy) + fabsf(sz) + 0.5f * d2;
        return sx + sy + sz > 0.5f * d2 - 1e-5f * mag;
    }

    __device__ __forceinline__ void put_vertex(int t, const float4 &v) {
        m.vtx[t] = v;
        m.vlen[t] = sqrtf(v.x * v.x + v.y * v.y + v.z * v.z);
    }

    // The domain box about the site: slots 0..5 = +x, -x, +y, -y, +z, -z.
    __device__ void init_box(const float3 &p) {
        for (int s = lane; s < MAXP; s += 32) m.pid[s] = kFreeSlot;
        for (int w = lane; w < MAXP * PW; w += 32) m.ebits[w] = 0u;
        if (lane < PW) m.src_seen[lane] = 0u;
        __syncwarp();
        if (lane < 6) {
            const int ax = lane >> 1;
            const float pa = ax == 0 ? p.x : ax == 1 ? p.y : p.z;
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            if (lane & 1) {
                (ax == 0 ? q.x : ax == 1 ? q.y : q.z) = -1.f;
                q.w = pa - P.dom[ax];
            } else {
                (ax == 0 ? q.x : ax == 1 ? q.y : q.z) = 1.f;
                q.w = P.dom[3 + ax] - pa;
            }
            m.pl[lane] = q;
            m.pid[lane] = -1 - lane;
        }
        __syncwarp();
        if (lane < 8) {
            const int sx = lane & 1, sy = (lane >> 1) & 1, sz = (lane >> 2) & 1;  // 1: minus side
            const uint32_t X = sx, Y = 2 + sy, Z = 4 + sz;
            // det(n_X, n_Y, n_Z) = (-1)^(sx+sy+sz): keep det > 0 (counter-clockwise seen from outside)
            const bool pos = ((sx + sy + sz) & 1) == 0;
            m.tri[lane] = pos ? (X | Y << 8 | Z << 16) : (X | Z << 8 | Y << 16);
            put_vertex(lane, vertex_of(m.pl[X], m.pl[pos ? Y : Z], m.pl[pos ? Z : Y]));
        }
        n_tri = 8;
        __syncwarp();
        update_bounds();
    }

    __device__ int alloc_slot() {
        for (int w = 0; w < PW; ++w) {
            const unsigned f = __ballot_sync(0xffffffffu, m.pid[w * 32 + lane] == kFreeSlot);
            if (f) return w * 32 + __ffs(f) - 1;
        }
        return -1;
    }

    __device__ bool has_site(int32_t k) {
        bool hit = false;
        for (int w = 0; w < PW; ++w) hit |= m.pid[w * 32 + lane] == k;
        return __any_sync(0xffffffffu, hit);
    }

    __device__ __forceinline__ void set_edge(uint32_t a, uint32_t b) {
        atomicOr(&m.ebits[a * PW + (b >> 5)], 1u << (b & 31));
    }
    __device__ __forceinline__ void clear_edge(uint32_t a, uint32_t b) {
        atomicAnd(&m.ebits[a * PW + (b >> 5)], ~(1u << (b & 31)));
    }
    __device__ __forceinline__ bool has_edge(uint32_t a, uint32_t b) const {
        return (m.ebits[a * PW + (b >> 5)] >> (b & 31)) & 1u;
    }

    // Cut the cell by the bisector of site k (n = p_k - p_i relative to the site).
    __device__ void cut(int32_t k, const float3 &n) {
        const unsigned full = 0xffffffffu;
        const int q = alloc_slot();
        if (q < 0) {
            status = kCellOverflow;
            return;
        }
        const float4 Q = make_float4(n.x, n.y, n.z, 0.5f * dot3f(n, n));
        const float nq = len3(n);
        // 1. which vertices lie outside
        uint32_t rem[MAXT / 32];
        int removed = 0;
        for (int c = 0; c < (n_tri + 31) / 32; ++c) {
            const int t = c * 32 + lane;
            bool out = false;
            if (t < n_tri) {
                const float4 v = m.vtx[t];
                const float s = Q.x * v.x + Q.y * v.y + Q.z * v.z - Q.w;
                const float bound = 2.f * (nq * v.w + 4.f * 5.96e-8f * (nq * m.vlen[t] + Q.w));
                if (fabsf(s) > bound) {
                    out = s > 0.f;
                } else {
                    const uint32_t tv = m.tri[t];
                    out = side64(P, pi, m.pid[tv & 255], m.pid[(tv >> 8) & 255], m.pid[(tv >> 16) & 255], k) > 0.0;
                    atomicAdd(P.counters + 3, 1);
                }
            }
            rem[c] = __ballot_sync(full, out);
            removed += __popc(rem[c]);
        }
        for (int c = (n_tri + 31) / 32; c < MAXT / 32; ++c) rem[c] = 0u;
        if (removed == 0) return;  // the plane misses the cell; slot q stays free
        if (removed == n_tri) {    // the site itself is always inside: cannot happen
            status = kCellBroken;
            return;
        }
        m.pl[q] = Q;
        m.pid[q] = k;
        // 2. directed edges of the removed vertices
        for (int c = 0; c < (n_tri + 31) / 32; ++c)
            if ((rem[c] >> lane) & 1u) {
                const uint32_t tv = m.tri[c * 32 + lane];
                const uint32_t a = tv & 255, b = (tv >> 8) & 255, d = (tv >> 16) & 255;
                set_edge(a, b);
                set_edge(b, d);
                set_edge(d, a);
            }
        __syncwarp();
        // 3. boundary: an edge whose reverse belongs to a kept vertex
        int nbound = 0, start = -1;
        bool clash = false;
        for (int c = 0; c < (n_tri + 31) / 32; ++c) {
            int mine = 0;
            if ((rem[c] >> lane) & 1u) {
                const uint32_t tv = m.tri[c * 32 + lane];
                const uint32_t e[3] = {tv & 255, (tv >> 8) & 255, (tv >> 16) & 255};
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const uint32_t a = e[j], b = e[(j + 1) % 3];
                    if (!has_edge(b, a)) {
                        const uint32_t old = atomicOr(&m.src_seen[a >> 5], 1u << (a & 31));
                        clash |= (old >> (a & 31)) & 1u;
                        m.nxt[a] = (uint8_t)b;
                        start = (int)a;
                        ++mine;
                    }
                }
            }
            nbound += mine;
        }
        for (int o = 16; o; o >>= 1) nbound += __shfl_xor_sync(full, nbound, o);
        clash = __any_sync(full, clash);
        const unsigned has = __ballot_sync(full, start >= 0);
        start = __shfl_sync(full, start, has ? __ffs(has) - 1 : 0);
        __syncwarp();
        // clear the edge bits and the source marks
        for (int c = 0; c < (n_tri + 31) / 32; ++c)
            if ((rem[c] >> lane) & 1u) {
                const uint32_t tv = m.tri[c * 32 + lane];
                const uint32_t a = tv & 255, b = (tv >> 8) & 255, d = (tv >> 16) & 255;
                clear_edge(a, b);
                clear_edge(b, d);
                clear_edge(d, a);
            }
        if (lane < PW) m.src_seen[lane] = 0u;
        if (clash || start < 0) {
            status = kCellBroken;
            __syncwarp();
            return;
        }
        // 4. walk the cycle
        int L = 0;
        if (lane == 0) {
            int a = start;
            do {
                m.cyc[L++] = (uint8_t)a;
                a = m.nxt[a];
            } while (a != start && L < MAXP);
            if (a != start) L = -1;
        }
        L = __shfl_sync(full, L, 0);
        __syncwarp();
        if (L != nbound || L < 3) {
            status = kCellBroken;
            return;
        }
        // 5. compact the kept vertices
        int kept = 0;
        for (int c = 0; c < (n_tri + 31) / 32; ++c) {
            const int t = c * 32 + lane;
            const unsigned valid = (n_tri - c * 32) >= 32 ? full : ((1u << (n_tri - c * 32)) - 1u);
            const unsigned keep = ~rem[c] & valid;
            uint32_t tv = 0;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            float vl = 0.f;
            const bool mine = (keep >> lane) & 1u;
            if (mine) {
                tv = m.tri[t];
                v = m.vtx[t];
                vl = m.vlen[t];
            }
            __syncwarp();
            if (mine) {
                const int dst = kept + __popc(keep & ((1u << lane) - 1u));
                m.tri[dst] = tv;
                m.vtx[dst] = v;
                m.vlen[dst] = vl;
            }
            kept += __popc(keep);
            __syncwarp();
        }
        if (kept + L > MAXT) {
            status = kCellOverflow;
            return;
        }
        // 6. close the hole: a fan of (cyc[j], cyc[j+1], q)
        for (int j = lane; j < L; j += 32) {
            const uint32_t a = m.cyc[j], b = m.cyc[(j + 1) % L];
            m.tri[kept + j] = a | b << 8 | (uint32_t)q << 16;
            put_vertex(kept + j, vertex_of(m.pl[a], m.pl[b], Q));
        }
        n_tri = kept + L;
        __syncwarp();
        // 7. planes that no vertex uses any more are redundant: free them;
        //    and the new radius
        uint32_t used[PW];
        for (int w = 0; w < PW; ++w) used[w] = 0u;
        for (int t = lane; t < n_tri; t += 32) {
            const uint32_t tv = m.tri[t];
            const uint32_t e[3] = {tv & 255, (tv >> 8) & 255, (tv >> 16) & 255};
#pragma unroll
            for (int j = 0; j < 3; ++j) used[e[j] >> 5] |= 1u << (e[j] & 31);
        }
        for (int w = 0; w < PW; ++w) {
            used[w] = __reduce_or_sync(full, used[w]);
            if (!((used[w] >> lane) & 1u)) m.pid[w * 32 + lane] = kFreeSlot;
        }
        update_bounds();
        __syncwarp();
    }

    // Every site not seen yet lies outside the block of grid cells c - s ..
    // c + s (the grid's own faces bound nothing: no site lies beyond).  A site
    // cuts the cell only if it lies inside the ball about some vertex v with
    // radius |v| (it is then closer to v than the site is), so the cell is
    // final once every such ball lies in the block.
    __device__ bool final_within(const int *c, const float3 &p, int s) {
        const float h = P.g.h, mg = 1e-5f * h;
        float blo[3], bhi[3];
        bool all = true;
        for (int a = 0; a < 3; ++a) {
            const float pa = a == 0 ? p.x : a == 1 ? p.y : p.z;
            blo[a] = c[a] - s > 0 ? P.g.lo[a] + (float)(c[a] - s) * h - pa + mg : -__int_as_float(0x7f800000);
            bhi[a] = c[a] + s < P.g.dims[a] - 1 ? P.g.lo[a] + (float)(c[a] + s + 1) * h - pa - mg
                                                 : __int_as_float(0x7f800000);
            all = all && c[a] - s <= 0 && c[a] + s >= P.g.dims[a] - 1;
        }
        if (all) return true;  // the block covers the grid
        bool inside = true;
        for (int t = lane; t < n_tri; t += 32) {
            const float4 v = m.vtx[t];
            const float r = m.vlen[t] + 2.f * v.w;
            inside = inside && v.x - r >= blo[0] && v.x + r <= bhi[0] && v.y - r >= blo[1] && v.y + r <= bhi[1] &&
                     v.z - r >= blo[2] && v.z + r <= bhi[2];
        }
        return __all_sync(0xffffffffu, inside);
    }

    // Offer one candidate per lane; cut by the qualifying ones nearest first.
    __device__ void offer(bool valid, int32_t k, const float3 &d, float d2, bool check_dup) {
        const unsigned full = 0xffffffffu;
        valid = valid && d2 > 0.f && d2 < 4.f * R2 && may_cut(d, d2);
        while (status == kCellOk) {
            const unsigned v = __ballot_sync(full, valid);
            if (!v) break;
            const unsigned key = valid ? __float_as_uint(d2) : 0xffffffffu;
            const unsigned mn = __reduce_min_sync(full, key);
            const int src = __ffs(__ballot_sync(full, valid && key == mn)) - 1;
            const int32_t kk = __shfl_sync(full, k, src);
            const float3 dd = make_float3(__shfl_sync(full, d.x, src), __shfl_sync(full, d.y, src),
                                          __shfl_sync(full, d.z, src));
            if (lane == src) valid = false;
            if (!check_dup || !has_site(kk)) cut(kk, dd);
            valid = valid && d2 < 4.f * R2 && may_cut(d, d2);
        }
    }
};

template <int MAXP, int WARPS, int MINB>
__global__ void __launch_bounds__(32 * WARPS, MINB) cell_kernel(const CellParams P) {
    __shared__ CellSmem<MAXP> smem[WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned full = 0xffffffffu;
    const int64_t n_items = P.site_list ? (int64_t)*P.n_list : P.n;
    const int64_t stride = (int64_t)gridDim.x * WARPS;
    for (int64_t item = (int64_t)blockIdx.x * WARPS + wid; item < n_items; item += stride) {
        const int32_t i = P.site_list ? P.site_list[item] : (int32_t)item;
        const float3 p = make_float3(P.pos[3 * (int64_t)i], P.pos[3 * (int64_t)i + 1], P.pos[3 * (int64_t)i + 2]);
        const double pi64[3] = {(double)p.x, (double)p.y, (double)p.z};
        Cell<MAXP> cell(smem[wid], P, lane, pi64);
        cell.init_box(p);
        // seeds: the previous neighbours (incremental rebuild)
        const bool seeded = P.seed_off != nullptr;
        if (seeded) {
            const int32_t b = P.seed_off[i], e = P.seed_off[i + 1];
            for (int32_t s = b; s < e && cell.status == kCellOk; s += 32) {
                const bool v = s + lane < e;
                const int32_t k = v ? P.seed_idx[s + lane] : -1;
                float3 d = make_float3(0.f, 0.f, 0.f);
                if (v) d = make_float3(P.pos[3 * (int64_t)k] - p.x, P.pos[3 * (int64_t)k + 1] - p.y,
                                       P.pos[3 * (int64_t)k + 2] - p.z);
                cell.offer(v && k != i, k, d, dot3f(d, d), true);
            }
        }
        // grid shells around the site's cell
        int c[3];
        const float pc[3] = {p.x, p.y, p.z};
        for (int a = 0; a < 3; ++a) {
            int v = (int)floorf((pc[a] - P.g.lo[a]) * P.g.inv_h);
            c[a] = v < 0 ? 0 : v >= P.g.dims[a] ? P.g.dims[a] - 1 : v;
        }
        const int smax = max(P.g.dims[0], max(P.g.dims[1], P.g.dims[2]));
        const float h = P.g.h;
        for (int s = 0; s <= smax && cell.status == kCellOk; ++s) {
            const int npairs = (2 * s + 1) * (2 * s + 1);
            for (int pi_ = 0; pi_ < npairs && cell.status == kCellOk; ++pi_) {
                int dz, dy;
                if (s <= 3) {
                    // pairs of shells 0..3 in the order of their distance (dz^2 + dy^2)
                    const int8_t *pr = kRowOrder[kRowStart[s] + pi_];
                    dz = pr[0];
                    dy = pr[1];
                } else {
                    dz = pi_ / (2 * s + 1) - s;
                    dy = pi_ % (2 * s + 1) - s;
                }
                if (max(abs(dz), abs(dy)) > s) continue;
                const int z = c[2] + dz;
                if (z < 0 || z >= P.g.dims[2]) continue;
                // distance from the site to the slab of cell layer z
                const float zl = P.g.lo[2] + (float)z * h - p.z, zh = zl + h;
                const float gz = fmaxf(0.f, fmaxf(zl, -zh));
                {
                    const int y = c[1] + dy;
                    if (y < 0 || y >= P.g.dims[1]) continue;
                    const float yl = P.g.lo[1] + (float)y * h - p.y, yh = yl + h;
                    const float gy = fmaxf(0.f, fmaxf(yl, -yh));
                    // only sites closer than 2 R can cut the cell: skip the row,
                    // or keep the cells of the row that reach the 2 R ball
                    const float reach2 = 4.f * cell.R2 - gy * gy - gz * gz;
                    if (!(reach2 > 0.f)) continue;
                    const float w = sqrtf(reach2) + 1e-5f * h;
                    const int rx0 = (int)floorf((p.x - w - P.g.lo[0]) * P.g.inv_h);
                    const int rx1 = (int)floorf((p.x + w - P.g.lo[0]) * P.g.inv_h);
                    const bool face = dz == -s || dz == s || dy == -s || dy == s;
                    // a full row of the shell, or its two end cells
                    for (int part = 0; part < (face ? 1 : 2); ++part) {
                        int x0, x1;
                        if (face) {
                            x0 = c[0] - s;
                            x1 = c[0] + s;
                        } else {
                            x0 = x1 = part == 0 ? c[0] - s : c[0] + s;
                        }
                        x0 = max(max(x0, 0), rx0);
                        x1 = min(min(x1, P.g.dims[0] - 1), rx1);
                        if (x0 > x1) continue;
                        const int64_t row = ((int64_t)z * P.g.dims[1] + y) * P.g.dims[0];
                        const int32_t b = P.g.cell_start[row + x0], e = P.g.cell_start[row + x1 + 1];
                        for (int32_t t = b; t < e && cell.status == kCellOk; t += 32) {
                            const bool v = t + lane < e;
                            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (v) q = P.g.sorted[t + lane];
                            const int32_t k = __float_as_int(q.w);
                            const float3 d = make_float3(q.x - p.x, q.y - p.y, q.z - p.z);
                            cell.offer(v && k != i, k, d, dot3f(d, d), seeded);
                        }
                    }
                }
            }
            if (cell.final_within(c, p, s)) break;
        }
        // the neighbours: site planes still holding a vertex
        if (cell.status == kCellOk) {
            int cnt = 0;
            for (int w = 0; w < MAXP / 32; ++w) cnt += __popc(__ballot_sync(full, smem[wid].pid[w * 32 + lane] >= 0));
            int32_t base = 0;
            if (lane == 0) base = atomicAdd(P.counters + 0, cnt);
            base = __shfl_sync(full, base, 0);
            if (base + cnt > P.edge_cap) {
                if (lane == 0) {
                    P.row_base[i] = 0;
                    P.row_cnt[i] = 0;
                }
            } else {
                int off = 0;
                for (int w = 0; w < MAXP / 32; ++w) {
                    const int32_t id = smem[wid].pid[w * 32 + lane];
                    const unsigned b = __ballot_sync(full, id >= 0);
                    if (id >= 0) P.edge_buf[base + off + __popc(b & ((1u << lane) - 1u))] = id;
                    off += __popc(b);
                }
                if (lane == 0) {
                    P.row_base[i] = base;
                    P.row_cnt[i] = cnt;
                }
            }
        } else if (lane == 0) {
            P.row_base[i] = 0;
            P.row_cnt[i] = 0;
            if (cell.status == kCellOverflow && P.wide_list) P.wide_list[atomicAdd(P.counters + 1, 1)] = i;
            else atomicAdd(P.counters + 2, 1);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Grid (counting sort of the sites by cell), symmetrisation and CSR assembly
// ---------------------------------------------------------------------------
__device__ __forceinline__ int fkey(float f) {
    const int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__host__ __device__ __forceinline__ float fkey_inv(int k) {
    const int b = k >= 0 ? k : k ^ 0x7fffffff;
    float f;
    memcpy(&f, &b, 4);
    return f;
}

__global__ void bbox_kernel(const float *__restrict__ pos, int64_t n, int32_t *keys, int32_t *bad) {
    int lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    int nonfinite = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < 3; ++a) {
            const float v = pos[3 * i + a];
            nonfinite |= !isfinite(v);
            const int k = fkey(v);
            lo[a] = min(lo[a], k);
            hi[a] = max(hi[a], k);
        }
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(keys + a, lo[a]);
            atomicMax(keys + 3 + a, hi[a]);
        }
    }
    if (nonfinite) atomicAdd(bad, 1);
}

struct Box6 {
    float v[6];
};

__global__ void grid_count_kernel(const float *__restrict__ pos, int64_t n, GridDev g, Box6 dom,
                                  int32_t *__restrict__ cell_of, int32_t *__restrict__ rank,
                                  int32_t *__restrict__ count, int32_t *outside) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c[3];
    for (int a = 0; a < 3; ++a) {
        const float v = pos[3 * i + a];
        if (!(v >= dom.v[a] && v <= dom.v[3 + a])) atomicAdd(outside, 1);
        int k = (int)floorf((v - g.lo[a]) * g.inv_h);
        c[a] = k < 0 ? 0 : k >= g.dims[a] ? g.dims[a] - 1 : k;
    }
    const int32_t cell = (c[2] * g.dims[1] + c[1]) * g.dims[0] + c[0];
    cell_of[i] = cell;
    rank[i] = atomicAdd(count + cell, 1);
}

__global__ void grid_scatter_kernel(const float *__restrict__ pos, int64_t n, const int32_t *__restrict__ cell_of,
                                    const int32_t *__restrict__ rank, const int32_t *__restrict__ start,
                                    float4 *__restrict__ sorted) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    sorted[start[cell_of[i]] + rank[i]] =
        make_float4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], __int_as_float((int32_t)i));
}

// exclusive scan of int32 counts (3 kernels: tiles, tile totals, offsets)
__global__ void __launch_bounds__(kScanThreads) iscan_tiles_kernel(const int32_t *__restrict__ in, int64_t n,
                                                                   int32_t *__restrict__ out, int32_t *__restrict__ sums) {
    __shared__ int32_t part[kScanThreads];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems], acc = 0;
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = acc;
        acc += base + k < n ? in[base + k] : 0;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
        const int32_t add = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += add;
        __syncthreads();
    }
    const int32_t before = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) out[base + k] = before + v[k];
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = part[threadIdx.x];
}

__global__ void __launch_bounds__(kScanThreads) iscan_sums_kernel(int32_t *__restrict__ sums, int64_t nb) {
    __shared__ int32_t part[kScanThreads];
    const int64_t base = (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems], acc = 0;
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = acc;
        acc += base + k < nb ? sums[base + k] : 0;
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 1; o < kScanThreads; o <<= 1) {
        const int32_t add = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += add;
        __syncthreads();
    }
    const int32_t before = threadIdx.x ? part[threadIdx.x - 1] : 0;
    __syncthreads();
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < nb) sums[base + k] = before + v[k];
    if (threadIdx.x == kScanThreads - 1) sums[nb] = part[threadIdx.x];
}

__global__ void iscan_add_kernel(int32_t *__restrict__ out, int64_t n, const int32_t *__restrict__ sums) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] += sums[e / kScanTile];
    if (e == n) out[n] = sums[(n + kScanTile - 1) / kScanTile];  // the total
}

// j lists i but i does not list j: record the missing reverse edge (j <- i)
__global__ void symmetry_kernel(int64_t n, const int32_t *__restrict__ base, const int32_t *__restrict__ cnt,
                                const int32_t *__restrict__ buf, int32_t *__restrict__ extra_cnt,
                                int2 *__restrict__ extra, int32_t cap, int32_t *counters) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t e = 0; e < cnt[i]; ++e) {
        const int32_t j = buf[base[i] + e];
        bool found = false;
        for (int32_t f = 0; f < cnt[j] && !found; ++f) found = buf[base[j] + f] == (int32_t)i;
        if (!found) {
            const int32_t slot = atomicAdd(counters + 4, 1);
            if (slot < cap) {
                extra[slot] = make_int2(j, (int32_t)i);
                atomicAdd(extra_cnt + j, 1);
            }
        }
    }
}

__global__ void row_total_kernel(int64_t n, const int32_t *__restrict__ cnt, const int32_t *__restrict__ extra_cnt,
                                 int32_t *__restrict__ total, int32_t *counters) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    total[i] = cnt[i] + extra_cnt[i];
    atomicMax(counters + 5, total[i]);
}

__global__ void fill_kernel(int64_t n, const int32_t *__restrict__ base, const int32_t *__restrict__ cnt,
                            const int32_t *__restrict__ buf, const int32_t *__restrict__ off,
                            int32_t *__restrict__ idx, int32_t *__restrict__ cursor) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t o = off[i];
    for (int32_t e = 0; e < cnt[i]; ++e) idx[o + e] = buf[base[i] + e];
    cursor[i] = o + cnt[i];
}

__global__ void fill_extra_kernel(const int2 *__restrict__ extra, const int32_t *counters, int32_t cap,
                                  int32_t *__restrict__ idx, int32_t *__restrict__ cursor) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t m = min(counters[4], cap);
    if (k >= m) return;
    const int2 e = extra[k];
    idx[atomicAdd(cursor + e.x, 1)] = e.y;
}

__global__ void sort_rows_kernel(int64_t n, const int32_t *__restrict__ off, int32_t *__restrict__ idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t *r = idx + off[i];
    const int32_t m = off[i + 1] - off[i];
    for (int32_t a = 1; a < m; ++a) {
        const int32_t v = r[a];
        int32_t b = a - 1;
        while (b >= 0 && r[b] > v) {
            r[b + 1] = r[b];
            --b;
        }
        r[b + 1] = v;
    }
}

}  // namespace
}  // namespace rf

using namespace rf;

struct rf_adjacency {
    int64_t n = 0;                  // sites of the current result
    rf_adjacency_stats stats{};
    int32_t *off = nullptr;         // [N + 1] current result
    int32_t *idx = nullptr;
    // workspace, grown on demand
    int64_t site_cap = 0;
    int32_t *cell_of = nullptr, *rank = nullptr, *row_base = nullptr, *row_cnt = nullptr;
    int32_t *extra_cnt = nullptr, *total = nullptr, *cursor = nullptr, *wide = nullptr;
    float4 *sorted = nullptr;
    int64_t cell_cap = 0;
    int32_t *cell_count = nullptr, *cell_start = nullptr;   // [ncell + 1]
    int64_t edge_cap = 0;
    int32_t *edge_buf = nullptr;
    int64_t extra_cap = 0;
    int2 *extra = nullptr;
    int64_t scan_cap = 0;
    int32_t *scan_sums = nullptr;
    int32_t *counters = nullptr;    // [8]
    int32_t *bbox = nullptr;        // [7]: float keys of the sites' box, non-finite count
    int32_t *host = nullptr;        // pinned [16]
};

namespace {

template <typename T>
rf_status grow(T **p, int64_t *cap, int64_t need, const char *what) {
    if (need <= *cap && *p) return RF_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    const int64_t n = need + need / 8 + 64;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (size_t)n);
    if (e != cudaSuccess) return cuda_fail(e, what);
    *cap = n;
    return RF_OK;
}

rf_status scan(rf_adjacency *a, const int32_t *in, int64_t n, int32_t *out, cudaStream_t st) {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb > kScanTile) return fail(RF_ERR_INVALID_ARG, "scan of %lld items is too long", (long long)n);
    int64_t cap = a->scan_cap;
    rf_status rc = grow(&a->scan_sums, &cap, nb + 1, "scan workspace");
    if (rc != RF_OK) return rc;
    a->scan_cap = cap;
    iscan_tiles_kernel<<<(unsigned)std::max<int64_t>(nb, 1), kScanThreads, 0, st>>>(in, n, out, a->scan_sums);
    iscan_sums_kernel<<<1, kScanThreads, 0, st>>>(a->scan_sums, nb);
    iscan_add_kernel<<<(unsigned)((n + 1 + 255) / 256), 256, 0, st>>>(out, n, a->scan_sums);
    RF_CUDA(cudaGetLastError());
    return RF_OK;
}

struct Freer {  // frees a pair of fresh result arrays unless released
    int32_t *p = nullptr, *q = nullptr;
    ~Freer() {
        if (p) cudaFree(p);
        if (q) cudaFree(q);
    }
};

}  // namespace

RF_API rf_status rf_adjacency_create(rf_adjacency **out) {
    if (!out) return fail(RF_ERR_INVALID_ARG, "out is NULL");
    rf_adjacency *a = new rf_adjacency();
    cudaError_t e;
    if ((e = cudaMalloc((void **)&a->counters, sizeof(int32_t) * 8)) != cudaSuccess ||
        (e = cudaMalloc((void **)&a->bbox, sizeof(int32_t) * 8)) != cudaSuccess ||
        (e = cudaMallocHost((void **)&a->host, sizeof(int32_t) * 16)) != cudaSuccess) {
        rf_adjacency_destroy(a);
        return cuda_fail(e, "adjacency create");
    }
    *out = a;
    return RF_OK;
}

RF_API rf_status rf_adjacency_destroy(rf_adjacency *a) {
    if (!a) return RF_OK;
    for (void *p : {(void *)a->off, (void *)a->idx, (void *)a->cell_of, (void *)a->rank, (void *)a->row_base,
                    (void *)a->row_cnt, (void *)a->extra_cnt, (void *)a->total, (void *)a->cursor, (void *)a->wide,
                    (void *)a->sorted, (void *)a->cell_count, (void *)a->cell_start, (void *)a->edge_buf,
                    (void *)a->extra, (void *)a->scan_sums, (void *)a->counters, (void *)a->bbox})
        if (p) cudaFree(p);
    if (a->host) cudaFreeHost(a->host);
    delete a;
    return RF_OK;
}

RF_API rf_status rf_adjacency_build(rf_adjacency *a, int64_t n, const float *pos, const float *domain6,
                                    int32_t incremental, void *stream) {
    if (!a || !pos) return fail(RF_ERR_INVALID_ARG, "adjacency and pos are required");
    // the lists are int32 CSR: ~16 edges per site keeps 10^8 sites below 2^31 edges
    if (n < 1 || n > 100000000) return fail(RF_ERR_INVALID_ARG, "n_sites must be in [1, 10^8]");
    if (incremental && (a->n != n || !a->off))
        return fail(RF_ERR_INVALID_ARG, "an incremental rebuild needs a previous build of as many sites");
    cudaStream_t st = (cudaStream_t)stream;
    rf_status rc;
    // per-site workspace
    if (n + 1 > a->site_cap) {
        int64_t cap = 0;
        for (int32_t **p : {&a->cell_of, &a->rank, &a->row_base, &a->row_cnt, &a->extra_cnt, &a->total,
                            &a->cursor, &a->wide}) {
            cap = 0;
            if ((rc = grow(p, &cap, n + 1, "adjacency site arrays")) != RF_OK) return rc;
        }
        int64_t c2 = 0;
        if ((rc = grow(&a->sorted, &c2, n + 1, "adjacency sorted sites")) != RF_OK) return rc;
        a->site_cap = std::min(cap, c2);
    }
    // 1. the sites' box (one wait), and the domain: the caller's, or that box
    //    grown by 5% of its extent (at least 1e-3) on every side
    const int32_t init[7] = {INT32_MAX, INT32_MAX, INT32_MAX, INT32_MIN, INT32_MIN, INT32_MIN, 0};
    RF_CUDA(cudaMemcpyAsync(a->bbox, init, sizeof init, cudaMemcpyHostToDevice, st));
    bbox_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, grid_cap(8)), 256, 0, st>>>(pos, n, a->bbox, a->bbox + 6);
    RF_CUDA(cudaGetLastError());
    RF_CUDA(cudaMemcpyAsync(a->host, a->bbox, sizeof init, cudaMemcpyDeviceToHost, st));
    RF_CUDA(cudaStreamSynchronize(st));
    if (a->host[6]) return fail(RF_ERR_INVALID_ARG, "site positions must be finite");
    Box6 dom;
    if (domain6) {
        for (int k = 0; k < 6; ++k) dom.v[k] = domain6[k];
        for (int k = 0; k < 3; ++k)
            if (!(dom.v[k] < dom.v[3 + k]) || !std::isfinite(dom.v[k]) || !std::isfinite(dom.v[3 + k]))
                return fail(RF_ERR_INVALID_ARG, "domain must hold finite min < max");
    } else {
        for (int k = 0; k < 3; ++k) {
            const double lo = fkey_inv(a->host[k]), hi = fkey_inv(a->host[3 + k]);
            const double m = std::max(0.05 * (hi - lo), 1e-3);
            dom.v[k] = (float)(lo - m);
            dom.v[3 + k] = (float)(hi + m);
        }
    }
    for (int k = 0; k < 3; ++k)
        if (fkey_inv(a->host[k]) < dom.v[k] || fkey_inv(a->host[3 + k]) > dom.v[3 + k])
            return fail(RF_ERR_INVALID_ARG, "every site must lie inside the domain box");
    // 2. uniform grid over the domain, about two sites per cell
    GridDev g{};
    double ext[3], vol = 1.0;
    for (int k = 0; k < 3; ++k) {
        ext[k] = (double)dom.v[3 + k] - dom.v[k];
        vol *= ext[k];
    }
    double h = std::cbrt(vol * 2.0 / (double)n);
    h = std::max({h, ext[0] / 1024.0, ext[1] / 1024.0, ext[2] / 1024.0});
    int64_t ncell = 1;
    for (int k = 0; k < 3; ++k) {
        g.dims[k] = (int)std::max(1.0, std::ceil(ext[k] / h));
        g.lo[k] = dom.v[k];
        ncell *= g.dims[k];
    }
    g.h = (float)h;
    g.inv_h = (float)(1.0 / h);
    {
        int64_t c1 = a->cell_cap, c2 = a->cell_cap;
        if ((rc = grow(&a->cell_count, &c1, ncell + 1, "adjacency grid")) != RF_OK) return rc;
        if ((rc = grow(&a->cell_start, &c2, ncell + 1, "adjacency grid")) != RF_OK) return rc;
        a->cell_cap = std::min(c1, c2);
    }
    RF_CUDA(cudaMemsetAsync(a->cell_count, 0, sizeof(int32_t) * (size_t)(ncell + 1), st));
    RF_CUDA(cudaMemsetAsync(a->counters, 0, sizeof(int32_t) * 8, st));
    grid_count_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pos, n, g, dom, a->cell_of, a->rank, a->cell_count,
                                                                     a->counters + 7);
    RF_CUDA(cudaGetLastError());
    if ((rc = scan(a, a->cell_count, ncell, a->cell_start, st)) != RF_OK) return rc;
    grid_scatter_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pos, n, a->cell_of, a->rank, a->cell_start,
                                                                       a->sorted);
    RF_CUDA(cudaGetLastError());
    g.sorted = a->sorted;
    g.cell_start = a->cell_start;
    // 3. the cells (edge buffer sized for a mean degree of 24; regrown and
    //    rebuilt once if short)
    for (int attempt = 0; attempt < 2; ++attempt) {
        {
            int64_t cap = a->edge_cap;
            if ((rc = grow(&a->edge_buf, &cap, std::max<int64_t>(24 * n, a->edge_cap), "adjacency edges")) != RF_OK)
                return rc;
            a->edge_cap = cap;
        }
        RF_CUDA(cudaMemsetAsync(a->counters, 0, sizeof(int32_t) * 7, st));
        CellParams P{};
        P.pos = pos;
        P.n = n;
        P.g = g;
        for (int k = 0; k < 6; ++k) P.dom[k] = dom.v[k];
        P.seed_off = incremental ? a->off : nullptr;
        P.seed_idx = incremental ? a->idx : nullptr;
        P.row_base = a->row_base;
        P.row_cnt = a->row_cnt;
        P.edge_buf = a->edge_buf;
        P.edge_cap = (int32_t)std::min<int64_t>(a->edge_cap, INT32_MAX);
        P.counters = a->counters;
        P.wide_list = a->wide;
        const int64_t blocks = std::min<int64_t>((n + kWarps - 1) / kWarps, grid_cap(256));
        cell_kernel<kMaxPlanes, kWarps, 7><<<(unsigned)blocks, 32 * kWarps, 0, st>>>(P);
        RF_CUDA(cudaGetLastError());
        // the cells that overflowed, again with room for more faces
        P.site_list = a->wide;
        P.n_list = a->counters + 1;
        P.wide_list = nullptr;
        cell_kernel<kWideMaxPlanes, kWideWarps, 1><<<grid_cap(8), 32 * kWideWarps, 0, st>>>(P);
        RF_CUDA(cudaGetLastError());
        RF_CUDA(cudaMemcpyAsync(a->host, a->counters, sizeof(int32_t) * 8, cudaMemcpyDeviceToHost, st));
        RF_CUDA(cudaStreamSynchronize(st));
        if (a->host[7]) return fail(RF_ERR_INVALID_ARG, "%d site coordinates lie outside the domain box", a->host[7]);
        if ((int64_t)a->host[0] <= a->edge_cap) break;
        if (attempt == 1) return fail(RF_ERR_OOM, "adjacency edge buffer overflow");
        int64_t cap = 0;
        if ((rc = grow(&a->edge_buf, &cap, (int64_t)a->host[0] + n, "adjacency edges")) != RF_OK) return rc;
        a->edge_cap = cap;
    }
    a->stats.wide_sites = a->host[1];
    a->stats.failed_sites = a->host[2];
    a->stats.fp64_tests = a->host[3];
    a->stats.edges_before_symmetry = a->host[0];
    // 4. symmetric lists: the reverse of every one-sided edge is added
    {
        int64_t cap = a->extra_cap;
        if ((rc = grow(&a->extra, &cap, std::max<int64_t>(n / 4, 1024), "adjacency extra edges")) != RF_OK) return rc;
        a->extra_cap = cap;
    }
    RF_CUDA(cudaMemsetAsync(a->extra_cnt, 0, sizeof(int32_t) * (size_t)n, st));
    symmetry_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a->row_base, a->row_cnt, a->edge_buf, a->extra_cnt,
                                                                   a->extra, (int32_t)a->extra_cap, a->counters);
    row_total_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a->row_cnt, a->extra_cnt, a->total, a->counters);
    RF_CUDA(cudaGetLastError());
    // 5. CSR into fresh arrays (the previous result served as the seeds)
    Freer fresh;
    int64_t cap = 0;
    if ((rc = grow(&fresh.p, &cap, n + 1, "adjacency offsets")) != RF_OK) return rc;
    if ((rc = scan(a, a->total, n, fresh.p, st)) != RF_OK) return rc;
    RF_CUDA(cudaMemcpyAsync(a->host, fresh.p + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RF_CUDA(cudaMemcpyAsync(a->host + 1, a->counters + 4, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, st));
    RF_CUDA(cudaStreamSynchronize(st));
    const int64_t n_edges = a->host[0];
    if (a->host[1] > a->extra_cap)
        return fail(RF_ERR_BAD_SCENE, "%d one-sided edges: the sites are too degenerate", a->host[1]);
    cap = 0;
    if ((rc = grow(&fresh.q, &cap, std::max<int64_t>(n_edges, 1), "adjacency ids")) != RF_OK) return rc;
    fill_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a->row_base, a->row_cnt, a->edge_buf, fresh.p, fresh.q,
                                                              a->cursor);
    fill_extra_kernel<<<(unsigned)((std::max<int64_t>(a->host[1], 1) + 255) / 256), 256, 0, st>>>(
        a->extra, a->counters, (int32_t)a->extra_cap, fresh.q, a->cursor);
    sort_rows_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, fresh.p, fresh.q);
    RF_CUDA(cudaGetLastError());
    RF_CUDA(cudaStreamSynchronize(st));
    if (a->off) cudaFree(a->off);
    if (a->idx) cudaFree(a->idx);
    a->off = fresh.p;
    a->idx = fresh.q;
    fresh.p = fresh.q = nullptr;
    a->n = n;
    a->stats.n_sites = n;
    a->stats.n_edges = n_edges;
    a->stats.max_degree = a->host[2];
    a->stats.asym_added = a->host[1];
    for (int k = 0; k < 6; ++k) a->stats.domain[k] = dom.v[k];
    return RF_OK;
}

RF_API rf_status rf_adjacency_result(rf_adjacency *a, const int32_t **adj_off, const int32_t **adj_idx,
                                     rf_adjacency_stats *stats) {
    if (!a) return fail(RF_ERR_INVALID_ARG, "adjacency is NULL");
    if (!a->off) return fail(RF_ERR_NOT_READY, "no adjacency built yet");
    if (adj_off) *adj_off = a->off;
    if (adj_idx) *adj_idx = a->idx;
    if (stats) *stats = a->stats;
    return RF_OK;
}

RF_API rf_status rf_adjacency_copy(rf_adjacency *a, int32_t *adj_off, int32_t *adj_idx, void *stream) {
    if (!a || !adj_off || (!adj_idx && a->stats.n_edges > 0)) return fail(RF_ERR_INVALID_ARG, "adjacency and outputs are required");
    if (!a->off) return fail(RF_ERR_NOT_READY, "no adjacency built yet");
    cudaStream_t st = (cudaStream_t)stream;
    RF_CUDA(cudaMemcpyAsync(adj_off, a->off, sizeof(int32_t) * (size_t)(a->n + 1), cudaMemcpyDeviceToDevice, st));
    if (a->stats.n_edges > 0)
        RF_CUDA(cudaMemcpyAsync(adj_idx, a->idx, sizeof(int32_t) * (size_t)a->stats.n_edges, cudaMemcpyDeviceToDevice, st));
    return RF_OK;
}
