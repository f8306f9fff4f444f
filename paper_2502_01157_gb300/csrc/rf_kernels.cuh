// rf_kernels.cuh -- forward, backward and trace kernels of the Radiant Foam
// renderer (arXiv 2502.01157) for sm_103a, templated on the attribute type,
// the SH degree, the output mode and FX.  FX kernels handle the ray-based
// effects of Fig. 2 -- fisheye cameras, rolling shutters and an analytic
// sphere met in the walk -- and the others only pinhole, global-shutter
// cameras without a sphere, so that the common path keeps its registers.
// rf_render.cu instantiates the plain kernels and rf_effects.cu the FX ones,
// so the two halves compile in parallel.
//
// One thread per ray.  A block renders a 16x8 pixel tile of one camera; each
// warp owns an 8x4 patch, so the rays of a warp enter mostly the same cells
// and their face loads hit the same L1 lines.  Tiles of all cameras of a call
// form one grid (multi-camera batches are one launch).
#pragma once

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
    float *quantile;    // [R] (mode kQuant)
    float *qaux;        // [R][5]: D, Q, W, Z1, Z2 (mode kQuant)
};

enum { kPlain = 0, kTrace = 1, kQuant = 2 };

// Forward: Alg. 1 per ray with Eq. (3)-(4) compositing; in mode kQuant the
// same walk also accumulates the quantile loss of Eq. (6).  With FX the walk
// meets the sphere of p.fx (if max_bounces > 0): a hit ends the segment, bends
// the ray and the walk carries on from the same cell (depth then measures the
// bent path).
template <typename AT, int DEG, int MODE, bool FX>
__global__ void __launch_bounds__(kBlock, FX ? 6 : 8) fwd_kernel(const RenderParams p, const FwdOut out) {
    constexpr bool TRACE = MODE == kTrace;
    constexpr bool QUANT = MODE == kQuant;
    const PixelTask px = pixel_of_thread(p.lc);
    if (!px.valid) return;
    const rf_camera &cam = p.lc.cam[px.cam];
    float3 o, d;
    camera_ray<FX>(cam, px.u, px.v, o, d);
    const int64_t r = p.lc.ray_begin[px.cam] + (int64_t)px.v * cam.width + px.u;

    float C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f, T = 1.f;
    float qP = 0.f, qQ = 0.f, qW = 0.f, qZ1 = 0.f, qZ2 = 0.f;  // quantile-loss sums
    int steps = 0;
    uint8_t st = RF_RAY_OK;
    float tmin, tmax;
    if (ray_interval(o, d, p.s, cam.t_near, cam.t_far, tmin, tmax)) {
        float Y[16];
        sh_basis<DEG>(d, Y);
        int i = start_cell<FX>(p, px.cam, o);
        float t0 = 0.f;
        FxRay f;
        if constexpr (FX) fx_begin(p.fx, o, d, f);
        // this lane's column of its warp's segment record
        uint32_t *rec = TRACE ? nullptr : record_column(p);
        while (T > p.eps) {
            if (steps >= p.max_steps) {
                st = RF_RAY_MAX_STEPS;
                break;
            }
            const CellHdr cell = load_cell(p.s, i);
            Segment g;
            float3 oc;
            cell_step<AT, DEG, FX>(p.s, i, cell, o, d, t0, tmin, tmax, Y, g, oc, FX ? f.ts : 0.f);
            if (rec && steps < p.rec_steps) record_store(rec, steps, g);
            if (TRACE && steps < out.max_trace) out.trace[r * out.max_trace + steps] = i;
            const float alpha = __fsub_rn(1.f, g.e);
            const float w = __fmul_rn(T, alpha);
            C0 = __fmaf_rn(w, fmaxf(g.pre[0], 0.f), C0);
            C1 = __fmaf_rn(w, fmaxf(g.pre[1], 0.f), C1);
            C2 = __fmaf_rn(w, fmaxf(g.pre[2], 0.f), C2);
            float z = __fmul_rn(0.5f, __fadd_rn(g.a, g.b));
            if constexpr (FX) z = __fadd_rn(f.soff, z);
            D = __fmaf_rn(w, z, D);
            if (QUANT && g.delta > 0.f) {
                const QuantSeg q = quant_seg(g.sigma, g.delta, g.e);
                qQ += qW * g.delta + T * q.f1d;                            // int W
                qP += qW * (qW * g.delta + 2.f * T * q.f1d) + T * T * q.f2d;  // int W^2
                qZ1 += T * ((1.f - 2.f * T) * q.A + 2.f * T * q.C);
                qZ2 += T * q.A;
                qW += T * q.alpha;                                         // weight so far
            }
            T = __fmul_rn(T, g.e);
            ++steps;
            if (FX && g.hit) {
                if (!fx_bounce(p.fx, p.s, f, o, d, tmin, tmax)) break;
                sh_basis<DEG>(d, Y);
                t0 = 0.f;
                continue;  // the new leg starts in the same cell
            }
            if (g.next < 0 || !(g.t1 < tmax)) break;
            t0 = g.t1 > t0 ? g.t1 : t0;
            i = g.next;
        }
    }
    if (QUANT) {
        const float qD = qW * qQ - qP;  // int W (W_tot - W) dt = int (1 - T)(T - T_f) dt
        out.quantile[r] = qW > 0.f ? 2.f * qD / (qW * qW) : 0.f;
        float *a = out.qaux + 5 * r;
        a[0] = qD;
        a[1] = qQ;
        a[2] = qW;
        a[3] = qZ1;
        a[4] = qZ2;
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
    float4 *g_acc;   // [n_sites] {position x, y, z, density} gradient sums, added
                     // to g_pos / g_density after the launch (null: neither is wanted)
    const float *qaux, *d_quantile;
};

// Backward: every ray is walked again, step by step.  A step the forward's
// segment record holds is rebuilt from it (exit, density, colour before the
// clamp); any other step (all of them without a record) searches the faces
// and reads the attributes with the forward's arithmetic, so both meet the
// same bits.  Per segment the adjoints follow from the stored final colour,
// transmittance and depth (C_rest = C_final - C_incl).
//
// Scatter.  Neighbouring rays of a warp mostly walk the same cells (a warp of
// an 8x4 patch meets ~5-7 distinct cells per iteration at 1920x1080 and reuses
// each ~25 times over its walk), so per-lane atomics would hit the same
// addresses many times.  Each iteration the lanes stage their contributions to
// the current cell (SH row, {position, density}) in shared memory; lanes in
// the same cell are summed column-wise and the sums are added with 16-byte
// vector atomics: the SH row into g_sh, the site terms into the
// {x, y, z, density} accumulator g_acc that a final pass adds to g_pos and
// g_density.  The rows of lanes alone in their cell are spread over the warp,
// one 16-byte column per lane.  The crossing that entered the cell also moves
// the previous cell's site; each lane adds those three terms to g_acc itself.
constexpr int kMaxGroups = 8;

// SHARED: the crossing terms of the previous cell (below) are summed over the
// lanes that share that cell before their atomic, in warp iterations whose
// live lanes are in at most kSharedCells distinct cells.  Where many rays cross
// the same cells (large cells, cameras far from the foam) this removes most
// same-address atomics, which the L2 serialises; on dense foams (~4 lanes per
// cell) the extra code costs more than it saves, so it is a separate kernel.
constexpr int kSharedCells = 2;

template <typename AT, int DEG, bool QUANT, bool FX, bool SHARED>
__global__ void __launch_bounds__(kBlock, 6) bwd_kernel(const RenderParams p, const BwdIO io) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int NV = 3 * K;              // SH gradient row
    constexpr int NVP = (NV + 3) / 4 * 4;  // padded to whole 16-byte columns
    constexpr int VP = NVP + 4;            // + {position of the cell, density}
    // row stride: a multiple of 4 floats (16-byte row stores) whose quarter is
    // odd, so the 8 lanes of a 128-bit store phase hit 8 different bank quads;
    // a column read (one row, consecutive columns) is conflict-free for any stride
    constexpr int SP = ((VP / 4) % 2 == 1) ? VP : VP + 4;
    // one row per lane (+ a zero row that absent members read in the FX kernels)
    constexpr int ROWS = FX ? 33 : 32;
    __shared__ __align__(16) float stage_all[kBlock / 32][ROWS * SP];
    // the lanes whose row is alone this iteration, and their cells, by rank
    __shared__ int alone_lane_all[kBlock / 32][32];
    __shared__ int alone_cell_all[kBlock / 32][32];
    const int lane = threadIdx.x & 31;
    float *stage = stage_all[threadIdx.x >> 5];
    int *alone_lane = alone_lane_all[threadIdx.x >> 5];
    int *alone_cell = alone_cell_all[threadIdx.x >> 5];
    const unsigned full = 0xffffffffu;
    if constexpr (FX) {
        for (int c = lane; c < SP; c += 32) stage[32 * SP + c] = 0.f;
        __syncwarp();
    }

    // per-lane set-up; no early return: every lane takes part in the
    // warp-wide scatter until the whole warp is done
    const PixelTask px = pixel_of_thread(p.lc);
    bool live = px.valid;
    float3 o = make_float3(0.f, 0.f, 0.f), d = make_float3(0.f, 0.f, 1.f);
    float tmin = 0.f, tmax = 0.f;
    int64_t r = 0;
    if (live) {
        const rf_camera &cam = p.lc.cam[px.cam];
        camera_ray<FX>(cam, px.u, px.v, o, d);
        r = p.lc.ray_begin[px.cam] + (int64_t)px.v * cam.width + px.u;
        live = ray_interval(o, d, p.s, cam.t_near, cam.t_far, tmin, tmax);
    }
    float gC[3] = {0.f, 0.f, 0.f}, gT = 0.f, gD = 0.f, Cf[3] = {0.f, 0.f, 0.f}, Tf = 0.f, Df = 0.f;
    if (live) {
        gC[0] = io.d_rgb[3 * r];
        gC[1] = io.d_rgb[3 * r + 1];
        gC[2] = io.d_rgb[3 * r + 2];
        gT = io.d_trans ? io.d_trans[r] : 0.f;
        gD = io.d_depth ? io.d_depth[r] : 0.f;
        live = !(gC[0] == 0.f && gC[1] == 0.f && gC[2] == 0.f && gT == 0.f && gD == 0.f);
        if (QUANT) live = live || io.d_quantile[r] != 0.f;
        Cf[0] = io.rgb[3 * r];
        Cf[1] = io.rgb[3 * r + 1];
        Cf[2] = io.rgb[3 * r + 2];
        Tf = io.trans[r];
        Df = io.depth ? io.depth[r] : 0.f;
    }
    // quantile loss L = 2 (P - T_f Q) / W^2: per-segment adjoints from the
    // forward's sums; suffix sums of Z1 + T_f Z2 carry the dependence of the
    // later segments on this segment's transmittance factor
    float gQ = 0.f, qk2 = 0.f, qdTf = 0.f, qZ1 = 0.f, qZ2 = 0.f, qW = 0.f;
    if (QUANT && live) {
        gQ = io.d_quantile[r];
        const float *a = io.qaux + 5 * r;
        qW = a[2];
        if (gQ != 0.f && qW > 0.f) {
            qk2 = 2.f / (qW * qW);
            qdTf = -qk2 * a[1] + 2.f * qk2 * a[0] / qW;  // dL/dT_f at fixed P, Q (a[0] = P - T_f Q)
            qZ1 = a[3];
            qZ2 = a[4];
        } else {
            gQ = 0.f;
        }
    }
    float qWn = 0.f;  // weight before the current segment
    float Y[16];
    sh_basis<DEG>(d, Y);
    int i = live ? start_cell<FX>(p, px.cam, o) : 0;
    FxRay f;
    if constexpr (FX) fx_begin(p.fx, o, d, f);
    // the forward's segment record of this warp (lane column), if given
    const uint32_t *rec = record_column(p);
    if (kRecAhead > 0 && rec && lane == 0) record_prefetch(p, 0, 2 * kRecAhead);
    int it = 0;  // warp iteration: step k of a live lane is iteration k
    float t0 = 0.f, T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f;
    int steps = 0;
    // the crossing that entered the current cell: (pa -> i) at pt; its adjoint
    // padj is complete once the current segment's t0 adjoint is known
    bool pend = false, pend_defines = false;
    int pa = -1;
    float3 pxa = make_float3(0.f, 0.f, 0.f), poca = pxa;
    float pt = 0.f, padj = 0.f;
    // the crossing that set the current t0 (t0 <- max(t0, t1))
    int da = -1, db = -1;
    float dt = 0.f;

    while (__any_sync(full, live)) {
        if constexpr (kRecAhead > 0) {
            if (rec && lane == 0 && it > 0 && it % kRecAhead == 0) record_prefetch(p, it + kRecAhead, kRecAhead);
        }
        ++it;
        // stop tests of Alg. 1 (before the step); a crossing still pending
        // (T fell to eps right after it) is scattered by this lane alone
        if (live && (!(T > p.eps) || steps >= p.max_steps)) {
            live = false;
            if (pend && padj != 0.f && io.g_pos) {
                const CellHdr cb = load_cell(p.s, i);
                const float3 xb = make_float3(cb.x, cb.y, cb.z);
                const float nx = xb.x - pxa.x, ny = xb.y - pxa.y, nz = xb.z - pxa.z;
                const float s_ = padj / (nx * d.x + ny * d.y + nz * d.z);
                const float qx = poca.x + pt * d.x, qy = poca.y + pt * d.y, qz = poca.z + pt * d.z;
                atomicAdd(io.g_pos + 3 * (int64_t)pa + 0, s_ * qx);
                atomicAdd(io.g_pos + 3 * (int64_t)pa + 1, s_ * qy);
                atomicAdd(io.g_pos + 3 * (int64_t)pa + 2, s_ * qz);
                atomicAdd(io.g_pos + 3 * (int64_t)i + 0, s_ * (nx - qx));
                atomicAdd(io.g_pos + 3 * (int64_t)i + 1, s_ * (ny - qy));
                atomicAdd(io.g_pos + 3 * (int64_t)i + 2, s_ * (nz - qz));
            }
        }
        float sig_bar = 0.f, cb[3] = {0.f, 0.f, 0.f};
        float gpos_i[3] = {0.f, 0.f, 0.f}, gpos_a[3] = {0.f, 0.f, 0.f};
        int key_prev = -1;
        Segment g;
        CellHdr cell;
        float3 oc = make_float3(0.f, 0.f, 0.f);
        if (live) {
            cell = load_cell(p.s, i);
            if (rec && steps < p.rec_steps)
                record_step<FX>(p.s, rec, steps, cell, o, t0, tmin, tmax, g, oc, FX ? f.ts : 0.f);
            else
                cell_step<AT, DEG, FX>(p.s, i, cell, o, d, t0, tmin, tmax, Y, g, oc, FX ? f.ts : 0.f);
            const float alpha = __fsub_rn(1.f, g.e);
            const float w = __fmul_rn(T, alpha);
            const float c[3] = {fmaxf(g.pre[0], 0.f), fmaxf(g.pre[1], 0.f), fmaxf(g.pre[2], 0.f)};
            float z = __fmul_rn(0.5f, __fadd_rn(g.a, g.b));
            if constexpr (FX) z = __fadd_rn(f.soff, z);
            C0 = __fmaf_rn(w, c[0], C0);
            C1 = __fmaf_rn(w, c[1], C1);
            C2 = __fmaf_rn(w, c[2], C2);
            D = __fmaf_rn(w, z, D);
            const float Tn = __fmul_rn(T, g.e);
            // dL/dsigma_n = delta_n * B, dL/ddelta_n = sigma_n * B with
            // B = g_C.(T_{n+1} c_n - C_rest) - g_T T_final + g_D (T_{n+1} z_n - D_rest)
            const float B = gC[0] * (Tn * c[0] - (Cf[0] - C0)) + gC[1] * (Tn * c[1] - (Cf[1] - C1)) +
                            gC[2] * (Tn * c[2] - (Cf[2] - C2)) - gT * Tf + gD * (Tn * z - (Df - D));
            float qsig = 0.f, qdel = 0.f;
            if (QUANT && gQ != 0.f) {
                float dP_ds = 0.f, dP_dd = 0.f, dQ_ds = 0.f, dQ_dd = 0.f;
                if (g.delta > 0.f) {
                    const QuantSeg q = quant_seg(g.sigma, g.delta, g.e);
                    qZ1 -= T * ((1.f - 2.f * T) * q.A + 2.f * T * q.C);  // now the suffix over later segments
                    qZ2 -= T * q.A;
                    dP_ds = T * (qWn * q.dA_ds + T * q.dC_ds);
                    dP_dd = T * g.e * (qWn + T * q.alpha);
                    dQ_ds = -T * q.dA_ds;
                    dQ_dd = qWn + T * q.alpha;
                    qWn += T * q.alpha;
                }
                const float later = qk2 * (qZ1 + Tf * qZ2) + qdTf * Tf;
                qsig = gQ * (qk2 * (dP_ds - Tf * dQ_ds) - g.delta * later);
                qdel = gQ * (qk2 * (dP_dd - Tf * dQ_dd) - g.sigma * later);
            }
            sig_bar = io.g_density ? g.delta * B + qsig : 0.f;
            if (io.g_sh) {
                cb[0] = g.pre[0] > 0.f ? gC[0] * w : 0.f;
                cb[1] = g.pre[1] > 0.f ? gC[1] * w : 0.f;
                cb[2] = g.pre[2] > 0.f ? gC[2] * w : 0.f;
            }
            // segment bounds: delta = max(b - a, 0), z = (a + b)/2,
            // a = max(t0, t_min), b = min(t1, t_max)
            const float dbar = g.sigma * B + qdel;
            float abar = 0.5f * gD * w, bbar = abar;
            if (g.b > g.a) {
                bbar += dbar;
                abar -= dbar;
            }
            const float t1bar = g.t1 < tmax ? bbar : 0.f;
            const float t0bar = t0 > tmin ? abar : 0.f;
            if (pend) {
                if (pend_defines) {
                    padj += t0bar;
                } else if (da >= 0 && t0bar != 0.f && io.g_pos) {
                    // t0 was set by an earlier crossing (floating-point tie)
                    const CellHdr ca = load_cell(p.s, da), cbh = load_cell(p.s, db);
                    const float nx = cbh.x - ca.x, ny = cbh.y - ca.y, nz = cbh.z - ca.z;
                    const float s_ = t0bar / (nx * d.x + ny * d.y + nz * d.z);
                    const float qx = (o.x - ca.x) + dt * d.x, qy = (o.y - ca.y) + dt * d.y,
                                qz = (o.z - ca.z) + dt * d.z;
                    atomicAdd(io.g_pos + 3 * (int64_t)da + 0, s_ * qx);
                    atomicAdd(io.g_pos + 3 * (int64_t)da + 1, s_ * qy);
                    atomicAdd(io.g_pos + 3 * (int64_t)da + 2, s_ * qz);
                    atomicAdd(io.g_pos + 3 * (int64_t)db + 0, s_ * (nx - qx));
                    atomicAdd(io.g_pos + 3 * (int64_t)db + 1, s_ * (ny - qy));
                    atomicAdd(io.g_pos + 3 * (int64_t)db + 2, s_ * (nz - qz));
                }
                // crossing (pa -> i) at pt: dt/dp_i = (p_i - x)/den, dt/dp_a = (x - p_a)/den,
                // x = o + pt d, den = (p_i - p_a).d
                if (padj != 0.f && io.g_pos) {
                    const float nx = cell.x - pxa.x, ny = cell.y - pxa.y, nz = cell.z - pxa.z;
                    const float s_ = padj / (nx * d.x + ny * d.y + nz * d.z);
                    const float qx = poca.x + pt * d.x, qy = poca.y + pt * d.y, qz = poca.z + pt * d.z;
                    gpos_a[0] = s_ * qx;
                    gpos_a[1] = s_ * qy;
                    gpos_a[2] = s_ * qz;
                    gpos_i[0] = s_ * (nx - qx);
                    gpos_i[1] = s_ * (ny - qy);
                    gpos_i[2] = s_ * (nz - qz);
                }
                key_prev = pa;
            }
            // this step's exit becomes the pending crossing; a segment that
            // ends on the (fixed) sphere has none, and the next leg's t0 = 0
            // is set by no crossing
            pend = g.next >= 0 && !(FX && g.hit);
            if (FX && g.hit) da = -1;
            pa = i;
            pxa = make_float3(cell.x, cell.y, cell.z);
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
        }

        // ---- warp-wide scatter of this iteration's contributions ----
        // The crossing that entered the cell also moves the previous cell's
        // site: each lane adds those three terms itself.
        if constexpr (!SHARED) {
            if (live && key_prev >= 0 && (gpos_a[0] != 0.f || gpos_a[1] != 0.f || gpos_a[2] != 0.f))
                atomicAdd(io.g_acc + key_prev, make_float4(gpos_a[0], gpos_a[1], gpos_a[2], 0.f));
        }
        // The rest goes to the current cell.  Lanes in the same cell are
        // summed over 16-byte columns of their staged rows, two cells per
        // pass; the rows of lanes alone in their cell (or of every lane, when
        // the warp is spread over more than kMaxGroups shared cells) are
        // spread over the whole warp, one (row, column) item per lane.
        const unsigned peers = __match_any_sync(full, live ? (unsigned)i : 0xffffffffu);
        if constexpr (SHARED) {
            // the previous cells' crossing terms, summed per cell when the
            // warp's lanes share few cells, else added lane by lane
            __shared__ float4 cross_all[kBlock / 32][32];
            const int ncell = __popc(__ballot_sync(full, live && lane == __ffs(peers) - 1));
            const bool has_a = live && key_prev >= 0 && (gpos_a[0] != 0.f || gpos_a[1] != 0.f || gpos_a[2] != 0.f);
            if (ncell > kSharedCells) {
                if (has_a) atomicAdd(io.g_acc + key_prev, make_float4(gpos_a[0], gpos_a[1], gpos_a[2], 0.f));
            } else {
                float4 *cross = cross_all[threadIdx.x >> 5];
                const unsigned am = __match_any_sync(full, has_a ? (unsigned)key_prev : 0xffffffffu);
                if (has_a) cross[lane] = make_float4(gpos_a[0], gpos_a[1], gpos_a[2], 0.f);
                __syncwarp();
                if (has_a && lane == __ffs(am) - 1) {
                    float4 sm = cross[lane];
                    for (unsigned mm = am & (am - 1); mm; mm &= mm - 1) {
                        const float4 v = cross[__ffs(mm) - 1];
                        sm.x += v.x;
                        sm.y += v.y;
                        sm.z += v.z;
                    }
                    atomicAdd(io.g_acc + key_prev, sm);
                }
            }
        }
        const bool in_group = live && __popc(peers) > 1;
        unsigned leaders = __ballot_sync(full, in_group && lane == __ffs(peers) - 1);
        if (__popc(leaders) > kMaxGroups) leaders = 0u;
        const bool alone = live && !(in_group && leaders != 0u);
        const unsigned lone = __ballot_sync(full, alone);
        if (leaders | lone) {
            if (live) {
                // this lane's row: SH gradient (zero padded), {position of the cell, density}
                float4 *row = reinterpret_cast<float4 *>(stage + lane * SP);
#pragma unroll
                for (int q4 = 0; q4 < VP / 4; ++q4) {
                    float v[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int c = 4 * q4 + e;
                        v[e] = c < NV ? cb[c % 3] * Y[c / 3]
                             : c < NVP ? 0.f
                             : c < NVP + 3 ? gpos_i[c - NVP] : sig_bar;
                    }
                    row[q4] = make_float4(v[0], v[1], v[2], v[3]);
                }
            }
            if (alone) {
                const int rank = __popc(lone & ((1u << lane) - 1u));
                alone_lane[rank] = lane;
                alone_cell[rank] = i;
            }
            __syncwarp();
            constexpr int NQ = VP / 4;
            constexpr int SQ = SP / 4;
            const float4 *stage4 = reinterpret_cast<const float4 *>(stage);
            // column c (floats 4c .. 4c+3) of a row of `cell` into the
            // gradients that were asked for (a zero column is added too:
            // testing for it costs more than the rare empty atomic)
            auto add_column = [&](int cell, int col, const float4 &v) {
                const int c = 4 * col;
                if (c >= NVP) {
                    if (io.g_acc) atomicAdd(io.g_acc + cell, v);   // {position, density} of the cell
                } else if (!io.g_sh) {
                    // no SH gradient wanted
                } else if (NV % 4 == 0 && io.sh_vec) {
                    atomicAdd(reinterpret_cast<float4 *>(io.g_sh + (size_t)cell * NV + c), v);
                } else {
                    const float v4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (c + j < NV && v4[j] != 0.f) atomicAdd(io.g_sh + (size_t)cell * NV + c + j, v4[j]);
                }
            };
            // (a) cells shared by several lanes: lanes 0..15 sum the first
            // cell of a pass, lanes 16..31 the second, four values per lane
            const int hl = lane & 15;
            while (leaders) {
                const int L0 = __ffs(leaders) - 1;
                leaders &= leaders - 1;
                const bool two = leaders != 0;
                const int L1 = two ? __ffs(leaders) - 1 : L0;
                if (two) leaders &= leaders - 1;
                const int L = lane >= 16 ? L1 : L0;
                const unsigned m = __shfl_sync(full, peers, L);
                const int cell_i = __shfl_sync(full, i, L);
                if ((lane < 16 || two) && hl < NQ) {
                    // three members per trip with independent loads; an absent
                    // member (-1) loads nothing
                    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    float4 sm = z4;
                    for (unsigned mm = m; mm;) {
                        const int k0 = __ffs(mm) - 1;
                        mm &= mm - 1;
                        const int k1 = __ffs(mm) - 1;
                        mm &= mm - 1;
                        const int k2 = __ffs(mm) - 1;
                        mm &= mm - 1;
                        const float4 a0 = stage4[k0 * SQ + hl];
                        float4 a1, a2;
                        if constexpr (FX) {
                            a1 = stage4[(k1 >= 0 ? k1 : 32) * SQ + hl];
                            a2 = stage4[(k2 >= 0 ? k2 : 32) * SQ + hl];
                        } else {
                            a1 = k1 >= 0 ? stage4[k1 * SQ + hl] : z4;
                            a2 = k2 >= 0 ? stage4[k2 * SQ + hl] : z4;
                        }
                        sm.x += (a0.x + a1.x) + a2.x;
                        sm.y += (a0.y + a1.y) + a2.y;
                        sm.z += (a0.z + a1.z) + a2.z;
                        sm.w += (a0.w + a1.w) + a2.w;
                    }
                    add_column(cell_i, hl, sm);
                }
            }
            // (b) rows alone: item t = (row rank t / NQ, column t % NQ)
            const int items = __popc(lone) * NQ;
            for (int t = lane; t < items; t += 32) {
                const int r = t / NQ, col = t - r * NQ;
                add_column(alone_cell[r], col, stage4[alone_lane[r] * SQ + col]);
            }
            __syncwarp();
        }

        if (live) {
            if (FX && g.hit) {
                if (fx_bounce(p.fx, p.s, f, o, d, tmin, tmax)) {
                    sh_basis<DEG>(d, Y);
                    t0 = 0.f;  // the new leg starts in the same cell
                } else {
                    live = false;
                }
            } else if (g.next < 0 || !(g.t1 < tmax)) {
                live = false;  // nothing pending: the exit lies at or beyond t_max
            } else {
                t0 = g.t1 > t0 ? g.t1 : t0;
                i = g.next;
            }
        }
    }
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

// Launch the forward (mode kPlain / kTrace / kQuant) or the backward over
// `tiles` blocks for the scene's attribute type and SH degree.
template <bool FX>
void launch_fwd_any(int dtype, int deg, int mode, int64_t tiles, const RenderParams &p, const FwdOut &o,
                    cudaStream_t st) {
    dispatch(dtype, deg, [&]<typename AT, int DEG>() {
        if (mode == kTrace) fwd_kernel<AT, DEG, kTrace, FX><<<(unsigned)tiles, kBlock, 0, st>>>(p, o);
        else if (mode == kQuant) fwd_kernel<AT, DEG, kQuant, FX><<<(unsigned)tiles, kBlock, 0, st>>>(p, o);
        else fwd_kernel<AT, DEG, kPlain, FX><<<(unsigned)tiles, kBlock, 0, st>>>(p, o);
    });
}

template <bool FX, bool SHARED>
void launch_bwd_any(int dtype, int deg, bool quant, int64_t tiles, const RenderParams &p, const BwdIO &io,
                    cudaStream_t st) {
    dispatch(dtype, deg, [&]<typename AT, int DEG>() {
        if (quant) bwd_kernel<AT, DEG, true, FX, SHARED><<<(unsigned)tiles, kBlock, 0, st>>>(p, io);
        else bwd_kernel<AT, DEG, false, FX, SHARED><<<(unsigned)tiles, kBlock, 0, st>>>(p, io);
    });
}

extern template void launch_fwd_any<false>(int, int, int, int64_t, const RenderParams &, const FwdOut &,
                                           cudaStream_t);
extern template void launch_fwd_any<true>(int, int, int, int64_t, const RenderParams &, const FwdOut &,
                                          cudaStream_t);
extern template void launch_bwd_any<false, false>(int, int, bool, int64_t, const RenderParams &, const BwdIO &,
                                                  cudaStream_t);
extern template void launch_bwd_any<true, false>(int, int, bool, int64_t, const RenderParams &, const BwdIO &,
                                                 cudaStream_t);
extern template void launch_bwd_any<false, true>(int, int, bool, int64_t, const RenderParams &, const BwdIO &,
                                                 cudaStream_t);
extern template void launch_bwd_any<true, true>(int, int, bool, int64_t, const RenderParams &, const BwdIO &,
                                                cudaStream_t);

}  // namespace rf
