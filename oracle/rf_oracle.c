/*
 * rf_oracle.c -- plain, slow FP64 CPU oracle for Radiant Foam ray tracing
 * (Govindarajan et al., "Radiant Foam: Real-Time Differentiable Ray Tracing",
 * arXiv 2502.01157).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline / reference leg load this file.  The CUDA renderer
 * never calls it and shares no code with it.
 *
 * What it computes (all in FP64, one ray at a time, in the paper's order):
 *
 *   - Ray generation for a pinhole or equidistant-fisheye camera (pixel
 *     centres, OpenCV frame), optionally with a rolling shutter that moves
 *     each row's origin (the ray-based effects figure, Fig. 2).
 *   - The initial cell nn(o): the site nearest to the ray origin (Alg. 1),
 *     per row for a rolling shutter.
 *   - The walk of Alg. 1 (Sec. 3.2): in cell i, over every neighbour j in
 *     N(i), intersect the ray with the bisector plane of x_i and x_j; a plane
 *     whose normal x_j - x_i makes an angle below 90 deg with d is an exit
 *     (Fig. 3); the nearest exit (strict <, first in adjacency order on ties)
 *     gives t_1 and the next cell.
 *   - Piecewise-constant compositing, Eq. (3)-(4): alpha = 1 - exp(-sigma
 *     delta), C += T alpha c, T *= (1 - alpha), while T > eps.
 *   - Optionally one analytic sphere met in the same walk (Fig. 2): a
 *     mirror, or clear glass with Snell refraction and total internal
 *     reflection; the ray bends at the hit point and the walk carries on in
 *     the same cell along the new direction.
 *   - Colour from real spherical harmonics of degree <= 3 in the ray
 *     direction, plus 0.5, clamped at 0 (Sec. 3.4 "Training").
 *   - The quantile loss of Eq. (6): the expected distance between two
 *     quantiles of the ray's weight distribution, E|W^-1(u1) - W^-1(u2)| with
 *     u1, u2 ~ U[0,1], which equals 2 * integral F(t)(1 - F(t)) dt for the
 *     normalised weight CDF F = (1 - T(t)) / (1 - T_final); per segment the
 *     integral has a closed form (exponential transmittance).
 *   - The gradient of (rgb, transmittance, depth, quantile loss) with respect to density,
 *     SH coefficients and site positions, by plain reverse-mode
 *     differentiation of the stored segment list; positions receive gradient
 *     only through the segment widths (Sec. 3.1).
 *
 * Readings where the paper is silent (shared with the CUDA path only as a
 * specification, not as code):
 *   - every ray is clipped to [t_min, t_max] = [max(t_near, box entry),
 *     min(t_far, box exit)] of the scene box; a ray that misses the box returns
 *     rgb 0, T 1, depth 0;
 *   - the walk starts at t_0 = 0 in nn(o); segments are composited over their
 *     part inside [t_min, t_max]; it stops when T <= eps (checked before each
 *     step), when the exit lies at or beyond t_max, or when the cell has no
 *     exit (an unbounded hull cell);
 *   - t_0 <- max(t_0, t_1) (equal to t_0 <- t_1 in exact arithmetic);
 *   - depth = sum_n T_n alpha_n (a_n + b_n) / 2, the weighted midpoint of the
 *     composited part [a_n, b_n] of each segment.
 *
 * Near-degenerate rays.  The per-ray flags say why a correct FP32 renderer
 * may differ from this FP64 walk on a ray (tau = the degeneracy distance):
 *   ORC_FLAG_EDGE    the ray passes within tau of a Voronoi edge or vertex
 *                    of a cell it walks: the distance from the ray to the
 *                    line where the exit plane meets another face plane of
 *                    the cell (or the scene box), or from a step's end point
 *                    to another face plane, is below tau (on a leg after a
 *                    sphere bounce, tau plus the FP32 error bound of the bent
 *                    ray).  Which cell comes next is then a tie at FP32.
 *   ORC_FLAG_CAMERA  the start point lies within tau of the bisector of its
 *                    two nearest sites (nn(o) is a tie).
 *   ORC_FLAG_STOP    the transmittance is within a relative 1e-3 of eps at a
 *                    stop test (the walk may end one step earlier or later).
 *   ORC_FLAG_GRAZE   a face is crossed at grazing incidence: the cells are
 *                    not in doubt, but the crossing's position gradient
 *                    (1 / cos) is ill-conditioned at FP32.
 *   ORC_FLAG_BEND    a sphere hit near tangency or a refraction near the
 *                    critical angle: the bent direction is ill-conditioned.
 * EDGE and CAMERA rays may visit other cells; STOP rays may stop one step
 * apart; GRAZE and BEND rays visit the same cells but their gradients carry
 * the conditioning error.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_RAY_OK 0
#define ORC_RAY_MAX_STEPS 1

#define ORC_FLAG_EDGE 1
#define ORC_FLAG_CAMERA 2
#define ORC_FLAG_STOP 4
#define ORC_FLAG_GRAZE 8
#define ORC_FLAG_BEND 16

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics (orthonormal on the unit sphere, no Condon-      */
/* Shortley phase), index l*l + l + m, written out in Cartesian form from    */
/* Y_l^m = sqrt(2) N_l^|m| P_l^|m|(cos th) {cos(m phi), sin(|m| phi)}.        */
/* ------------------------------------------------------------------------ */
int orc_sh_basis(int degree, const double *d, double *Y)
{
    const double pi = 3.14159265358979323846;
    const double x = d[0], y = d[1], z = d[2];
    if (degree < 0 || degree > 3) return -1;
    Y[0] = 0.5 * sqrt(1.0 / pi);
    if (degree >= 1) {
        const double c1 = sqrt(3.0 / (4.0 * pi));
        Y[1] = c1 * y;
        Y[2] = c1 * z;
        Y[3] = c1 * x;
    }
    if (degree >= 2) {
        const double a = 0.5 * sqrt(15.0 / pi);
        Y[4] = a * x * y;
        Y[5] = a * y * z;
        Y[6] = 0.25 * sqrt(5.0 / pi) * (3.0 * z * z - 1.0);
        Y[7] = a * x * z;
        Y[8] = 0.25 * sqrt(15.0 / pi) * (x * x - y * y);
    }
    if (degree >= 3) {
        const double b = 0.25 * sqrt(35.0 / (2.0 * pi));
        const double c = 0.25 * sqrt(21.0 / (2.0 * pi));
        Y[9] = b * y * (3.0 * x * x - y * y);
        Y[10] = 0.5 * sqrt(105.0 / pi) * x * y * z;
        Y[11] = c * y * (5.0 * z * z - 1.0);
        Y[12] = 0.25 * sqrt(7.0 / pi) * (5.0 * z * z * z - 3.0 * z);
        Y[13] = c * x * (5.0 * z * z - 1.0);
        Y[14] = 0.25 * sqrt(105.0 / pi) * z * (x * x - y * y);
        Y[15] = b * x * (x * x - 3.0 * y * y);
    }
    return 0;
}

int orc_sh_basis_batch(int degree, int64_t n, const double *dirs, double *Y)
{
    const int K = (degree + 1) * (degree + 1);
    for (int64_t r = 0; r < n; ++r)
        if (orc_sh_basis(degree, dirs + 3 * r, Y + K * r)) return -1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Camera: cam[0..11] = c2w (3x4 row-major [R|t]), cam[12..15] = fx fy cx cy, */
/* cam[16..17] = width height, cam[18..19] = t_near t_far, cam[20] = model    */
/* (0 pinhole, 1 equidistant fisheye), cam[21..23] = rolling-shutter          */
/* velocity (the centre moves by it from the first row to the last).          */
/* Pixel p = v * width + u; its ray passes through the pixel centre.          */
/* ------------------------------------------------------------------------ */
void orc_camera_ray(const double *cam, int64_t pixel, double *o, double *d)
{
    const int64_t W = (int64_t)cam[16];
    const int64_t H = (int64_t)cam[17];
    const int64_t u = pixel % W, v = pixel / W;
    const double x = ((double)u + 0.5 - cam[14]) / cam[12];
    const double y = ((double)v + 0.5 - cam[15]) / cam[13];
    double xc = x, yc = y, zc = 1.0;
    if ((int)cam[20] == 1) {
        /* equidistant fisheye: the angle from the optical axis equals the
         * radius in normalised image coordinates */
        const double th = sqrt(x * x + y * y);
        const double sc = th > 0.0 ? sin(th) / th : 1.0;
        xc = x * sc;
        yc = y * sc;
        zc = cos(th);
    }
    const double row = ((double)v + 0.5) / (double)H - 0.5;
    double w[3];
    for (int r = 0; r < 3; ++r) {
        w[r] = cam[4 * r + 0] * xc + cam[4 * r + 1] * yc + cam[4 * r + 2] * zc;
        o[r] = cam[4 * r + 3] + row * cam[21 + r];
    }
    const double len = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    for (int r = 0; r < 3; ++r) d[r] = w[r] / len;
}

static int has_shutter(const double *cam) { return cam[21] != 0.0 || cam[22] != 0.0 || cam[23] != 0.0; }

/* Nearest site (lowest index on exact ties); *gap receives the distance from
 * q to the bisector plane of its two nearest sites (HUGE_VAL if N < 2). */
int64_t orc_nearest_site(int64_t n, const double *pos, const double *q, double *gap)
{
    int64_t b0 = -1, b1 = -1;
    double d0 = HUGE_VAL, d1 = HUGE_VAL;
    for (int64_t i = 0; i < n; ++i) {
        const double dx = pos[3 * i] - q[0], dy = pos[3 * i + 1] - q[1], dz = pos[3 * i + 2] - q[2];
        const double dd = dx * dx + dy * dy + dz * dz;
        if (dd < d0) { d1 = d0; b1 = b0; d0 = dd; b0 = i; }
        else if (dd < d1) { d1 = dd; b1 = i; }
    }
    if (gap) {
        if (b1 < 0) *gap = HUGE_VAL;
        else {
            double s = 0.0;
            for (int a = 0; a < 3; ++a) {
                const double t = pos[3 * b1 + a] - pos[3 * b0 + a];
                s += t * t;
            }
            *gap = (d1 - d0) / (2.0 * sqrt(s));
        }
    }
    return b0;
}

/* Ray / scene-box slab test intersected with [t_near, t_far]. */
static int ray_interval(const double *o, const double *d, const double *box,
                        double t_near, double t_far, double *tmin, double *tmax)
{
    double lo = t_near > 0.0 ? t_near : 0.0;
    double hi = t_far > 0.0 ? t_far : HUGE_VAL;
    for (int a = 0; a < 3; ++a) {
        if (d[a] != 0.0) {
            double t1 = (box[a] - o[a]) / d[a];
            double t2 = (box[3 + a] - o[a]) / d[a];
            if (t1 > t2) { double s = t1; t1 = t2; t2 = s; }
            if (t1 > lo) lo = t1;
            if (t2 < hi) hi = t2;
        } else if (o[a] < box[a] || o[a] > box[3 + a]) {
            return 0;
        }
    }
    *tmin = lo;
    *tmax = hi;
    return lo < hi;
}

/* ------------------------------------------------------------------------ */
/* Scene                                                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    const double *pos;     /* [n,3] */
    const int64_t *off;    /* [n+1] */
    const int32_t *adj;    /* [E] */
    const double *sigma;   /* [n] */
    const double *sh;      /* [n,K,3] */
    int deg, K;
    const double *box;     /* min xyz, max xyz */
} scene_t;

typedef struct {
    int64_t cell, next;   /* next = -1: no exit */
    double t0, t1;        /* raw entry / exit parameters (t1: the sphere hit if bounce) */
    double a, b;          /* composited part [a,b] (a >= b: nothing) */
    double delta, sigma, e, T;   /* T: transmittance before the segment */
    double pre[3], c[3];  /* colour before / after the clamp at 0 */
    double o[3], d[3];    /* the ray this segment lies on */
    double tmin, tmax;    /* that ray's compositing interval */
    double soff;          /* path length before that ray's origin (bounces) */
    int bounce;           /* the segment ends on the sphere, not on a face */
} seg_t;

/* Optional analytic sphere the rays bounce off (mirror) or through (clear
 * glass, Snell's law with total internal reflection): fx = {max_bounces,
 * cx, cy, cz, radius, ior}, ior = 0 for a mirror. */
typedef struct {
    int max_bounces;
    double c[3], r, ior;
} effects_t;

static int effects_of(const double *fx, effects_t *E)
{
    if (!fx || !(fx[4] > 0.0) || fx[0] < 1.0) return 0;
    E->max_bounces = (int)fx[0];
    for (int a = 0; a < 3; ++a) E->c[a] = fx[1 + a];
    E->r = fx[4];
    E->ior = fx[5];
    return 1;
}

/* Parameter of the next sphere crossing of the ray: the entry (near root)
 * from outside, the exit (far root) from inside; HUGE_VAL if none ahead.
 * *disc_out returns the discriminant relative to r^2 (tangency test). */
static double sphere_hit(const effects_t *E, const double *o, const double *d, int inside,
                         double *disc_out)
{
    double oc[3], b = 0.0, cc = 0.0;
    for (int a = 0; a < 3; ++a) {
        oc[a] = o[a] - E->c[a];
        b += d[a] * oc[a];
        cc += oc[a] * oc[a];
    }
    cc -= E->r * E->r;
    const double disc = b * b - cc;
    *disc_out = disc / (E->r * E->r);
    if (disc < 0.0) return HUGE_VAL;
    const double t = inside ? -b + sqrt(disc) : -b - sqrt(disc);
    return t > 0.0 ? t : HUGE_VAL;
}

/* New direction at the hit point p: mirror reflection, or refraction with
 * relative index n1/n2 (total internal reflection when impossible).
 * Returns 1 if the ray crossed into the other side. *kout: Snell's k. */
static int sphere_bounce(const effects_t *E, const double *p, double *d, int inside, double *kout)
{
    double n[3], dn = 0.0;
    for (int a = 0; a < 3; ++a) {
        n[a] = (p[a] - E->c[a]) / E->r;
        dn += d[a] * n[a];
    }
    *kout = 1.0;
    int crossed = 0;
    if (E->ior > 0.0) {
        const double sgn = inside ? -1.0 : 1.0;  /* normal on the incoming side */
        const double eta = inside ? E->ior : 1.0 / E->ior;
        const double cosi = -dn * sgn;
        const double k = 1.0 - eta * eta * (1.0 - cosi * cosi);
        *kout = k;
        if (k >= 0.0) {
            const double f = eta * cosi - sqrt(k);
            for (int a = 0; a < 3; ++a) d[a] = eta * d[a] + f * sgn * n[a];
            crossed = 1;
        }
    }
    if (!crossed)
        for (int a = 0; a < 3; ++a) d[a] -= 2.0 * dn * n[a];
    const double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int a = 0; a < 3; ++a) d[a] /= len;
    return crossed;
}

typedef struct {
    seg_t *s;
    int64_t n, cap;
} seglist_t;

static void seg_push(seglist_t *L, const seg_t *s)
{
    if (!L) return;
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 256;
        L->s = (seg_t *)realloc(L->s, (size_t)L->cap * sizeof(seg_t));
    }
    L->s[L->n++] = *s;
}

/* Colour of cell i for the basis values Y (Sec. 3.4: SH of degree <= 3). */
static void cell_colour(const scene_t *S, int64_t i, const double *Y, double *pre, double *c)
{
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int k = 0; k < S->K; ++k) acc += S->sh[(i * S->K + k) * 3 + ch] * Y[k];
        pre[ch] = acc + 0.5;
        c[ch] = pre[ch] > 0.0 ? pre[ch] : 0.0;
    }
}

/* Unit normal n and offset h of the bisector plane of sites i and k
 * ({x : n.x = h}, n pointing from x_i to x_k); returns |x_k - x_i|. */
static double bisector_plane(const scene_t *S, int64_t i, int64_t k, double *n, double *h)
{
    double len2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        n[a] = S->pos[3 * k + a] - S->pos[3 * i + a];
        len2 += n[a] * n[a];
    }
    const double len = sqrt(len2);
    *h = 0.0;
    for (int a = 0; a < 3; ++a) {
        n[a] /= len;
        *h += n[a] * 0.5 * (S->pos[3 * k + a] + S->pos[3 * i + a]);
    }
    return len;
}

/* Distance from p to the bisector plane of sites i and k. */
static double plane_dist(const scene_t *S, int64_t i, int64_t k, const double *p)
{
    double n[3], h;
    bisector_plane(S, i, k, n, &h);
    return fabs(n[0] * p[0] + n[1] * p[1] + n[2] * p[2] - h);
}

/* Distance between the ray's line x(t) = o + t d and the line where two
 * planes it crosses meet (unit normals na, nb; ca = na.d and cb = nb.d its
 * cosines to them, both > 0; it crosses them at ta and tb).  The signed
 * distances to the planes are s_a = ca (t - ta) and s_b = cb (t - tb), a
 * point's squared distance to the line is (s_a^2 + s_b^2 - 2 g s_a s_b) /
 * (1 - g^2) with g = na.nb, and its minimum over t is
 * (tb - ta)^2 ca^2 cb^2 / |cb na - ca nb|^2. */
static double ray_line_dist(const double *na, double ca, double ta, const double *nb, double cb,
                            double tb)
{
    double w2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double w = cb * na[k] - ca * nb[k];
        w2 += w * w;
    }
    if (!(w2 > 0.0)) return HUGE_VAL;  /* the same plane */
    return fabs(tb - ta) * ca * cb / sqrt(w2);
}

/* Is the ray within tol of the Voronoi edge where the plane it leaves the
 * cell by ({ne.x = he}, crossed at te: the exit face `skip` or a face of the
 * scene box) meets the plane of another exit candidate (a front-facing face
 * of cell i)?  Those two are the candidates whose order at FP32 decides the
 * next cell; a grazing candidate keeps the ray near the edge although the
 * crossing points lie apart. */
static int near_edge(const scene_t *S, int64_t i, int64_t skip, const double *ne, double te,
                     const double *o, const double *d, double tol)
{
    const double ce = ne[0] * d[0] + ne[1] * d[1] + ne[2] * d[2];
    if (!(ce > 0.0)) return 0;
    for (int64_t f = S->off[i]; f < S->off[i + 1]; ++f) {
        const int64_t k = S->adj[f];
        if (k == skip) continue;
        double nk[3], hk;
        bisector_plane(S, i, k, nk, &hk);
        const double ck = nk[0] * d[0] + nk[1] * d[1] + nk[2] * d[2];
        if (!(ck > 0.0)) continue;
        const double tk = (hk - (nk[0] * o[0] + nk[1] * o[1] + nk[2] * o[2])) / ck;
        if (ray_line_dist(ne, ce, te, nk, ck, tk) < tol) return 1;
    }
    return 0;
}

typedef struct {
    double rgb[3], T, depth;
    int32_t steps;
    uint8_t status, flags;
} ray_out_t;

/* FP32 error bound of the current leg's ray: its origin is off by up to e_pos
 * and its direction by up to e_dir (relative), so a point at parameter t is
 * off by e_pos + e_dir t.  Both are 0 for the camera's own ray, whose FP32
 * rounding the degeneracy distance tau already covers. */
typedef struct {
    double e_pos, e_dir;
} leg_err_t;

/*
 * Alg. 1 for one ray.  Segments are appended to L (if non-NULL); the visited
 * cells and raw exit parameters to trace_cells / trace_t (up to max_trace).
 */
static void render_ray(const scene_t *S, int64_t start, const double *o_in, const double *d_in,
                       double tmin, double tmax, double eps, int max_steps, double tau,
                       double *Y, ray_out_t *R, seglist_t *L,
                       int max_trace, int32_t *trace_cells, double *trace_t, const effects_t *E)
{
    double T = 1.0, C[3] = {0.0, 0.0, 0.0}, D = 0.0, t0 = 0.0, s_off = 0.0;
    double o[3] = {o_in[0], o_in[1], o_in[2]}, d[3] = {d_in[0], d_in[1], d_in[2]};
    int64_t i = start;
    int steps = 0, bounces = 0, inside = 0;
    leg_err_t err = {0.0, 0.0};
    if (E) {
        double r2 = 0.0;
        for (int a = 0; a < 3; ++a) r2 += (o[a] - E->c[a]) * (o[a] - E->c[a]);
        inside = r2 < E->r * E->r;
    }
    R->status = ORC_RAY_OK;
    while (T > eps) {
        if (fabs(T - eps) <= 1e-3 * eps) R->flags |= ORC_FLAG_STOP;
        if (steps >= max_steps) { R->status = ORC_RAY_MAX_STEPS; break; }
        const double *x = S->pos + 3 * i;
        /* nearest front-facing bisector plane (Fig. 3) */
        double t1 = HUGE_VAL, cos_exit = 1.0, len_exit = HUGE_VAL, len_min = 1.0;
        int64_t nxt = -1;
        for (int64_t f = S->off[i]; f < S->off[i + 1]; ++f) {
            const int64_t j = S->adj[f];
            const double *xp = S->pos + 3 * j;
            double den = 0.0, num = 0.0, nn = 0.0;
            for (int a = 0; a < 3; ++a) {
                const double n = xp[a] - x[a];
                const double m = 0.5 * (xp[a] + x[a]);
                den += n * d[a];
                num += n * (m - o[a]);
                nn += n * n;
            }
            if (f == S->off[i] || sqrt(nn) < len_min) len_min = sqrt(nn);
            if (den > 0.0) {
                const double t = num / den;
                if (t < t1) { t1 = t; nxt = j; cos_exit = den / sqrt(nn); len_exit = sqrt(nn); }
            }
        }
        if (nxt < 0) len_exit = len_min;  /* a cell-sized length for the tests below */
        /* degeneracy distance on this leg at the far end of this step */
        const double tol_at = tau > 0.0 ? tau + err.e_pos + err.e_dir * (fabs(t1 < tmax ? t1 : tmax) + len_exit)
                                        : -1.0;
        /* does the ray meet the sphere inside this cell? */
        int hit = 0;
        double ts = HUGE_VAL, disc_hit = 1.0;
        if (E && bounces < E->max_bounces) {
            double disc;
            ts = sphere_hit(E, o, d, inside, &disc);
            disc_hit = disc;
            /* near-grazing: the hit point's error grows as 1/sqrt(disc), so the
             * bent direction (and all that follows) is ill-conditioned */
            if (fabs(disc) < 1e-2) R->flags |= ORC_FLAG_BEND;
            hit = ts >= t0 && ts < t1 && ts < tmax;
            if (isfinite(ts) && nxt >= 0 && tau > 0.0) {
                /* a hit next to the exit face: which cell it falls in is a tie
                 * (the FP32 hit parameter is off by ~1e-7 (|ts| + r / sqrt(disc))) */
                double ps[3];
                for (int a = 0; a < 3; ++a) ps[a] = o[a] + ts * d[a];
                const double e_ts = 1e-7 * (fabs(ts) + E->r / sqrt(fabs(disc) > 1e-12 ? fabs(disc) : 1e-12));
                if (plane_dist(S, i, nxt, ps) < tol_at + cos_exit * e_ts) R->flags |= ORC_FLAG_EDGE;
            }
        }
        const double tend = hit ? ts : t1;
        /* a crossing at grazing incidence: a rounding of the direction
         * (~1e-7 relative) or of the coordinates (~tau / 10) moves its point
         * along the face by (1e-7 |t| + tau / 10) / cos; flagged when that
         * exceeds 1e-3 of the distance between the two sites, where the
         * crossing's position gradient is ill-conditioned at FP32 */
        if (!hit && nxt >= 0 && t1 < tmax && tau > 0.0 &&
            (1e-7 * fabs(t1) + 0.1 * tau) > 1e-3 * cos_exit * len_exit)
            R->flags |= ORC_FLAG_GRAZE;
        if (tau > 0.0) {
            /* near a Voronoi edge or vertex: the step's end point within tol
             * of another face plane of the cell ... */
            const double te = (hit || (nxt >= 0 && t1 < tmax)) ? tend : tmax;
            double p[3];
            for (int a = 0; a < 3; ++a) p[a] = o[a] + te * d[a];
            for (int64_t f = S->off[i]; f < S->off[i + 1]; ++f) {
                const int64_t k = S->adj[f];
                if (!hit && k == nxt && te == t1) continue;
                if (plane_dist(S, i, k, p) < tol_at) { R->flags |= ORC_FLAG_EDGE; break; }
            }
            /* ... or the ray within tol of the edge between the plane it
             * leaves by and another exit candidate */
            if (!hit && !(R->flags & ORC_FLAG_EDGE)) {
                double ne[3], he;
                int64_t skip = -1;
                int have = 0;
                if (nxt >= 0 && t1 < tmax) {
                    bisector_plane(S, i, nxt, ne, &he);
                    skip = nxt;
                    have = 1;
                } else {
                    /* the step ends on the scene box: the face whose slab gives tmax */
                    for (int a = 0; a < 3 && !have; ++a) {
                        if (d[a] == 0.0) continue;
                        const double bnd = d[a] > 0.0 ? S->box[3 + a] : S->box[a];
                        if (fabs((bnd - o[a]) / d[a] - tmax) <= 1e-12 * (1.0 + fabs(tmax))) {
                            ne[0] = ne[1] = ne[2] = 0.0;
                            ne[a] = d[a] > 0.0 ? 1.0 : -1.0;
                            have = 1;
                        }
                    }
                }
                if (have && near_edge(S, i, skip, ne, te, o, d, tol_at)) R->flags |= ORC_FLAG_EDGE;
            }
        }
        seg_t s;
        s.cell = i;
        s.next = hit ? i : nxt;
        s.bounce = hit;
        s.t0 = t0;
        s.t1 = tend;
        s.a = t0 > tmin ? t0 : tmin;
        s.b = tend < tmax ? tend : tmax;
        s.delta = s.b > s.a ? s.b - s.a : 0.0;
        s.sigma = S->sigma[i];
        s.e = exp(-s.sigma * s.delta);
        s.T = T;
        s.tmin = tmin;
        s.tmax = tmax;
        s.soff = s_off;
        for (int a = 0; a < 3; ++a) { s.o[a] = o[a]; s.d[a] = d[a]; }
        cell_colour(S, i, Y, s.pre, s.c);
        const double alpha = 1.0 - s.e;
        for (int ch = 0; ch < 3; ++ch) C[ch] += T * alpha * s.c[ch];
        D += T * alpha * (s_off + 0.5 * (s.a + s.b));
        T *= s.e;
        seg_push(L, &s);
        if (steps < max_trace) {
            trace_cells[steps] = (int32_t)i;
            trace_t[steps] = tend;
        }
        ++steps;
        if (hit) {
            /* bounce: the new ray starts at the hit point, in the same cell */
            double p[3], k;
            for (int a = 0; a < 3; ++a) p[a] = o[a] + ts * d[a];
            const double eta = E->ior > 0.0 ? (inside ? E->ior : 1.0 / E->ior) : 0.0;
            const int crossed = sphere_bounce(E, p, d, inside, &k);
            if (crossed) inside = !inside;
            if (E->ior > 0.0 && fabs(k) < 1e-2) R->flags |= ORC_FLAG_BEND;  /* near the critical angle */
            /* error bound of the new leg: the FP32 hit point (its parameter
             * carries ~1e-7 r / sqrt(disc)) and the normal through it; a
             * reflection keeps the direction's error and adds up to 4 times the
             * normal's, a refraction scales both by up to eta + eta^2 / sqrt(k)
             * (taken twice for safety) */
            {
                double oc2 = 0.0;
                for (int a = 0; a < 3; ++a) oc2 += (s.o[a] - E->c[a]) * (s.o[a] - E->c[a]);
                const double dh = fabs(disc_hit) > 1e-12 ? fabs(disc_hit) : 1e-12;
                const double e_p = err.e_pos + err.e_dir * ts + 1e-7 * (ts + sqrt(oc2) + E->r / sqrt(dh));
                const double e_n = e_p / E->r;
                if (crossed) {
                    const double rk = 1.0 / sqrt(fabs(k) > 1e-12 ? fabs(k) : 1e-12);
                    err.e_dir = 2.0 * (eta + eta * eta * rk) * (err.e_dir + e_n) + 1e-7 * (1.0 + rk);
                } else {
                    err.e_dir = err.e_dir + 4.0 * e_n + 1e-7;
                }
                err.e_pos = e_p;
            }
            for (int a = 0; a < 3; ++a) o[a] = p[a];
            s_off += ts;
            t0 = 0.0;
            ++bounces;
            orc_sh_basis(S->deg, d, Y);
            if (!ray_interval(o, d, S->box, 0.0, 0.0, &tmin, &tmax)) break;
            continue;
        }
        if (nxt < 0 || t1 >= tmax) break;
        if (t1 > t0) t0 = t1;
        i = nxt;
    }
    if (T <= eps && fabs(T - eps) <= 1e-3 * eps) R->flags |= ORC_FLAG_STOP;
    for (int ch = 0; ch < 3; ++ch) R->rgb[ch] = C[ch];
    R->T = T;
    R->depth = D;
    R->steps = steps;
}

/* a = (1 - e^{-s d}) / s and b = (1 - e^{-2 s d}) / (2 s): the integrals of
 * T(t)/T_n and (T(t)/T_n)^2 over a segment of width d and density s, with
 * their partial derivatives in s and d. */
static void seg_integrals(double s, double d, double *a, double *b, double *da_ds, double *da_dd,
                          double *db_ds, double *db_dd)
{
    const double x = s * d;
    const double e = exp(-x);
    if (x < 1e-4) {
        /* series in x (exact to O(x^4)) */
        *a = d * (1.0 - x / 2.0 + x * x / 6.0 - x * x * x / 24.0);
        *b = d * (1.0 - x + 2.0 * x * x / 3.0 - x * x * x / 3.0);
        *da_ds = -d * d * (0.5 - x / 3.0 + x * x / 8.0 - x * x * x / 30.0);
        *db_ds = d * d * (-1.0 + 4.0 * x / 3.0 - x * x + 8.0 * x * x * x / 15.0);
    } else {
        *a = -expm1(-x) / s;
        *b = -expm1(-2.0 * x) / (2.0 * s);
        *da_ds = (x * e + expm1(-x)) / (s * s);
        *db_ds = (2.0 * x * e * e + expm1(-2.0 * x)) / (2.0 * s * s);
    }
    *da_dd = e;
    *db_dd = e * e;
}

/* Quantile loss of Eq. (6) for one ray: with F = (1 - T)/(1 - T_f),
 * 2 * int F (1 - F) dt = 2/(1 - T_f)^2 * sum_n int_seg (1 - T)(T - T_f) dt and
 * int_seg (1 - T)(T - T_f) = (1 + T_f) T_n a_n - T_n^2 b_n - T_f delta_n. */
static double quantile_loss(const seglist_t *L, double Tf)
{
    const double W = 1.0 - Tf;
    if (!(W > 0.0)) return 0.0;
    double S = 0.0;
    for (int64_t k = 0; k < L->n; ++k) {
        const seg_t *g = &L->s[k];
        if (!(g->delta > 0.0)) continue;
        double a, b, t1, t2, t3, t4;
        seg_integrals(g->sigma, g->delta, &a, &b, &t1, &t2, &t3, &t4);
        S += (1.0 + Tf) * g->T * a - g->T * g->T * b - Tf * g->delta;
    }
    return 2.0 * S / (W * W);
}

/* Adjoints of the quantile loss (scaled by gq) with respect to each
 * segment's density and width, by reverse-mode differentiation of
 * quantile_loss through T_n = prod_{k<n} e_k and T_f = prod_k e_k. */
static void quantile_adjoints(const seglist_t *L, double Tf, double gq, double *qsig, double *qdel)
{
    const double W = 1.0 - Tf;
    for (int64_t k = 0; k < L->n; ++k) qsig[k] = qdel[k] = 0.0;
    if (!(W > 0.0) || gq == 0.0) return;
    double S = 0.0, dS_dTf = 0.0;
    for (int64_t k = 0; k < L->n; ++k) {
        const seg_t *g = &L->s[k];
        if (!(g->delta > 0.0)) continue;
        double a, b, t1, t2, t3, t4;
        seg_integrals(g->sigma, g->delta, &a, &b, &t1, &t2, &t3, &t4);
        S += (1.0 + Tf) * g->T * a - g->T * g->T * b - Tf * g->delta;
        dS_dTf += g->T * a - g->delta;
    }
    const double c = 2.0 / (W * W);
    const double Sbar = gq * c;
    /* L = c(T_f) S(T_f, ...): dc/dT_f = 4 / W^3 */
    double Tbar = gq * S * 4.0 / (W * W * W) + Sbar * dS_dTf;  /* adjoint of T after the last segment */
    for (int64_t k = L->n - 1; k >= 0; --k) {
        const seg_t *g = &L->s[k];
        double a = g->delta, b = g->delta, da_ds = 0, da_dd = 1, db_ds = 0, db_dd = 1;
        if (g->delta > 0.0) seg_integrals(g->sigma, g->delta, &a, &b, &da_ds, &da_dd, &db_ds, &db_dd);
        else a = b = 0.0;
        const double ebar = Tbar * g->T;   /* T_{k+1} = T_k e_k */
        const double dI_dT = g->delta > 0.0 ? (1.0 + Tf) * a - 2.0 * g->T * b : 0.0;
        if (g->delta > 0.0) {
            qsig[k] = Sbar * ((1.0 + Tf) * g->T * da_ds - g->T * g->T * db_ds);
            qdel[k] = Sbar * ((1.0 + Tf) * g->T * da_dd - g->T * g->T * db_dd - Tf);
        }
        /* e_k = exp(-sigma_k delta_k) */
        qsig[k] += ebar * (-g->delta * g->e);
        qdel[k] += ebar * (-g->sigma * g->e);
        Tbar = Tbar * g->e + Sbar * dI_dT;
    }
}

static int setup_scene(scene_t *S, int64_t n, const double *pos, const int64_t *off,
                       const int32_t *adj, const double *sigma, const double *sh, int deg,
                       const double *box)
{
    if (deg < 0 || deg > 3 || n < 1) return -1;
    S->n = n; S->pos = pos; S->off = off; S->adj = adj; S->sigma = sigma; S->sh = sh;
    S->deg = deg; S->K = (deg + 1) * (deg + 1); S->box = box;
    return 0;
}

/* Start cell of Alg. 1: nn(o).  All rays of a global-shutter camera share
 * one origin; a rolling shutter gives every row its own. */
typedef struct {
    int64_t start;
    int degen;
} cam_start_t;

/* start_info, if given, holds {nn(centre), its gap} found by an earlier
 * call of orc_camera_start for the same scene and camera. */
static cam_start_t camera_start(const scene_t *S, const double *cam, double tau, const double *start_info)
{
    const double o[3] = {cam[3], cam[7], cam[11]};  /* the centre (mid-frame for a rolling shutter) */
    double gap;
    cam_start_t c;
    if (start_info) {
        c.start = (int64_t)start_info[0];
        gap = start_info[1];
    } else {
        c.start = orc_nearest_site(S->n, S->pos, o, &gap);
    }
    c.degen = gap < tau;
    return c;
}

/* nn of the camera centre and its gap (out2 = {site, gap}), for reuse by
 * later calls on the same scene and camera. */
void orc_camera_start(int64_t n_sites, const double *pos, const double *cam, double *out2)
{
    const double o[3] = {cam[3], cam[7], cam[11]};
    double gap;
    out2[0] = (double)orc_nearest_site(n_sites, pos, o, &gap);
    out2[1] = gap;
}

static int64_t ray_start(const scene_t *S, const double *cam, const cam_start_t *c,
                         const double *ro, double tau, int *degen)
{
    if (!has_shutter(cam)) {
        if (c->degen) *degen = 1;
        return c->start;
    }
    double gap;
    const int64_t s = orc_nearest_site(S->n, S->pos, ro, &gap);
    if (gap < tau) *degen = 1;
    return s;
}

/*
 * Forward render of n_rays pixels of one camera (pixels == NULL: all pixels
 * in order).  Outputs per ray: rgb[3], trans, depth, steps, status, flags
 * (ORC_FLAG_*).
 * Optional trace (max_trace > 0): cells visited and raw exit parameters,
 * row-major [n_rays, max_trace].  Returns 0, or -1 on bad arguments.
 */
int orc_render(int64_t n_sites, const double *pos, const int64_t *off, const int32_t *adj,
               const double *sigma, const double *sh, int sh_degree, const double *box,
               const double *cam, int64_t n_rays, const int64_t *pixels,
               double eps, int max_steps, double tau,
               double *rgb, double *trans, double *depth, int32_t *steps, uint8_t *status,
               uint8_t *flags, int max_trace, int32_t *trace_cells, double *trace_t,
               const double *effects, const double *start_info, int n_threads)
{
    scene_t S;
    if (setup_scene(&S, n_sites, pos, off, adj, sigma, sh, sh_degree, box)) return -1;
    effects_t E;
    const effects_t *EP = effects_of(effects, &E) ? &E : NULL;
    const cam_start_t cs = camera_start(&S, cam, tau, start_info);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t r = 0; r < n_rays; ++r) {
        const int64_t px = pixels ? pixels[r] : r;
        double ro[3], rd[3], Y[16], tmin, tmax;
        orc_camera_ray(cam, px, ro, rd);
        orc_sh_basis(S.deg, rd, Y);
        ray_out_t R;
        memset(&R, 0, sizeof R);
        R.T = 1.0;
        int32_t *tc = max_trace > 0 ? trace_cells + r * (int64_t)max_trace : NULL;
        double *tt = max_trace > 0 ? trace_t + r * (int64_t)max_trace : NULL;
        int sdeg = 0;
        const int64_t start = ray_start(&S, cam, &cs, ro, tau, &sdeg);
        if (ray_interval(ro, rd, box, cam[18], cam[19], &tmin, &tmax)) {
            render_ray(&S, start, ro, rd, tmin, tmax, eps, max_steps, tau, Y, &R, NULL,
                       max_trace, tc, tt, EP);
        }
        if (sdeg) R.flags |= ORC_FLAG_CAMERA;
        for (int ch = 0; ch < 3; ++ch) rgb[3 * r + ch] = R.rgb[ch];
        trans[r] = R.T;
        depth[r] = R.depth;
        if (steps) steps[r] = R.steps;
        if (status) status[r] = R.status;
        if (flags) flags[r] = R.flags;
    }
    return 0;
}

/* Quantile loss of Eq. (6) per ray (0 for a ray with no weight). */
int orc_render_quantile(int64_t n_sites, const double *pos, const int64_t *off, const int32_t *adj,
                        const double *sigma, const double *sh, int sh_degree, const double *box,
                        const double *cam, int64_t n_rays, const int64_t *pixels, double eps,
                        int max_steps, double *quantile, const double *effects,
                        const double *start_info, int n_threads)
{
    scene_t S;
    if (setup_scene(&S, n_sites, pos, off, adj, sigma, sh, sh_degree, box)) return -1;
    effects_t E;
    const effects_t *EP = effects_of(effects, &E) ? &E : NULL;
    const cam_start_t cs = camera_start(&S, cam, -1.0, start_info);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t r = 0; r < n_rays; ++r) {
        const int64_t px = pixels ? pixels[r] : r;
        double ro[3], rd[3], Y[16], tmin, tmax;
        orc_camera_ray(cam, px, ro, rd);
        orc_sh_basis(S.deg, rd, Y);
        quantile[r] = 0.0;
        if (!ray_interval(ro, rd, box, cam[18], cam[19], &tmin, &tmax)) continue;
        int sdeg = 0;
        const int64_t start = ray_start(&S, cam, &cs, ro, -1.0, &sdeg);
        ray_out_t R;
        memset(&R, 0, sizeof R);
        seglist_t L = {NULL, 0, 0};
        render_ray(&S, start, ro, rd, tmin, tmax, eps, max_steps, -1.0, Y, &R, &L, 0, NULL, NULL,
                   EP);
        quantile[r] = quantile_loss(&L, R.T);
        free(L.s);
    }
    return 0;
}

#ifdef _OPENMP
#define ORC_ATOMIC _Pragma("omp atomic")
#else
#define ORC_ATOMIC
#endif

/*
 * Gradient of L = g_rgb . rgb + g_trans * T + g_depth * depth + g_quantile *
 * quantile for n_rays pixels of one camera, accumulated (+=) into g_sigma
 * [N], g_sh [N,K,3] and g_pos [N,3].  g_trans / g_depth / g_quantile may be
 * NULL (zero).  The forward walk is
 * repeated with its segments stored, then differentiated in reverse order.
 */
int orc_render_bwd(int64_t n_sites, const double *pos, const int64_t *off, const int32_t *adj,
                   const double *sigma, const double *sh, int sh_degree, const double *box,
                   const double *cam, int64_t n_rays, const int64_t *pixels,
                   double eps, int max_steps,
                   const double *g_rgb, const double *g_trans, const double *g_depth,
                   const double *g_quantile, double *g_sigma, double *g_sh, double *g_pos,
                   const double *effects, const double *start_info, int n_threads)
{
    scene_t S;
    if (setup_scene(&S, n_sites, pos, off, adj, sigma, sh, sh_degree, box)) return -1;
    effects_t E;
    const effects_t *EP = effects_of(effects, &E) ? &E : NULL;
    const cam_start_t cs = camera_start(&S, cam, -1.0, start_info);
    const int K = S.K;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t r = 0; r < n_rays; ++r) {
        const int64_t px = pixels ? pixels[r] : r;
        double ro[3], rd[3], Y[16], tmin, tmax;
        orc_camera_ray(cam, px, ro, rd);
        orc_sh_basis(S.deg, rd, Y);
        if (!ray_interval(ro, rd, box, cam[18], cam[19], &tmin, &tmax)) continue;
        int sdeg = 0;
        const int64_t start = ray_start(&S, cam, &cs, ro, -1.0, &sdeg);
        ray_out_t R;
        memset(&R, 0, sizeof R);
        seglist_t L = {NULL, 0, 0};
        render_ray(&S, start, ro, rd, tmin, tmax, eps, max_steps, -1.0, Y, &R,
                   &L, 0, NULL, NULL, EP);
        const double gC[3] = {g_rgb[3 * r], g_rgb[3 * r + 1], g_rgb[3 * r + 2]};
        const double gT = g_trans ? g_trans[r] : 0.0;
        const double gD = g_depth ? g_depth[r] : 0.0;
        const double gQ = g_quantile ? g_quantile[r] : 0.0;
        double *qsig = (double *)calloc((size_t)(L.n > 0 ? 2 * L.n : 2), sizeof(double));
        double *qdel = qsig + (L.n > 0 ? L.n : 1);
        quantile_adjoints(&L, R.T, gQ, qsig, qdel);
        double Tbar = gT;       /* adjoint of the transmittance after segment k */
        double t0bar_next = 0.0;  /* adjoint of t0 of segment k+1 */
        for (int64_t k = L.n - 1; k >= 0; --k) {
            const seg_t *s = &L.s[k];
            const double w = s->T * (1.0 - s->e);
            const double z = s->soff + 0.5 * (s->a + s->b);
            double wbar = gD * z;
            for (int ch = 0; ch < 3; ++ch) wbar += gC[ch] * s->c[ch];
            /* T_{k+1} = T_k e_k;  C += T_k (1 - e_k) c_k;  D += T_k (1 - e_k) z_k */
            const double ebar = Tbar * s->T - wbar * s->T;
            Tbar = Tbar * s->e + wbar * (1.0 - s->e);
            const double sigbar = ebar * (-s->delta * s->e) + qsig[k];
            const double dbar = ebar * (-s->sigma * s->e) + qdel[k];
            const double zbar = gD * w;
            double abar = 0.5 * zbar, bbar = 0.5 * zbar;
            if (s->b > s->a) { bbar += dbar; abar -= dbar; }
            double t1bar = (s->t1 < s->tmax) ? bbar : 0.0;
            double t0bar = (s->t0 > s->tmin) ? abar : 0.0;
            /* t0 of segment k+1 = max(t0_k, t1_k); a bounce restarts at t0 = 0
             * on a new ray, and the sphere hit itself does not move with the
             * sites */
            if (s->bounce) t1bar = 0.0;
            else if (k + 1 < L.n) {
                if (s->t1 >= s->t0) t1bar += t0bar_next;
                else t0bar += t0bar_next;
            }
            t0bar_next = t0bar;
            const int64_t i = s->cell;
            orc_sh_basis(S.deg, s->d, Y);
            ORC_ATOMIC
            g_sigma[i] += sigbar;
            for (int ch = 0; ch < 3; ++ch) {
                if (!(s->pre[ch] > 0.0)) continue;
                const double cbar = gC[ch] * w;
                for (int kk = 0; kk < K; ++kk) {
                    ORC_ATOMIC
                    g_sh[(i * K + kk) * 3 + ch] += cbar * Y[kk];
                }
            }
            /* exit parameter t1 of the bisector plane (i, j): dt/dx_j = (x_j - p)/den,
             * dt/dx_i = (p - x_i)/den with p = o + t1 d, den = (x_j - x_i).d */
            if (s->next >= 0 && t1bar != 0.0 && isfinite(s->t1)) {
                const int64_t j = s->next;
                double den = 0.0, p[3];
                for (int a = 0; a < 3; ++a) {
                    den += (pos[3 * j + a] - pos[3 * i + a]) * s->d[a];
                    p[a] = s->o[a] + s->t1 * s->d[a];
                }
                for (int a = 0; a < 3; ++a) {
                    const double gj = t1bar * (pos[3 * j + a] - p[a]) / den;
                    const double gi = t1bar * (p[a] - pos[3 * i + a]) / den;
                    ORC_ATOMIC
                    g_pos[3 * j + a] += gj;
                    ORC_ATOMIC
                    g_pos[3 * i + a] += gi;
                }
            }
        }
        free(qsig);
        free(L.s);
    }
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
