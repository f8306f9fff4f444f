/*
 * adjacency.c -- plain FP64 CPU oracle for the Voronoi adjacency that the
 * walk of Alg. 1 needs: N(i), the sites whose Voronoi cells share a face of
 * positive area with the cell of site i (the Delaunay neighbours, Sec. 3.2 and
 * the Voronoi optimisation paragraph of Sec. 4).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite and the benchmark's CPU-baseline
 * leg load this file.  The CUDA adjacency builder shares no code with it.
 *
 * Definition, computed literally: the face between sites i and j is the part
 * of their bisector plane {x : |x - p_i| = |x - p_j|} that lies in the domain
 * box and is no farther from p_i than from any other site k, i.e. inside every
 * half-space (p_k - p_i) . x <= (|p_k|^2 - |p_i|^2) / 2.  It is built as a
 * polygon: a square of the bisector plane that covers the domain, cut by the
 * six box planes and by the half-space of every candidate k (Sutherland-Hodgman
 * clipping of a convex polygon by a line).  i and j are adjacent iff the
 * polygon keeps a positive area.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FACE_MAXV 160

typedef struct {
    double p[FACE_MAXV][3];
    int n;
} poly_t;

/* Keep the part of the polygon with a . x <= c. */
static void clip_poly(poly_t *P, const double *a, double c, poly_t *tmp)
{
    tmp->n = 0;
    for (int k = 0; k < P->n; ++k) {
        const double *u = P->p[k];
        const double *v = P->p[(k + 1) % P->n];
        const double su = a[0] * u[0] + a[1] * u[1] + a[2] * u[2] - c;
        const double sv = a[0] * v[0] + a[1] * v[1] + a[2] * v[2] - c;
        if (su <= 0.0 && tmp->n < FACE_MAXV) memcpy(tmp->p[tmp->n++], u, sizeof(double) * 3);
        if ((su < 0.0 && sv > 0.0) || (su > 0.0 && sv < 0.0)) {
            const double t = su / (su - sv);
            if (tmp->n < FACE_MAXV) {
                for (int a3 = 0; a3 < 3; ++a3) tmp->p[tmp->n][a3] = u[a3] + t * (v[a3] - u[a3]);
                ++tmp->n;
            }
        }
    }
    memcpy(P->p, tmp->p, sizeof(double) * 3 * (size_t)tmp->n);
    P->n = tmp->n;
}

static double poly_area(const poly_t *P)
{
    if (P->n < 3) return 0.0;
    double s[3] = {0.0, 0.0, 0.0};
    for (int k = 1; k + 1 < P->n; ++k) {
        double e1[3], e2[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = P->p[k][a] - P->p[0][a];
            e2[a] = P->p[k + 1][a] - P->p[0][a];
        }
        s[0] += e1[1] * e2[2] - e1[2] * e2[1];
        s[1] += e1[2] * e2[0] - e1[0] * e2[2];
        s[2] += e1[0] * e2[1] - e1[1] * e2[0];
    }
    return 0.5 * sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
}

/*
 * Face between sites i and j, cut by the candidates cand[0..n_cand) (i and j
 * themselves are skipped) and the domain box (min xyz, max xyz).  Returns its
 * area; *rmax receives the largest distance from p_i to a polygon vertex (0
 * for an empty face).
 */
static double face_area(const double *pos, int64_t i, int64_t j, const int64_t *cand,
                        int64_t n_cand, const double *dom, double *rmax, poly_t *P, poly_t *tmp)
{
    const double *pi = pos + 3 * i, *pj = pos + 3 * j;
    double n[3], m[3], nn = 0.0;
    for (int a = 0; a < 3; ++a) {
        n[a] = pj[a] - pi[a];
        m[a] = 0.5 * (pi[a] + pj[a]);
        nn += n[a] * n[a];
    }
    *rmax = 0.0;
    if (!(nn > 0.0)) return 0.0;
    /* orthonormal basis (u, w) of the bisector plane */
    const double ln = sqrt(nn);
    const double e[3] = {n[0] / ln, n[1] / ln, n[2] / ln};
    double u[3];
    if (fabs(e[0]) < 0.6) { u[0] = 0.0; u[1] = e[2]; u[2] = -e[1]; }
    else { u[0] = -e[2]; u[1] = 0.0; u[2] = e[0]; }
    const double lu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int a = 0; a < 3; ++a) u[a] /= lu;
    const double w[3] = {e[1] * u[2] - e[2] * u[1], e[2] * u[0] - e[0] * u[2], e[0] * u[1] - e[1] * u[0]};
    /* a square of the plane, centred at the projection of the box centre,
     * larger than the box's diagonal */
    double half = 0.0, cen[3];
    for (int a = 0; a < 3; ++a) {
        half += (dom[3 + a] - dom[a]) * (dom[3 + a] - dom[a]);
        cen[a] = 0.5 * (dom[a] + dom[3 + a]);
    }
    half = 2.0 * sqrt(half) + 1.0;
    double off = 0.0;
    for (int a = 0; a < 3; ++a) off += e[a] * (cen[a] - m[a]);
    for (int a = 0; a < 3; ++a) cen[a] -= off * e[a];
    static const double sq[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
    P->n = 4;
    for (int k = 0; k < 4; ++k)
        for (int a = 0; a < 3; ++a) P->p[k][a] = cen[a] + half * (sq[k][0] * u[a] + sq[k][1] * w[a]);
    /* the domain box */
    for (int a = 0; a < 3; ++a) {
        double ax[3] = {0.0, 0.0, 0.0};
        ax[a] = 1.0;
        clip_poly(P, ax, dom[3 + a], tmp);
        ax[a] = -1.0;
        clip_poly(P, ax, -dom[a], tmp);
        if (P->n == 0) return 0.0;
    }
    /* no farther from p_i than from any candidate k */
    const double ii = pi[0] * pi[0] + pi[1] * pi[1] + pi[2] * pi[2];
    for (int64_t c = 0; c < n_cand && P->n > 0; ++c) {
        const int64_t k = cand[c];
        if (k == i || k == j) continue;
        const double *pk = pos + 3 * k;
        const double a3[3] = {pk[0] - pi[0], pk[1] - pi[1], pk[2] - pi[2]};
        if (a3[0] == 0.0 && a3[1] == 0.0 && a3[2] == 0.0) continue;
        const double kk = pk[0] * pk[0] + pk[1] * pk[1] + pk[2] * pk[2];
        clip_poly(P, a3, 0.5 * (kk - ii), tmp);
    }
    const double area = poly_area(P);
    if (area > 0.0) {
        for (int k = 0; k < P->n; ++k) {
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) d2 += (P->p[k][a] - pi[a]) * (P->p[k][a] - pi[a]);
            if (d2 > *rmax * *rmax) *rmax = sqrt(d2);
        }
    }
    return area;
}

/* Largest distance from p_i to a vertex of the cell's face on box side b
 * (0..5: +x, -x, +y, -y, +z, -z), cut by the candidates; 0 if empty. */
static double box_face_rmax(const double *pos, int64_t i, int b, const int64_t *cand, int64_t n_cand,
                            const double *dom, poly_t *P, poly_t *tmp)
{
    const int ax = b >> 1, a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
    const double v = (b & 1) ? dom[ax] : dom[3 + ax];
    static const int sq[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
    P->n = 4;
    for (int k = 0; k < 4; ++k) {
        P->p[k][ax] = v;
        P->p[k][a1] = sq[k][0] ? dom[3 + a1] : dom[a1];
        P->p[k][a2] = sq[k][1] ? dom[3 + a2] : dom[a2];
    }
    const double *pi = pos + 3 * i;
    const double ii = pi[0] * pi[0] + pi[1] * pi[1] + pi[2] * pi[2];
    for (int64_t c = 0; c < n_cand && P->n > 0; ++c) {
        const int64_t k = cand[c];
        if (k == i) continue;
        const double *pk = pos + 3 * k;
        const double a3[3] = {pk[0] - pi[0], pk[1] - pi[1], pk[2] - pi[2]};
        if (a3[0] == 0.0 && a3[1] == 0.0 && a3[2] == 0.0) continue;
        const double kk = pk[0] * pk[0] + pk[1] * pk[1] + pk[2] * pk[2];
        clip_poly(P, a3, 0.5 * (kk - ii), tmp);
    }
    double r = 0.0;
    if (poly_area(P) > 0.0)
        for (int k = 0; k < P->n; ++k) {
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) d2 += (P->p[k][a] - pi[a]) * (P->p[k][a] - pi[a]);
            if (d2 > r * r) r = sqrt(d2);
        }
    return r;
}

/*
 * For each query q: site qi[q] and its candidate list cand[off[q] .. off[q+1]).
 * area[c] = area of the face between qi[q] and cand[c], cut by all the other
 * candidates of q and the domain box; rmax[q] = the largest distance from the
 * site to a vertex of the cell (its faces with the candidates and with the
 * domain box): the radius about p_i of the cell cut by the candidates, which
 * contains the true cell.  Returns 0.
 */
int orc_voronoi_faces(int64_t n_sites, const double *pos, int64_t n_query, const int64_t *qi,
                      const int64_t *off, const int64_t *cand, const double *domain, double *area,
                      double *rmax, int n_threads)
{
    (void)n_sites;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
        poly_t *P = (poly_t *)malloc(sizeof(poly_t)), *tmp = (poly_t *)malloc(sizeof(poly_t));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t q = 0; q < n_query; ++q) {
            const int64_t i = qi[q];
            double rq = 0.0;
            for (int64_t c = off[q]; c < off[q + 1]; ++c) {
                double r;
                area[c] = face_area(pos, i, cand[c], cand + off[q], off[q + 1] - off[q], domain, &r, P, tmp);
                if (r > rq) rq = r;
            }
            /* the cell's faces on the domain box also hold vertices */
            for (int b = 0; b < 6; ++b) {
                const double r = box_face_rmax(pos, i, b, cand + off[q], off[q + 1] - off[q], domain, P, tmp);
                if (r > rq) rq = r;
            }
            rmax[q] = rq;
        }
        free(P);
        free(tmp);
    }
    return 0;
}
