"""Seeded synthetic inputs: Voronoi sites, their Delaunay adjacency, per-cell
attributes and pinhole cameras.

This module only *draws* inputs.  It holds none of the rendering arithmetic
(no ray generation, no plane tests, no spherical-harmonic evaluation, no
compositing), so both the CUDA path and the FP64 oracle can consume what it
produces without sharing any of the method.

Workloads (the paper's datasets are not available; these stand in for them):

* ``c1`` -- 4,096 sites uniform in [-1,1]^3; density LogNormal(0,1); SH degree 0
  with base colours uniform in [0,1]; one 64x64 camera at the origin, 60 deg FOV.
* ``c2`` -- 1,000,000 sites: 90% from 64 anisotropic Gaussians (centres uniform
  in [-8,8]^3, per-axis std uniform in [0.1,1], random rotation), 10% uniform in
  [-10,10]^3; density LogNormal(0,1); SH degree 3 with 48 coefficients ~ N(0,0.3);
  one 1280x720 camera at the origin looking along +z.
* ``c3`` -- the c1 recipe with 3,000,000 sites and SH degree 3 (DC from colours
  uniform in [0,1], higher orders ~ N(0,0.3)); one 1920x1080 camera at the origin.
* ``c4``/``c5`` -- the c2 recipe scaled to 3,000,000 sites; cameras on a sphere
  of radius 12 looking at the origin.

The Delaunay adjacency (the neighbour lists N(i) of the ray-tracing algorithm,
Sec. 3.2) is an *input* of the renderer.  It is built with Qhull through
scipy.  Large point sets are triangulated in parallel, block by block, and every
block result is validated with the empty-circumsphere criterion against all
sites before it is accepted (see :func:`delaunay_csr`).
"""
from __future__ import annotations

import dataclasses
import hashlib
import math
import os
import time
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Scenes with at most this many sites are triangulated in one Qhull call.
_GLOBAL_DELAUNAY_MAX = 250_000


# ----------------------------------------------------------------------------
# Cameras
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Camera:
    """Pinhole or equidistant-fisheye camera, global or rolling shutter.

    ``c2w`` is a 3x4 row-major matrix [R | t]: a point ``x_c`` in the camera
    frame (OpenCV: +x right, +y down, +z forward) maps to ``R @ x_c + t`` in the
    world; ``t`` is the camera centre.  Intrinsics are in pixels.  ``t_near`` and
    ``t_far`` bound the rendered depth along each unit ray (``t_far <= 0``: no
    bound beyond the scene box).  ``model``: ``PINHOLE`` or ``FISHEYE``
    (equidistant: the angle to the optical axis equals the normalised image
    radius).  ``shutter``: world-space displacement of the centre from the first
    image row to the last (rolling shutter); row ``v`` is exposed from
    ``t + ((v + 1/2)/height - 1/2) * shutter``.
    """

    c2w: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    t_near: float = 0.0
    t_far: float = 0.0
    model: int = 0
    shutter: Tuple[float, float, float] = (0.0, 0.0, 0.0)

    PINHOLE = 0
    FISHEYE = 1

    def __post_init__(self):
        self.c2w = np.asarray(self.c2w, dtype=np.float32).reshape(3, 4)
        # Every real number the renderer sees is an FP32 value.
        for f in ("fx", "fy", "cx", "cy", "t_near", "t_far"):
            setattr(self, f, float(np.float32(getattr(self, f))))
        self.width = int(self.width)
        self.height = int(self.height)
        self.model = int(self.model)
        self.shutter = tuple(float(v) for v in np.asarray(self.shutter, np.float32).reshape(3))

    @property
    def n_rays(self) -> int:
        return self.width * self.height

    def as_f64(self) -> np.ndarray:
        """24 doubles: c2w(12), fx, fy, cx, cy, width, height, t_near, t_far,
        model, shutter(3)."""
        return np.array(list(self.c2w.reshape(-1).astype(np.float64)) +
                        [self.fx, self.fy, self.cx, self.cy, self.width,
                         self.height, self.t_near, self.t_far, self.model] +
                        list(self.shutter), dtype=np.float64)


def fisheye(width: int, height: int, fov_deg: float, c2w=None) -> Camera:
    """Equidistant fisheye whose image circle of diameter ``min(width,
    height)`` spans ``fov_deg`` (up to 360)."""
    f = (min(width, height) / 2.0) / math.radians(fov_deg / 2.0)
    if c2w is None:
        c2w = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    return Camera(c2w, f, f, width / 2.0, height / 2.0, width, height, model=Camera.FISHEYE)


@dataclasses.dataclass
class Sphere:
    """Analytic sphere in the foam: a perfect mirror (``ior == 0``) or clear
    glass of refractive index ``ior`` (Snell refraction, total internal
    reflection).  A ray interacts with it at most ``max_bounces`` times and
    then passes through it."""

    centre: Tuple[float, float, float]
    radius: float
    ior: float = 0.0
    max_bounces: int = 8

    def __post_init__(self):
        self.centre = tuple(float(v) for v in np.asarray(self.centre, np.float32).reshape(3))
        self.radius = float(np.float32(self.radius))
        self.ior = float(np.float32(self.ior))
        self.max_bounces = int(self.max_bounces)

    def as_f64(self) -> np.ndarray:
        """6 doubles: max_bounces, centre(3), radius, ior."""
        return np.array([self.max_bounces, *self.centre, self.radius, self.ior], np.float64)


def pinhole(width: int, height: int, fov_y_deg: float, c2w=None,
            t_near: float = 0.0, t_far: float = 0.0) -> Camera:
    """Camera with square pixels and a vertical field of view ``fov_y_deg``;
    the principal point is the image centre."""
    f = (height / 2.0) / math.tan(math.radians(fov_y_deg) / 2.0)
    if c2w is None:
        c2w = np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1)
    return Camera(c2w, f, f, width / 2.0, height / 2.0, width, height,
                  t_near, t_far)


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """3x4 camera-to-world matrix for an OpenCV camera at ``eye`` looking at
    ``target``; ``up`` is re-drawn if it is within 1 deg of the view axis."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    up = np.asarray(up, np.float64)
    if abs(np.dot(fwd, up / np.linalg.norm(up))) > math.cos(math.radians(1.0)):
        up = np.array([1.0, 0.0, 0.0]) if abs(fwd[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], axis=1)
    return np.concatenate([R, eye[:, None]], axis=1)


def sphere_poses(n: int, radius: float, seed: int) -> List[np.ndarray]:
    """``n`` camera poses uniform on a sphere, each looking at the origin."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return [look_at(radius * v[k]) for k in range(n)]


# ----------------------------------------------------------------------------
# Sites and attributes
# ----------------------------------------------------------------------------
def uniform_sites(n: int, lo: float, hi: float, rng) -> np.ndarray:
    return rng.uniform(lo, hi, size=(n, 3)).astype(np.float32)


def mixture_sites(n: int, rng, n_gauss: int = 64, frac_gauss: float = 0.9,
                  centre_box: float = 8.0, bg_box: float = 10.0) -> np.ndarray:
    """Anisotropic Gaussian mixture plus a uniform background."""
    n_g = int(round(n * frac_gauss))
    n_u = n - n_g
    centres = rng.uniform(-centre_box, centre_box, size=(n_gauss, 3))
    stds = rng.uniform(0.1, 1.0, size=(n_gauss, 3))
    rots = []
    for _ in range(n_gauss):
        q, r = np.linalg.qr(rng.normal(size=(3, 3)))
        rots.append(q * np.sign(np.diag(r)))
    comp = rng.integers(0, n_gauss, size=n_g)
    z = rng.normal(size=(n_g, 3)) * stds[comp]
    pts_g = np.einsum("nij,nj->ni", np.stack(rots)[comp], z) + centres[comp]
    pts_u = rng.uniform(-bg_box, bg_box, size=(n_u, 3))
    pts = np.concatenate([pts_g, pts_u], axis=0)
    return pts[rng.permutation(n)].astype(np.float32)


def dedupe_sites(pts: np.ndarray, rng) -> np.ndarray:
    """Re-draw exact duplicates (possible after FP32 rounding) by a tiny jitter."""
    for _ in range(8):
        order = np.lexsort((pts[:, 2], pts[:, 1], pts[:, 0]))
        q = pts[order]
        dup = np.zeros(len(pts), bool)
        dup[order[1:]] = np.all(q[1:] == q[:-1], axis=1)
        if not dup.any():
            return pts
        pts[dup] += rng.normal(scale=1e-4, size=(int(dup.sum()), 3)).astype(np.float32)
    return pts


def lognormal_density(n: int, rng) -> np.ndarray:
    return rng.lognormal(0.0, 1.0, size=n).astype(np.float32)


def sh_coeffs(n: int, degree: int, rng, dc: str = "normal",
              std: float = 0.3) -> np.ndarray:
    """[n, (degree+1)^2, 3] coefficients.

    ``dc='normal'``: every coefficient ~ N(0, std).  ``dc='uniform_colour'``:
    the DC coefficient is uniform on [-sqrt(pi), sqrt(pi)] (base colours uniform
    in [0,1] after the +0.5 offset) and the rest ~ N(0, std).
    """
    k = (degree + 1) ** 2
    out = rng.normal(0.0, std, size=(n, k, 3))
    if dc == "uniform_colour":
        a = math.sqrt(math.pi)
        out[:, 0, :] = rng.uniform(-a, a, size=(n, 3))
    return out.astype(np.float32)


# ----------------------------------------------------------------------------
# Delaunay adjacency (CSR)
# ----------------------------------------------------------------------------
def _ghost_shell(centre: np.ndarray, radius: float, n: int = 512) -> np.ndarray:
    """Far points on a Fibonacci sphere.  They bound every Voronoi cell of the
    real sites so each site's star is closed; their own cells only claim space
    more than ``radius/2`` from the centre and they are dropped from the CSR."""
    k = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * k / n)
    th = math.pi * (1 + 5 ** 0.5) * k
    v = np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)
    return centre[None, :] + radius * v


def _sorted_unique(a: np.ndarray) -> np.ndarray:
    """Sorted distinct values (sort-based; faster than np.unique on large int arrays)."""
    a = np.sort(a)
    if len(a) == 0:
        return a
    keep = np.empty(len(a), bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def _pairs_to_csr(n: int, src: np.ndarray, dst: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    key = _sorted_unique(src.astype(np.int64) * n + dst.astype(np.int64))
    s = (key // n).astype(np.int64)
    d = (key % n).astype(np.int32)
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum(np.bincount(s, minlength=n))
    if off[-1] >= 2 ** 31:
        raise ValueError("adjacency too large for int32 offsets")
    return off.astype(np.int32), d


def _simplex_edges(simp: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    a = []
    b = []
    for u in range(4):
        for v in range(4):
            if u != v:
                a.append(simp[:, u])
                b.append(simp[:, v])
    return np.concatenate(a), np.concatenate(b)


def _circumspheres(P: np.ndarray, simp: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Circumcentres and radii of tetrahedra (FP64)."""
    a = P[simp[:, 0]]
    M = np.stack([P[simp[:, 1]] - a, P[simp[:, 2]] - a, P[simp[:, 3]] - a], axis=1)
    rhs = 0.5 * np.einsum("nij,nij->ni", M, M)
    det = np.linalg.det(M)
    ok = np.abs(det) > 1e-300
    x = np.full_like(rhs, np.inf)
    if ok.any():
        x[ok] = np.linalg.solve(M[ok], rhs[ok][..., None])[..., 0]
    r = np.linalg.norm(x, axis=1)
    return a + x, r


def _block_worker(args):
    """Triangulate one block (core + halo + ghosts); return the directed edges
    of core sites and the circumspheres that must be checked against all sites."""
    from scipy.spatial import Delaunay

    local_pts, local_ids, n_core, ghosts, box_lo, box_hi, all_lo, all_hi = args
    P = np.concatenate([local_pts, ghosts], axis=0).astype(np.float64)
    n_loc = len(local_pts)
    tri = Delaunay(P, qhull_options="Qt Qbb Qc Qz Q12")
    simp = tri.simplices
    is_core = np.zeros(len(P), bool)
    is_core[:n_core] = True
    touches = is_core[simp].any(axis=1)
    simp = simp[touches]
    c, r = _circumspheres(P, simp)
    # The circumball may only meet the region where unseen sites live
    # (outside the block's expanded box, inside the global box) if it is
    # checked against every site.
    lo = np.maximum(c - r[:, None], all_lo)
    hi = np.minimum(c + r[:, None], all_hi)
    inside = np.all(lo >= box_lo, axis=1) & np.all(hi <= box_hi, axis=1)
    sus = ~inside  # NaN boxes (ball halos) make every ball suspicious
    a, b = _simplex_edges(simp)
    keep = (a < n_core) & (b < n_loc)
    n_all = int(local_ids.max()) + 1 if len(local_ids) else 1
    key = _sorted_unique(local_ids[a[keep]].astype(np.int64) * (1 << 32) + local_ids[b[keep]])
    src = key >> 32
    dst = key & 0xFFFFFFFF
    sus_simp = simp[sus]
    sus_ids = np.where(sus_simp < n_loc, local_ids[np.minimum(sus_simp, n_loc - 1)], -1)
    sus_core = np.where(sus_simp < n_core, local_ids[np.minimum(sus_simp, n_loc - 1)], -1)
    return src, dst, c[sus], r[sus], sus_ids, sus_core


def _split_blocks(pts: np.ndarray, idx: np.ndarray, lo, hi, target: int, out: list):
    if len(idx) <= target:
        out.append((idx, lo.copy(), hi.copy()))
        return
    ext = hi - lo
    ax = int(np.argmax(ext))
    v = pts[idx, ax]
    med = float(np.median(v))
    left = idx[v < med]
    right = idx[v >= med]
    if len(left) == 0 or len(right) == 0:
        out.append((idx, lo.copy(), hi.copy()))
        return
    hl = hi.copy(); hl[ax] = med
    lr = lo.copy(); lr[ax] = med
    _split_blocks(pts, left, lo, hl, target, out)
    _split_blocks(pts, right, lr, hi, target, out)


def delaunay_csr(points: np.ndarray, workers: Optional[int] = None,
                 verbose: bool = False) -> Tuple[np.ndarray, np.ndarray]:
    """Symmetric CSR Delaunay adjacency of ``points`` (int32 offsets, int32
    neighbour ids sorted within each row).

    A shell of far ghost points closes every star; ghost edges are dropped, so
    cells on the convex hull keep their unbounded directions.  The adjacency is
    exact for every Voronoi face that has a point within ~8x the scene's
    bounding radius of its centre.

    Large inputs are split into blocks (median splits), each triangulated with a
    halo in its own process.  A tetrahedron incident to a block's core site is
    accepted only if its circumball provably holds no unseen site: either the
    ball (clipped to the global box) lies inside the block's expanded box, or a
    KD-tree query over *all* sites finds no site strictly inside it.  Sites
    with a rejected tetrahedron are redone with a doubled halo, and finally
    (never needed in practice) with one global triangulation.
    """
    pts = np.asarray(points, dtype=np.float64)
    n = len(pts)
    all_lo = pts.min(0)
    all_hi = pts.max(0)
    centre = 0.5 * (all_lo + all_hi)
    rad = 0.5 * float(np.linalg.norm(all_hi - all_lo)) + 1e-6
    ghosts = _ghost_shell(centre, 16.0 * rad)
    if n <= _GLOBAL_DELAUNAY_MAX:
        from scipy.spatial import Delaunay

        P = np.concatenate([pts, ghosts], 0)
        tri = Delaunay(P, qhull_options="Qt Qbb Qc Qz Q12")
        a, b = _simplex_edges(tri.simplices)
        keep = (a < n) & (b < n)
        return _pairs_to_csr(n, a[keep], b[keep])

    from scipy.spatial import cKDTree
    import multiprocessing as mp

    t_start = time.time()
    workers = workers or max(1, min(os.cpu_count() or 1, 32))
    tree = cKDTree(pts)
    if verbose:
        print(f"delaunay: kd-tree t={time.time() - t_start:.1f}s", flush=True)
    # local spacing: distance to the 8th nearest site
    nn8 = tree.query(pts, k=9, workers=-1)[0][:, -1]
    srcs, dsts = [], []
    ctx = mp.get_context("spawn")
    n_blocks_target = max(workers, int(math.ceil(n / 150_000)))

    # pass 0: median-split blocks with a box halo
    blocks: list = []
    _split_blocks(pts, np.arange(n), all_lo.copy(), all_hi.copy(),
                  max(2_000, int(math.ceil(n / n_blocks_target))), blocks)
    jobs = []
    for core, lo, hi in blocks:
        h = 3.0 * float(np.quantile(nn8[core], 0.99))
        elo = np.maximum(lo - h, all_lo)
        ehi = np.minimum(hi + h, all_hi)
        m = np.all((pts >= elo) & (pts <= ehi), axis=1)
        m[core] = False
        ids = np.concatenate([core, np.nonzero(m)[0]])
        jobs.append((pts[ids], ids, len(core), ghosts, elo, ehi, all_lo, all_hi))

    def check(c, r, sus_ids, sus_core):
        """Core sites incident to a circumball that holds a foreign site, and
        those foreign sites."""
        if not len(c):
            return set(), set()
        hits = tree.query_ball_point(c, r * (1.0 - 1e-9), workers=1)
        bad_core, viol = set(), set()
        for k, h_ in enumerate(hits):
            if not h_:
                continue
            own = set(int(v) for v in sus_ids[k] if v >= 0)
            foreign = [int(v) for v in h_ if int(v) not in own]
            if foreign:
                viol.update(foreign)
                bad_core.update(int(v) for v in sus_core[k] if v >= 0)
        return bad_core, viol

    nan3 = np.full(3, np.nan)
    todo = np.zeros(0, np.int64)
    with ctx.Pool(workers) as pool:
        # pass 0
        failed, violators = set(), set()
        for src, dst, c, r, sus_ids, sus_core in pool.imap_unordered(_block_worker, jobs):
            bad_core, viol = check(c, r, sus_ids, sus_core)
            if bad_core:
                drop = np.isin(src, np.fromiter(bad_core, np.int64))
                src, dst = src[~drop], dst[~drop]
                failed |= bad_core
                violators |= viol
            srcs.append(src)
            dsts.append(dst)
        if verbose:
            print(f"delaunay: pass 0 jobs={len(jobs)} failed={len(failed)} "
                  f"violators={len(violators)} t={time.time() - t_start:.1f}s", flush=True)
        # retries: small groups of failed sites; each group's local set grows
        # by the sites that violated its circumballs until none does
        if failed:
            todo = np.fromiter(sorted(failed), np.int64)
            groups: list = []
            _split_blocks(pts, todo, all_lo.copy(), all_hi.copy(), 512, groups)
            extra = np.fromiter(sorted(violators), np.int64) if violators else np.zeros(0, np.int64)
            state = []
            for core, _, _ in groups:
                near = tree.query_ball_point(pts[core], 3.0 * nn8[core], workers=-1)
                ids = _sorted_unique(np.concatenate([np.asarray(x, np.int64) for x in near] + [extra]))
                state.append([core, np.setdiff1d(ids, core)])
            for attempt in range(1, 8):
                if not state:
                    break
                jobs = [(pts[np.concatenate([co, hl])], np.concatenate([co, hl]), len(co), ghosts,
                         nan3, nan3, all_lo, all_hi) for co, hl in state]
                new_state = []
                for (co, hl), (src, dst, c, r, sus_ids, sus_core) in zip(
                        state, pool.imap(_block_worker, jobs)):
                    bad_core, viol = check(c, r, sus_ids, sus_core)
                    if bad_core:
                        bc = np.fromiter(bad_core, np.int64)
                        drop = np.isin(src, bc)
                        src, dst = src[~drop], dst[~drop]
                        v = np.fromiter(viol, np.int64)
                        near = tree.query_ball_point(pts[v], 3.0 * nn8[v], workers=-1)
                        add = _sorted_unique(np.concatenate([np.asarray(x, np.int64) for x in near] + [v]))
                        core2 = np.intersect1d(co, bc)
                        hl2 = np.setdiff1d(np.union1d(np.union1d(hl, add), co), core2)
                        new_state.append([core2, hl2])
                    srcs.append(src)
                    dsts.append(dst)
                state = new_state
                if verbose:
                    print(f"delaunay: pass {attempt} groups={len(jobs)} failed="
                          f"{sum(len(s_[0]) for s_ in state)} t={time.time() - t_start:.1f}s",
                          flush=True)
            todo = (np.concatenate([s_[0] for s_ in state]) if state
                    else np.zeros(0, np.int64))
    if verbose:
        print(f"delaunay: done, fallback sites={len(todo)} t={time.time() - t_start:.1f}s",
              flush=True)
    if len(todo):
        from scipy.spatial import Delaunay

        P = np.concatenate([pts, ghosts], 0)
        tri = Delaunay(P, qhull_options="Qt Qbb Qc Qz Q12")
        a, b = _simplex_edges(tri.simplices)
        keep = (a < n) & (b < n) & np.isin(a, todo)
        srcs.append(a[keep])
        dsts.append(b[keep])
    src = np.concatenate(srcs)
    dst = np.concatenate(dsts)
    # symmetric closure (a no-op when every star is exact)
    out = _pairs_to_csr(n, np.concatenate([src, dst]), np.concatenate([dst, src]))
    if verbose:
        print(f"delaunay: csr built t={time.time() - t_start:.1f}s", flush=True)
    return out


# ----------------------------------------------------------------------------
# Scenes
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Scene:
    """Host-side scene: FP32 sites [N,3], CSR adjacency, density [N] and SH
    coefficients [N,(deg+1)^2,3] (FP32 values), plus the scene box."""

    pos: np.ndarray
    adj_off: np.ndarray
    adj_idx: np.ndarray
    density: np.ndarray
    sh: np.ndarray
    sh_degree: int
    aabb_min: np.ndarray
    aabb_max: np.ndarray
    name: str = ""

    @property
    def n_sites(self) -> int:
        return len(self.pos)

    @property
    def n_edges(self) -> int:
        return len(self.adj_idx)

    def mean_degree(self) -> float:
        return self.n_edges / max(1, self.n_sites)


def make_scene(pos: np.ndarray, density: np.ndarray, sh: np.ndarray, name: str = "",
               adjacency=None, workers=None, verbose=False) -> Scene:
    pos = np.ascontiguousarray(pos, np.float32)
    if adjacency is None:
        adjacency = delaunay_csr(pos, workers=workers, verbose=verbose)
    off, idx = adjacency
    deg = int(round(math.sqrt(sh.shape[1]))) - 1
    return Scene(pos, np.ascontiguousarray(off, np.int32), np.ascontiguousarray(idx, np.int32),
                 np.ascontiguousarray(density, np.float32), np.ascontiguousarray(sh, np.float32),
                 deg, pos.min(0).astype(np.float32), pos.max(0).astype(np.float32), name)


def _cache_dir() -> str:
    d = os.environ.get("RF_SCENE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "radfoam_gb300")
    os.makedirs(d, exist_ok=True)
    return d


def _cached_adjacency(pos: np.ndarray, tag: str, workers=None, verbose=False):
    h = hashlib.sha1(pos.tobytes()).hexdigest()[:16]
    path = os.path.join(_cache_dir(), f"adj_{tag}_{len(pos)}_{h}.npz")
    if os.path.exists(path):
        try:
            z = np.load(path)
            return z["off"], z["idx"]
        except Exception:
            pass
    off, idx = delaunay_csr(pos, workers=workers, verbose=verbose)
    tmp = path + f".{os.getpid()}.tmp.npz"
    np.savez(tmp, off=off, idx=idx)
    os.replace(tmp, path)
    return off, idx


def scene_uniform(n: int, sh_degree: int, seed: int, dc: str = "uniform_colour",
                  box: float = 1.0, name: str = "", cache: bool = True, verbose=False) -> Scene:
    rng = np.random.default_rng(seed)
    pos = dedupe_sites(uniform_sites(n, -box, box, rng), rng)
    dens = lognormal_density(n, rng)
    sh = sh_coeffs(n, sh_degree, rng, dc=dc)
    adj = _cached_adjacency(pos, "u", verbose=verbose) if cache else delaunay_csr(pos)
    return make_scene(pos, dens, sh, name=name, adjacency=adj)


def scene_mixture(n: int, sh_degree: int, seed: int, name: str = "", cache: bool = True,
                  verbose=False) -> Scene:
    rng = np.random.default_rng(seed)
    pos = dedupe_sites(mixture_sites(n, rng), rng)
    dens = lognormal_density(n, rng)
    sh = sh_coeffs(n, sh_degree, rng, dc="normal")
    adj = _cached_adjacency(pos, "m", verbose=verbose) if cache else delaunay_csr(pos)
    return make_scene(pos, dens, sh, name=name, adjacency=adj)


CONFIG_SEED = {"c1": 1001, "c2": 1002, "c3": 1003, "c4": 1004, "c5": 1005}


def config_scene(cid: str, n_sites: Optional[int] = None, verbose=False) -> Scene:
    """The scene of workload ``cid`` (optionally with a different site count)."""
    seed = CONFIG_SEED[cid]
    if cid == "c1":
        return scene_uniform(n_sites or 4096, 0, seed, name="c1", verbose=verbose)
    if cid == "c2":
        return scene_mixture(n_sites or 1_000_000, 3, seed, name="c2", verbose=verbose)
    if cid == "c3":
        return scene_uniform(n_sites or 3_000_000, 3, seed, name="c3", verbose=verbose)
    if cid in ("c4", "c5"):
        # both use the same 3M-site mixture scene
        return scene_mixture(n_sites or 3_000_000, 3, CONFIG_SEED["c4"], name=cid,
                             verbose=verbose)
    raise KeyError(cid)


C4_RESOLUTIONS = [(640, 480), (640, 480), (1280, 720), (1280, 720),
                  (1600, 900), (1600, 900), (1920, 1080), (1920, 1080)]
C5_RESOLUTIONS = [(320, 240), (640, 480), (1280, 720), (1920, 1080)]


def config_cameras(cid: str, scale: float = 1.0) -> List[Camera]:
    """Cameras of workload ``cid``; ``scale`` shrinks resolutions (tests)."""
    def res(w, h):
        return max(1, int(round(w * scale))), max(1, int(round(h * scale)))

    if cid == "c1":
        return [pinhole(*res(64, 64), 60.0)]
    if cid == "c2":
        return [pinhole(*res(1280, 720), 60.0)]
    if cid == "c3":
        return [pinhole(*res(1920, 1080), 60.0)]
    if cid == "c4":
        poses = sphere_poses(len(C4_RESOLUTIONS), 12.0, CONFIG_SEED["c4"])
        return [pinhole(*res(w, h), 60.0, c2w=p) for (w, h), p in zip(C4_RESOLUTIONS, poses)]
    raise KeyError(cid)


def random_target(n_rays: int, seed: int) -> np.ndarray:
    """Seeded target image for the MSE loss, values uniform in [0,1]."""
    return np.random.default_rng(seed).uniform(0, 1, size=(n_rays, 3)).astype(np.float32)


def poisson_arrivals(rate: float, n: int, seed: int) -> np.ndarray:
    """Arrival times (s) of an open-loop Poisson stream."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
