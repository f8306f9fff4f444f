"""FP64 CPU oracle for Radiant Foam ray tracing (arXiv 2502.01157).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package.  The CUDA
renderer does not use it, and the two share no code.

The arithmetic lives in ``rf_oracle.c`` (plain C, FP64, OpenMP over rays); this
module compiles it with gcc on first use and marshals numpy arrays.  Every
function follows the paper's statement of the method:

* :func:`camera_rays`  -- pinhole or equidistant-fisheye rays through pixel
  centres, with an optional rolling shutter (the inputs o, d of Alg. 1).
* :func:`nearest_site` -- nn(o), the initial cell of Alg. 1.
* :func:`render`       -- Alg. 1 with Eq. (3)-(4) compositing (Sec. 3.1-3.2).
* :func:`render_bwd`   -- reverse-mode gradient of the rendered outputs; sites
  receive gradient only through segment widths (Sec. 3.1).
* :func:`sh_basis`     -- real spherical harmonics of degree <= 3 (Sec. 3.4).
* :func:`render_quantile` -- the quantile loss of Eq. (6) per ray (Sec. 3.3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rf_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "adjacency.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "librf_oracle.so")
_lock = threading.Lock()
_lib = None

RAY_OK = 0
RAY_MAX_STEPS = 1

# Near-degenerate ray classes (bit flags of ``render(...)["flags"]``): why a
# correct FP32 renderer may differ from this FP64 walk on a ray.
FLAG_EDGE = 1     # passes within tau of a Voronoi edge or vertex: the next cell is a tie
FLAG_CAMERA = 2   # the start point is within tau of the bisector of its two nearest sites
FLAG_STOP = 4     # T within a relative 1e-3 of eps at a stop test: may stop one step apart
FLAG_GRAZE = 8    # a face crossed at grazing incidence: ill-conditioned position gradient
FLAG_BEND = 16    # sphere hit near tangency / refraction near the critical angle
FLAG_NAMES = {FLAG_EDGE: "edge", FLAG_CAMERA: "camera", FLAG_STOP: "stop", FLAG_GRAZE: "graze",
              FLAG_BEND: "bend"}


def flag_counts(flags) -> dict:
    """Number of rays in each near-degenerate class (a ray may be in several)."""
    f = np.asarray(flags)
    out = {name: int(np.count_nonzero(f & bit)) for bit, name in FLAG_NAMES.items()}
    out["any"] = int(np.count_nonzero(f))
    out["rays"] = int(f.size)
    return out

_d = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.POINTER(ctypes.c_int64)
_i32 = ctypes.POINTER(ctypes.c_int32)
_u8 = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile rf_oracle.c into a shared library (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", *_SRCS, "-o", tmp, "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:  # no OpenMP runtime: build serial
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_sh_basis_batch.argtypes = [ctypes.c_int, ctypes.c_int64, _d, _d]
            L.orc_sh_basis_batch.restype = ctypes.c_int
            L.orc_camera_ray.argtypes = [_d, ctypes.c_int64, _d, _d]
            L.orc_camera_ray.restype = None
            L.orc_nearest_site.argtypes = [ctypes.c_int64, _d, _d, _d]
            L.orc_nearest_site.restype = ctypes.c_int64
            L.orc_camera_start.argtypes = [ctypes.c_int64, _d, _d, _d]
            L.orc_camera_start.restype = None
            L.orc_render.argtypes = [ctypes.c_int64, _d, _i64, _i32, _d, _d, ctypes.c_int, _d,
                                     _d, ctypes.c_int64, _i64, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_double, _d, _d, _d, _i32, _u8, _u8, ctypes.c_int,
                                     _i32, _d, _d, _d, ctypes.c_int]
            L.orc_render.restype = ctypes.c_int
            L.orc_render_bwd.argtypes = [ctypes.c_int64, _d, _i64, _i32, _d, _d, ctypes.c_int, _d,
                                         _d, ctypes.c_int64, _i64, ctypes.c_double, ctypes.c_int,
                                         _d, _d, _d, _d, _d, _d, _d, _d, _d, ctypes.c_int]
            L.orc_render_quantile.argtypes = [ctypes.c_int64, _d, _i64, _i32, _d, _d, ctypes.c_int,
                                              _d, _d, ctypes.c_int64, _i64, ctypes.c_double,
                                              ctypes.c_int, _d, _d, _d, ctypes.c_int]
            L.orc_render_quantile.restype = ctypes.c_int
            L.orc_render_bwd.restype = ctypes.c_int
            L.orc_voronoi_faces.argtypes = [ctypes.c_int64, _d, ctypes.c_int64, _i64, _i64, _i64, _d,
                                             _d, _d, ctypes.c_int]
            L.orc_voronoi_faces.restype = ctypes.c_int
            L.orc_num_threads.argtypes = []
            L.orc_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _cam(cam) -> np.ndarray:
    c = _f64(cam.as_f64() if hasattr(cam, "as_f64") else cam)
    if len(c) == 20:  # pinhole, global shutter
        c = np.concatenate([c, np.zeros(4)])
    return c


def _fx(effects):
    """Sphere effect as 6 doubles {max_bounces, centre, radius, ior}, or None."""
    if effects is None:
        return None
    return _f64(effects.as_f64() if hasattr(effects, "as_f64") else effects)


def default_tau(scene, cam) -> float:
    """Degeneracy distance: 1e-6 in units of the scene's coordinate magnitude
    (at least 1), i.e. a fixed number of FP32 ulps of the coordinates."""
    c = _cam(cam)
    mag = max(1.0, float(np.max(np.abs(scene.aabb_min))), float(np.max(np.abs(scene.aabb_max))),
              float(np.max(np.abs(c[[3, 7, 11]]))))
    return 1e-6 * mag


class _SceneF64:
    """FP64 copies of a scene's arrays in the layout the C code reads."""

    def __init__(self, scene):
        self.n = int(len(scene.pos))
        self.pos = _f64(scene.pos).reshape(-1)
        self.off = np.ascontiguousarray(scene.adj_off, dtype=np.int64)
        self.adj = np.ascontiguousarray(scene.adj_idx, dtype=np.int32)
        self.sigma = _f64(scene.density).reshape(-1)
        self.sh = _f64(scene.sh).reshape(-1)
        self.deg = int(scene.sh_degree)
        self.box = _f64(np.concatenate([np.asarray(scene.aabb_min, np.float64).reshape(3),
                                        np.asarray(scene.aabb_max, np.float64).reshape(3)]))


class Prepared:
    """A scene converted to FP64 once, for many oracle calls on it (the
    conversion of a 3M-site scene's SH rows takes longer than rendering a
    few thousand rays).  The start cell nn(o) of each camera centre is also
    found once and kept.  Pass it wherever a scene is expected."""

    def __init__(self, scene):
        self.f64 = _SceneF64(scene)
        self.aabb_min = np.asarray(scene.aabb_min)
        self.aabb_max = np.asarray(scene.aabb_max)
        self.n_sites = self.f64.n
        self.sh_degree = self.f64.deg
        self._starts = {}

    def start_info(self, cam) -> np.ndarray:
        c = _cam(cam)
        key = c[:12].tobytes()
        if key not in self._starts:
            out = np.zeros(2)
            lib().orc_camera_start(self.f64.n, _p(self.f64.pos, _d), _p(c, _d), _p(out, _d))
            self._starts[key] = out
        return self._starts[key]


def prepare(scene) -> Prepared:
    return scene if isinstance(scene, Prepared) else Prepared(scene)


def _scene_args(scene, cam):
    """(FP64 scene, start info or None) for a scene or a Prepared one."""
    if isinstance(scene, Prepared):
        return scene.f64, scene.start_info(cam)
    return _SceneF64(scene), None


def sh_basis(degree: int, dirs) -> np.ndarray:
    d = _f64(dirs).reshape(-1, 3)
    K = (degree + 1) ** 2
    out = np.zeros((len(d), K))
    if lib().orc_sh_basis_batch(int(degree), len(d), _p(d, _d), _p(out, _d)):
        raise ValueError("degree must be 0..3")
    return out


def camera_rays(cam, pixels=None):
    c = _cam(cam)
    n = int(c[16]) * int(c[17])
    px = np.arange(n, dtype=np.int64) if pixels is None else np.asarray(pixels, np.int64)
    o = np.zeros((len(px), 3))
    d = np.zeros((len(px), 3))
    L = lib()
    for k, p in enumerate(px):
        L.orc_camera_ray(_p(c, _d), int(p), _p(o[k], _d), _p(d[k], _d))
    return o, d


def nearest_site(pos, q):
    P = _f64(pos).reshape(-1)
    Q = _f64(q).reshape(3)
    gap = np.zeros(1)
    i = lib().orc_nearest_site(len(P) // 3, _p(P, _d), _p(Q, _d), _p(gap, _d))
    return int(i), float(gap[0])


def render(scene, cam, pixels=None, eps: float = 1e-4, max_steps: int = 1 << 16,
           tau=None, trace: int = 0, threads: int = 0, effects=None) -> dict:
    """Forward render (Alg. 1, Eq. 3-4).  Returns rgb [R,3], trans [R], depth [R],
    steps [R], status [R] and, if ``trace > 0``, trace_cells [R,trace] (-1
    padded) and trace_t [R,trace].  ``effects``: an analytic sphere the rays
    reflect off or refract through (``scenes.Sphere``).

    Near-degenerate rays: ``flags`` [R] (FLAG_* bits) and three views of it:
    ``tie`` (EDGE or CAMERA: the visited cells may differ at FP32), ``stop_tie``
    (STOP: the walk may end one step earlier or later) and ``degen`` (any
    flag: the gradient may carry the conditioning error)."""
    fx = _fx(effects)
    S, st0 = _scene_args(scene, cam)
    c = _cam(cam)
    n_all = int(c[16]) * int(c[17])
    px = None if pixels is None else np.ascontiguousarray(pixels, np.int64)
    R = n_all if px is None else len(px)
    tau = default_tau(scene, cam) if tau is None else float(tau)
    rgb = np.zeros((R, 3))
    tr = np.zeros(R)
    dp = np.zeros(R)
    st = np.zeros(R, np.int32)
    ss = np.zeros(R, np.uint8)
    fl = np.zeros(R, np.uint8)
    tc = np.full((R, max(trace, 1)), -1, np.int32)
    tt = np.full((R, max(trace, 1)), np.nan)
    rc = lib().orc_render(S.n, _p(S.pos, _d), _p(S.off, _i64), _p(S.adj, _i32), _p(S.sigma, _d),
                          _p(S.sh, _d), S.deg, _p(S.box, _d), _p(c, _d), R, _p(px, _i64),
                          float(eps), int(max_steps), tau, _p(rgb, _d), _p(tr, _d), _p(dp, _d),
                          _p(st, _i32), _p(ss, _u8), _p(fl, _u8), int(trace), _p(tc, _i32),
                          _p(tt, _d), _p(fx, _d), _p(st0, _d), int(threads))
    if rc:
        raise ValueError("oracle render: bad arguments")
    out = dict(rgb=rgb, trans=tr, depth=dp, steps=st, status=ss, flags=fl, tau=tau,
               tie=(fl & (FLAG_EDGE | FLAG_CAMERA)) != 0, stop_tie=(fl & FLAG_STOP) != 0,
               degen=fl != 0)
    if trace > 0:
        out["trace_cells"] = tc
        out["trace_t"] = tt
    return out


def render_quantile(scene, cam, pixels=None, eps: float = 1e-4, max_steps: int = 1 << 16,
                    threads: int = 0, effects=None) -> np.ndarray:
    """Quantile loss of Eq. (6) per ray: E|W^-1(u1) - W^-1(u2)|, u1, u2 ~ U[0,1],
    W^-1 the quantile function of the ray's normalised weight distribution."""
    fx = _fx(effects)
    S, st0 = _scene_args(scene, cam)
    c = _cam(cam)
    n_all = int(c[16]) * int(c[17])
    px = None if pixels is None else np.ascontiguousarray(pixels, np.int64)
    R = n_all if px is None else len(px)
    q = np.zeros(R)
    rc = lib().orc_render_quantile(S.n, _p(S.pos, _d), _p(S.off, _i64), _p(S.adj, _i32),
                                   _p(S.sigma, _d), _p(S.sh, _d), S.deg, _p(S.box, _d), _p(c, _d),
                                   R, _p(px, _i64), float(eps), int(max_steps), _p(q, _d),
                                   _p(fx, _d), _p(st0, _d), int(threads))
    if rc:
        raise ValueError("oracle render_quantile: bad arguments")
    return q


def render_bwd(scene, cam, g_rgb, g_trans=None, g_depth=None, pixels=None, eps: float = 1e-4,
               max_steps: int = 1 << 16, threads: int = 0, g_quantile=None,
               effects=None) -> dict:
    """Gradient of sum(g_rgb*rgb) + sum(g_trans*trans) + sum(g_depth*depth)
    + sum(g_quantile*quantile) with respect to density [N], SH [N,K,3] and
    positions [N,3]."""
    fx = _fx(effects)
    S, st0 = _scene_args(scene, cam)
    c = _cam(cam)
    n_all = int(c[16]) * int(c[17])
    px = None if pixels is None else np.ascontiguousarray(pixels, np.int64)
    R = n_all if px is None else len(px)
    gr = _f64(g_rgb).reshape(R, 3)
    gt = None if g_trans is None else _f64(g_trans).reshape(R)
    gd = None if g_depth is None else _f64(g_depth).reshape(R)
    gq = None if g_quantile is None else _f64(g_quantile).reshape(R)
    K = (S.deg + 1) ** 2
    g_sigma = np.zeros(S.n)
    g_sh = np.zeros((S.n, K, 3))
    g_pos = np.zeros((S.n, 3))
    rc = lib().orc_render_bwd(S.n, _p(S.pos, _d), _p(S.off, _i64), _p(S.adj, _i32),
                              _p(S.sigma, _d), _p(S.sh, _d), S.deg, _p(S.box, _d), _p(c, _d), R,
                              _p(px, _i64), float(eps), int(max_steps), _p(gr, _d), _p(gt, _d),
                              _p(gd, _d), _p(gq, _d), _p(g_sigma, _d), _p(g_sh, _d), _p(g_pos, _d),
                              _p(fx, _d), _p(st0, _d), int(threads))
    if rc:
        raise ValueError("oracle render_bwd: bad arguments")
    return dict(density=g_sigma, sh=g_sh, pos=g_pos)
