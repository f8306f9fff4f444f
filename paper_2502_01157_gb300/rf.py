"""Python binding of the C-ABI renderer ``librf.so`` (argument marshalling only).

Every step of the ray-tracing path runs in the library's CUDA kernels; this
module passes device pointers of torch tensors and the current CUDA stream.
There is no CPU fallback: if the library is missing or no GPU is present the
calls raise.

Main entry points:

* :class:`Foam` -- a packed scene (sites, Delaunay CSR adjacency, density and
  SH attributes) resident on the GPU;
* :meth:`Foam.render` / :meth:`Foam.backward` -- ``rf_render_fwd`` /
  ``rf_render_bwd``;
* :func:`render` -- differentiable render (``torch.autograd.Function``) with
  respect to density, SH coefficients and site positions.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import build as _build

RF_OK = 0
RF_F32, RF_BF16, RF_F16 = 0, 1, 2
RAY_OK, RAY_MAX_STEPS = 0, 1
_DTYPES = {torch.float32: RF_F32, torch.bfloat16: RF_BF16, torch.float16: RF_F16}


class rf_camera(ctypes.Structure):
    _fields_ = [("c2w", ctypes.c_float * 12), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("t_near", ctypes.c_float), ("t_far", ctypes.c_float),
                ("model", ctypes.c_int32), ("shutter", ctypes.c_float * 3)]


class rf_scene_desc(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int64), ("n_edges", ctypes.c_int64),
                ("pos", ctypes.c_void_p), ("adj_off", ctypes.c_void_p),
                ("adj_idx", ctypes.c_void_p), ("density", ctypes.c_void_p),
                ("sh", ctypes.c_void_p), ("sh_degree", ctypes.c_int32),
                ("attr_dtype", ctypes.c_int32), ("aabb_min", ctypes.c_float * 3),
                ("aabb_max", ctypes.c_float * 3)]


class rf_render_opts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_float), ("max_steps", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_int32),
                ("max_bounces", ctypes.c_int32), ("sphere", ctypes.c_float * 4),
                ("sphere_ior", ctypes.c_float)]


class rf_serve_config(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int32),
                ("n_streams", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("eps", ctypes.c_float), ("max_steps", ctypes.c_int32)]


class rf_serve_metrics(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("rays_done", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("mrays_s", ctypes.c_double), ("mean_batch", ctypes.c_double),
                ("max_busy_streams", ctypes.c_int32), ("inflight", ctypes.c_int32)]


class rf_fwd_outputs(ctypes.Structure):
    _fields_ = [("rgb", ctypes.c_void_p), ("trans", ctypes.c_void_p), ("depth", ctypes.c_void_p),
                ("steps", ctypes.c_void_p), ("ray_status", ctypes.c_void_p),
                ("quantile", ctypes.c_void_p), ("quantile_aux", ctypes.c_void_p),
                ("walk_record", ctypes.c_void_p), ("walk_record_bytes", ctypes.c_size_t),
                ("walk_record_steps", ctypes.c_int32)]


class rf_bwd_inputs(ctypes.Structure):
    _fields_ = [("rgb", ctypes.c_void_p), ("trans", ctypes.c_void_p), ("depth", ctypes.c_void_p),
                ("quantile_aux", ctypes.c_void_p), ("d_rgb", ctypes.c_void_p),
                ("d_trans", ctypes.c_void_p), ("d_depth", ctypes.c_void_p),
                ("d_quantile", ctypes.c_void_p), ("walk_record", ctypes.c_void_p),
                ("walk_record_bytes", ctypes.c_size_t), ("walk_record_steps", ctypes.c_int32)]


class rf_grads(ctypes.Structure):
    _fields_ = [("density", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("pos", ctypes.c_void_p)]


class rf_adjacency_stats(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int64), ("n_edges", ctypes.c_int64),
                ("edges_before_symmetry", ctypes.c_int64), ("asym_added", ctypes.c_int64),
                ("wide_sites", ctypes.c_int64), ("failed_sites", ctypes.c_int64),
                ("fp64_tests", ctypes.c_int64), ("max_degree", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("domain", ctypes.c_float * 6)]


class RFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rf error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None
_P = ctypes.c_void_p
_S = ctypes.c_int32

# name -> (restype, argtypes); every symbol include/rf.h declares
SIGNATURES = {
    "rf_version": (ctypes.c_int32, []),
    "rf_last_error": (ctypes.c_char_p, []),
    "rf_scene_create": (_S, [ctypes.POINTER(rf_scene_desc), _P, ctypes.POINTER(_P)]),
    "rf_scene_set_attributes": (_S, [_P, _P, _P, ctypes.c_int32]),
    "rf_scene_update_positions": (_S, [_P, _P, _P]),
    "rf_scene_info": (_S, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                           ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_size_t)]),
    "rf_scene_destroy": (_S, [_P]),
    "rf_render_fwd": (_S, [_P, ctypes.POINTER(rf_camera), ctypes.c_int32,
                           ctypes.POINTER(rf_render_opts), _P, _P, _P, _P, _P, _P]),
    "rf_render_bwd": (_S, [_P, ctypes.POINTER(rf_camera), ctypes.c_int32,
                           ctypes.POINTER(rf_render_opts), _P, _P, _P, _P, _P, _P, _P, _P, _P,
                           _P]),
    "rf_render_fwd_ex": (_S, [_P, ctypes.POINTER(rf_camera), ctypes.c_int32,
                              ctypes.POINTER(rf_render_opts), ctypes.POINTER(rf_fwd_outputs), _P]),
    "rf_render_bwd_ex": (_S, [_P, ctypes.POINTER(rf_camera), ctypes.c_int32,
                              ctypes.POINTER(rf_render_opts), ctypes.POINTER(rf_bwd_inputs),
                              ctypes.POINTER(rf_grads), _P]),
    "rf_trace_cells": (_S, [_P, ctypes.POINTER(rf_camera), ctypes.POINTER(rf_render_opts),
                            ctypes.c_int32, _P, _P, _P]),
    "rf_mse_grad": (_S, [_P, _P, ctypes.c_int64, ctypes.c_float, _P, _P, _P]),
    "rf_walk_record_bytes": (ctypes.c_size_t, [ctypes.POINTER(rf_camera), ctypes.c_int32, ctypes.c_int32]),
    "rf_adjacency_create": (_S, [ctypes.POINTER(_P)]),
    "rf_adjacency_build": (_S, [_P, ctypes.c_int64, _P, ctypes.POINTER(ctypes.c_float), ctypes.c_int32,
                                _P]),
    "rf_adjacency_result": (_S, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                 ctypes.POINTER(rf_adjacency_stats)]),
    "rf_adjacency_copy": (_S, [_P, _P, _P, _P]),
    "rf_adjacency_destroy": (_S, [_P]),
    "rf_serve_create": (_S, [_P, ctypes.POINTER(rf_serve_config), ctypes.POINTER(_P)]),
    "rf_serve_submit": (_S, [_P, ctypes.POINTER(rf_camera), ctypes.POINTER(ctypes.c_uint64)]),
    "rf_serve_poll": (_S, [_P, ctypes.c_uint64, _P, ctypes.POINTER(ctypes.c_int32),
                           ctypes.POINTER(ctypes.c_double)]),
    "rf_serve_wait": (_S, [_P, ctypes.c_uint64, ctypes.c_int32, _P,
                           ctypes.POINTER(ctypes.c_double)]),
    "rf_serve_stats": (_S, [_P, ctypes.POINTER(rf_serve_metrics)]),
    "rf_serve_reset_stats": (_S, [_P]),
    "rf_serve_destroy": (_S, [_P]),
    "rf_densify_scores": (_S, [_P, _P, _P, _P]),
    "rf_prune_mask": (_S, [_P, ctypes.c_float, _P, _P]),
    "rf_multinomial_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int64]),
    "rf_sample_multinomial": (_S, [_P, ctypes.c_int64, _P, ctypes.c_int64, _P, ctypes.c_size_t, _P,
                                   _P]),
    "rf_render_fwd_noalloc": (_S, [ctypes.c_int64, ctypes.c_int64, _P, _P, _P, _P, _P,
                                   ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_float),
                                   ctypes.POINTER(rf_camera), ctypes.c_int32,
                                   ctypes.POINTER(rf_render_opts), _P, _P, _P, _P]),
}


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load librf.so (building it with nvcc if absent)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"{path} not built")
                _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc: int):
    if rc != RF_OK:
        raise RFError(rc, lib().rf_last_error().decode(errors="replace"))


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _addr(t: Optional[torch.Tensor]):
    p = _ptr(t)
    return None if p is None else p.value


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def camera_struct(cam) -> rf_camera:
    c = rf_camera()
    c.c2w[:] = [float(v) for v in np.asarray(cam.c2w, np.float32).reshape(-1)]
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.width, c.height = int(cam.width), int(cam.height)
    c.t_near, c.t_far = cam.t_near, cam.t_far
    c.model = int(getattr(cam, "model", 0))
    c.shutter[:] = [float(v) for v in getattr(cam, "shutter", (0.0, 0.0, 0.0))]
    return c


def camera_array(cams) -> "ctypes.Array":
    cams = list(cams) if isinstance(cams, (list, tuple)) else [cams]
    arr = (rf_camera * len(cams))()
    for k, c in enumerate(cams):
        arr[k] = camera_struct(c)
    return arr


def walk_record_bytes(cams, steps: int) -> int:
    """Bytes of a walk record of ``steps`` steps per ray for ``cams``."""
    ca = camera_array(cams)
    return int(lib().rf_walk_record_bytes(ca, len(ca), int(steps)))


RF_RENDER_SHARED_CELLS = 1


def opts_struct(eps: float = 1e-4, max_steps: int = 0, effects=None, shared_cells: bool = False) -> rf_render_opts:
    """Render options; ``effects`` is an analytic sphere with ``centre``,
    ``radius``, ``ior`` (0: mirror) and ``max_bounces`` (e.g. ``scenes.Sphere``);
    ``shared_cells`` selects the backward for frames whose rays share cells
    heavily (``RF_RENDER_SHARED_CELLS``)."""
    o = rf_render_opts()
    o.eps = float(eps)
    o.max_steps = int(max_steps)
    o.flags = RF_RENDER_SHARED_CELLS if shared_cells else 0
    if effects is not None:
        o.max_bounces = int(effects.max_bounces)
        o.sphere[:] = [float(v) for v in effects.centre] + [float(effects.radius)]
        o.sphere_ior = float(effects.ior)
    return o


def n_rays_of(cams) -> int:
    cams = list(cams) if isinstance(cams, (list, tuple)) else [cams]
    return sum(int(c.width) * int(c.height) for c in cams)


class Foam:
    """A Voronoi foam packed for traversal on the current CUDA device.

    ``pos`` [N,3] float32, ``adj_off`` [N+1] / ``adj_idx`` [E] int32 and the
    attributes ``density`` [N] and ``sh`` [N,(deg+1)^2,3] (float32, bfloat16
    or float16) are CUDA tensors.  The attributes are borrowed by the library:
    this object keeps references to them.
    """

    def __init__(self, pos, adj_off, adj_idx, density, sh, aabb=None, stream=None):
        self.pos = pos.contiguous()
        self._aabb = aabb
        self._topology = 0     # bumped when the neighbour lists are replaced
        self._attrs(density, sh)
        self._create(adj_off, adj_idx, stream)

    def _create(self, adj_off, adj_idx, stream=None):
        L = lib()
        aabb = self._aabb
        self.adj_off = adj_off.to(torch.int32).contiguous()
        self.adj_idx = adj_idx.to(torch.int32).contiguous()
        d = rf_scene_desc()
        d.n_sites = int(self.pos.shape[0])
        d.n_edges = int(self.adj_idx.shape[0])
        d.pos = _ptr(self.pos).value
        d.adj_off = _ptr(self.adj_off).value
        d.adj_idx = _ptr(self.adj_idx).value if d.n_edges else None
        d.density = _ptr(self.density).value
        d.sh = _ptr(self.sh).value
        d.sh_degree = self.sh_degree
        d.attr_dtype = self.attr_dtype
        if aabb is None:
            d.aabb_min[:] = [1.0, 1.0, 1.0]
            d.aabb_max[:] = [0.0, 0.0, 0.0]  # min > max: computed on the device
        else:
            d.aabb_min[:] = [float(v) for v in aabb[0]]
            d.aabb_max[:] = [float(v) for v in aabb[1]]
        h = ctypes.c_void_p()
        _check(L.rf_scene_create(ctypes.byref(d), _stream(stream), ctypes.byref(h)))
        self._h = h
        self._pos_version = self.pos._version
        self._topology = getattr(self, "_topology", 0) + 1

    def _attrs(self, density, sh):
        if density.dtype not in _DTYPES or sh.dtype != density.dtype:
            raise ValueError("density and sh must share one of float32/bfloat16/float16")
        self.density = density.contiguous()
        self.sh = sh.contiguous()
        K = int(self.sh.shape[1])
        deg = int(round(K ** 0.5)) - 1
        if (deg + 1) ** 2 != K or self.sh.shape[2] != 3 or not 0 <= deg <= 3:
            raise ValueError("sh must be [N,(deg+1)^2,3] with deg <= 3")
        self.sh_degree = deg
        self.attr_dtype = _DTYPES[density.dtype]

    @classmethod
    def from_scene(cls, scene, device="cuda", attr_dtype=torch.float32, stream=None):
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(device=device, dtype=dt)
        return cls(t(scene.pos, torch.float32), t(scene.adj_off, torch.int32),
                   t(scene.adj_idx, torch.int32), t(scene.density, attr_dtype),
                   t(scene.sh, attr_dtype),
                   aabb=(scene.aabb_min, scene.aabb_max), stream=stream)

    @classmethod
    def from_sites(cls, pos, density, sh, domain=None, aabb=None, adjacency=None, stream=None):
        """A foam whose neighbour lists are built on the GPU from ``pos`` (an
        :class:`Adjacency` may be passed to reuse its buffers)."""
        builder = adjacency if adjacency is not None else Adjacency()
        off, idx = builder.build(pos, domain=domain, stream=stream)
        foam = cls(pos, off, idx, density, sh, aabb=aabb, stream=stream)
        foam.adjacency_stats = builder.stats
        foam._builder = builder
        return foam

    def rebuild_adjacency(self, builder=None, domain=None, incremental: bool = False, stream=None):
        """Rebuild the neighbour lists on the GPU from the current positions
        (after position steps) and re-pack the foam with them.  ``builder``:
        an :class:`Adjacency` kept between rebuilds (one is made and kept on
        the foam otherwise); ``incremental`` seeds each cell with its previous
        neighbours (the builder's previous result)."""
        if builder is None:
            builder = getattr(self, "_builder", None) or Adjacency()
            self._builder = builder
        off, idx = builder.build(self.pos, domain=domain, incremental=incremental, stream=stream)
        old = self._h
        self._h = None
        self._create(off, idx, stream)
        if old is not None:
            lib().rf_scene_destroy(old)
        self.adjacency_stats = builder.stats
        return builder.stats

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("foam is closed")
        return self._h

    @property
    def n_sites(self) -> int:
        return int(self.pos.shape[0])

    def info(self) -> dict:
        n, e = ctypes.c_int64(), ctypes.c_int64()
        box = (ctypes.c_float * 6)()
        b = ctypes.c_size_t()
        _check(lib().rf_scene_info(self.handle, ctypes.byref(n), ctypes.byref(e), box,
                                   ctypes.byref(b)))
        return dict(n_sites=n.value, n_edges=e.value, aabb=list(box), device_bytes=b.value)

    def state(self):
        """What a render reads from this foam: the adjacency generation and
        the attribute / position tensors with their in-place versions."""
        return (self._topology, self.density, self.sh, self.pos,
                (self.density._version, self.sh._version, self.pos._version))

    def set_attributes(self, density, sh):
        self._attrs(density, sh)
        _check(lib().rf_scene_set_attributes(self.handle, _ptr(self.density), _ptr(self.sh),
                                             self.attr_dtype))

    def update_positions(self, pos=None, stream=None):
        if pos is not None:
            self.pos = pos.contiguous()
        _check(lib().rf_scene_update_positions(self.handle, _ptr(self.pos), _stream(stream)))
        self._pos_version = self.pos._version

    def _sync_positions(self, pos):
        if pos is not None and (pos is not self.pos or pos._version != self._pos_version):
            self.update_positions(pos.detach())

    def render(self, cams, eps: float = 1e-4, max_steps: int = 0, steps: bool = False,
               status: bool = False, quantile: bool = False, out=None, stream=None,
               effects=None, record: int = 0) -> dict:
        """Forward render; returns rgb [R,3], trans [R], depth [R] (+ steps,
        status; + quantile [R] and quantile_aux [R,5] with ``quantile``) as
        CUDA tensors, rays of the cameras concatenated.  ``effects``: an
        analytic sphere the rays reflect off or refract through.  ``record``
        > 0: also keep a segment record of that many steps per ray
        (``out["walk_record"]``, 24 bytes per step), which lets
        :meth:`backward` rebuild the walk without the face search and the
        attribute reads."""
        ca = camera_array(cams)
        R = n_rays_of(cams)
        dev = self.pos.device
        if out is None:
            out = dict(rgb=torch.empty(R, 3, device=dev), trans=torch.empty(R, device=dev),
                       depth=torch.empty(R, device=dev))
            if steps:
                out["steps"] = torch.empty(R, dtype=torch.int32, device=dev)
            if status:
                out["status"] = torch.empty(R, dtype=torch.uint8, device=dev)
            if quantile:
                out["quantile"] = torch.empty(R, device=dev)
                out["quantile_aux"] = torch.empty(R, 5, device=dev)
            if record:
                out["walk_record"] = (torch.empty(walk_record_bytes(cams, record), dtype=torch.uint8,
                                                  device=dev), int(record))
        o = opts_struct(eps, max_steps, effects)
        rec = out.get("walk_record")
        fo = rf_fwd_outputs(_addr(out["rgb"]), _addr(out["trans"]), _addr(out["depth"]),
                            _addr(out.get("steps")), _addr(out.get("status")),
                            _addr(out.get("quantile")), _addr(out.get("quantile_aux")),
                            _addr(rec[0]) if rec is not None else None,
                            rec[0].numel() if rec is not None else 0,
                            rec[1] if rec is not None else 0)
        _check(lib().rf_render_fwd_ex(self.handle, ca, len(ca), ctypes.byref(o), ctypes.byref(fo),
                                      _stream(stream)))
        return out

    def backward(self, cams, fwd: dict, d_rgb, d_trans=None, d_depth=None, grads=None,
                 eps: float = 1e-4, max_steps: int = 0, d_quantile=None, stream=None,
                 effects=None, shared_cells: bool = False) -> dict:
        """Accumulate gradients (density, sh, pos; float32) of the forward
        outputs (and of the quantile loss, with ``d_quantile``) into ``grads``
        (zero-initialised if None).  A ``fwd`` that holds a ``walk_record``
        (a segment record) has its walk rebuilt from it instead of searched
        again.  The first backward that asks for density or position
        gradients allocates a 16-byte-per-site workspace owned by the scene.
        ``shared_cells``: the backward for frames whose rays share cells
        heavily (``RF_RENDER_SHARED_CELLS``)."""
        if grads is None:
            dev = self.pos.device
            grads = dict(density=torch.zeros(self.n_sites, device=dev),
                         sh=torch.zeros(tuple(self.sh.shape), device=dev),
                         pos=torch.zeros(self.n_sites, 3, device=dev))
        ca = camera_array(cams)
        o = opts_struct(eps, max_steps, effects, shared_cells)
        rec = fwd.get("walk_record")
        bi = rf_bwd_inputs(_addr(fwd["rgb"]), _addr(fwd["trans"]), _addr(fwd.get("depth")),
                           _addr(fwd.get("quantile_aux")), _addr(d_rgb), _addr(d_trans),
                           _addr(d_depth), _addr(d_quantile),
                           _addr(rec[0]) if rec is not None else None,
                           rec[0].numel() if rec is not None else 0,
                           rec[1] if rec is not None else 0)
        go = rf_grads(_addr(grads.get("density")), _addr(grads.get("sh")), _addr(grads.get("pos")))
        _check(lib().rf_render_bwd_ex(self.handle, ca, len(ca), ctypes.byref(o), ctypes.byref(bi),
                                      ctypes.byref(go), _stream(stream)))
        return grads

    def trace(self, cam, max_per_ray: int = 256, eps: float = 1e-4, max_steps: int = 0,
              stream=None, effects=None):
        """Visited cells per ray [R, max_per_ray] (-1 padded) and counts [R]."""
        R = int(cam.width) * int(cam.height)
        dev = self.pos.device
        cells = torch.empty(R, max_per_ray, dtype=torch.int32, device=dev)
        counts = torch.empty(R, dtype=torch.int32, device=dev)
        o = opts_struct(eps, max_steps, effects)
        ca = camera_array([cam])
        _check(lib().rf_trace_cells(self.handle, ca, ctypes.byref(o), int(max_per_ray),
                                    _ptr(cells), _ptr(counts), _stream(stream)))
        return cells, counts

    def densify_scores(self, g_pos, stream=None):
        """|dL/dp_i| * (half the mean distance to the Delaunay neighbours), [N]."""
        score = torch.empty(self.n_sites, device=self.pos.device)
        _check(lib().rf_densify_scores(self.handle, _ptr(g_pos.contiguous().float()), _ptr(score),
                                       _stream(stream)))
        return score

    def prune_mask(self, threshold: float, stream=None):
        """Sites whose density and all neighbours' densities are below ``threshold``."""
        mask = torch.empty(self.n_sites, dtype=torch.uint8, device=self.pos.device)
        _check(lib().rf_prune_mask(self.handle, float(threshold), _ptr(mask), _stream(stream)))
        return mask.bool()

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().rf_scene_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Adjacency:
    """GPU Voronoi adjacency builder (``rf_adjacency_*``): the neighbour lists
    the walk needs, from the site positions alone."""

    def __init__(self):
        h = _P()
        _check(lib().rf_adjacency_create(ctypes.byref(h)))
        self._h = h
        self.stats = None

    def build(self, pos, domain=None, incremental: bool = False, stream=None):
        """Returns (adj_off [N+1], adj_idx [E]) int32 CUDA tensors and keeps the
        build statistics in ``self.stats``; ``domain`` = (min xyz, max xyz)."""
        if self._h is None:
            raise RuntimeError("adjacency builder is closed")
        pos = pos.contiguous().float()
        n = int(pos.shape[0])
        dom = None if domain is None else (ctypes.c_float * 6)(*[float(v) for v in np.ravel(domain)])
        _check(lib().rf_adjacency_build(self._h, n, _ptr(pos), dom, int(bool(incremental)),
                                        _stream(stream)))
        st = rf_adjacency_stats()
        _check(lib().rf_adjacency_result(self._h, None, None, ctypes.byref(st)))
        self.stats = {f[0]: (list(getattr(st, f[0])) if f[0] == "domain" else getattr(st, f[0]))
                      for f in st._fields_ if f[0] != "reserved"}
        off = torch.empty(n + 1, dtype=torch.int32, device=pos.device)
        idx = torch.empty(max(int(st.n_edges), 1), dtype=torch.int32, device=pos.device)[: int(st.n_edges)]
        _check(lib().rf_adjacency_copy(self._h, _ptr(off), _ptr(idx) if st.n_edges else None,
                                       _stream(stream)))
        return off, idx

    def close(self):
        if self._h is not None:
            lib().rf_adjacency_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sample_multinomial(weights, u, stream=None):
    """Indices drawn with probability proportional to ``weights`` (device
    float [n]); ``u``: device float [m] of uniform numbers in [0, 1)."""
    w = weights.contiguous().float()
    uu = u.contiguous().float()
    n = w.numel()
    nbytes = int(lib().rf_multinomial_workspace_bytes(n))
    ws = torch.empty((nbytes + 7) // 8, dtype=torch.float64, device=w.device)
    out = torch.empty(uu.numel(), dtype=torch.int32, device=w.device)
    _check(lib().rf_sample_multinomial(_ptr(w), n, _ptr(uu), uu.numel(), _ptr(ws), nbytes,
                                       _ptr(out), _stream(stream)))
    return out


def mse_grad(rgb, target, scale: float, loss=None, stream=None):
    """d_rgb = 2 scale (rgb - target) and loss += scale * sum (rgb - target)^2
    (both on the device)."""
    d = torch.empty_like(rgb)
    if loss is None:
        loss = torch.zeros(1, device=rgb.device)
    _check(lib().rf_mse_grad(_ptr(rgb), _ptr(target), rgb.numel(), float(scale), _ptr(d),
                             _ptr(loss), _stream(stream)))
    return d, loss


def render_noalloc(pos, adj_off, adj_idx, density, sh, aabb, cams, eps: float = 1e-4,
                   max_steps: int = 0, out=None, stream=None, effects=None) -> dict:
    """``rf_render_fwd_noalloc``: forward render straight from the caller's
    arrays, with no device allocation inside the library (its only scratch is
    a fixed 64-camera array).  Same outputs as :meth:`Foam.render`."""
    ca = camera_array(cams)
    R = n_rays_of(cams)
    if out is None:
        dev = pos.device
        out = dict(rgb=torch.empty(R, 3, device=dev), trans=torch.empty(R, device=dev),
                   depth=torch.empty(R, device=dev))
    K = int(sh.shape[1])
    box = (ctypes.c_float * 6)(*[float(v) for v in list(aabb[0]) + list(aabb[1])])
    o = opts_struct(eps, max_steps, effects)
    _check(lib().rf_render_fwd_noalloc(int(pos.shape[0]), int(adj_idx.shape[0]), _ptr(pos),
                                       _ptr(adj_off), _ptr(adj_idx) if adj_idx.numel() else None,
                                       _ptr(density), _ptr(sh), int(round(K ** 0.5)) - 1,
                                       _DTYPES[density.dtype], box, ca, len(ca), ctypes.byref(o),
                                       _ptr(out["rgb"]), _ptr(out["trans"]), _ptr(out["depth"]),
                                       _stream(stream)))
    return out


class _scene_as_rendered:
    """Context manager for a backward: puts the foam back into the state its
    forward rendered (another render may have swapped the attribute tensors
    or moved the sites since, e.g. with gradient accumulation over several
    renders) and restores the newer state afterwards.  Attributes or
    positions edited in place, or replaced neighbour lists, cannot be undone:
    that raises instead of returning wrong gradients."""

    def __init__(self, foam, state):
        self.foam = foam
        self.topo, self.density, self.sh, self.pos, self.versions = state
        self.swapped = None

    def __enter__(self):
        f = self.foam
        if f._topology != self.topo:
            raise RuntimeError("the foam's adjacency was rebuilt between this render and its backward")
        if (self.density._version, self.sh._version, self.pos._version) != self.versions:
            raise RuntimeError("density, sh or positions were modified in place between this render "
                               "and its backward")
        cur = (f.density, f.sh, f.pos)
        if cur[0] is self.density and cur[1] is self.sh and cur[2] is self.pos \
                and f._pos_version == self.pos._version:
            return self
        self.swapped = cur
        if cur[0] is not self.density or cur[1] is not self.sh:
            f.set_attributes(self.density, self.sh)
        if cur[2] is not self.pos or f._pos_version != self.pos._version:
            f.update_positions(self.pos)
        return self

    def __exit__(self, *exc):
        if self.swapped is not None:
            d, s, p = self.swapped
            f = self.foam
            if f.density is not d or f.sh is not s:
                f.set_attributes(d, s)
            if f.pos is not p:
                f.update_positions(p)
        return False


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, foam, cams, eps, max_steps, quantile, effects, record, shared_cells, density, sh, pos):
        foam._sync_positions(pos)
        out = foam.render(cams, eps=eps, max_steps=max_steps, quantile=quantile, effects=effects,
                          record=record)
        ctx.walk_record = out.get("walk_record")
        ctx.foam_state = foam.state()
        ctx.foam, ctx.cams, ctx.eps, ctx.max_steps, ctx.quantile = foam, cams, eps, max_steps, quantile
        ctx.effects = effects
        ctx.shared_cells = shared_cells
        ctx.dtypes = (density.dtype, sh.dtype)
        if quantile:
            ctx.save_for_backward(out["rgb"], out["trans"], out["depth"], out["quantile_aux"])
            return out["rgb"], out["trans"], out["depth"], out["quantile"]
        ctx.save_for_backward(out["rgb"], out["trans"], out["depth"])
        return out["rgb"], out["trans"], out["depth"]

    @staticmethod
    def backward(ctx, g_rgb, g_trans, g_depth, g_quant=None):
        saved = ctx.saved_tensors
        rgb, trans, depth = saved[:3]
        foam = ctx.foam
        need = ctx.needs_input_grad
        dev = rgb.device
        grads = {}
        if need[8]:
            grads["density"] = torch.zeros(foam.n_sites, device=dev)
        if need[9]:
            grads["sh"] = torch.zeros(tuple(foam.sh.shape), device=dev)
        if need[10]:
            grads["pos"] = torch.zeros(foam.n_sites, 3, device=dev)
        if grads:
            z = lambda g: None if g is None else g.contiguous().float()
            fwd = dict(rgb=rgb, trans=trans, depth=depth)
            if ctx.quantile:
                fwd["quantile_aux"] = saved[3]
            if ctx.walk_record is not None:
                fwd["walk_record"] = ctx.walk_record
            with _scene_as_rendered(foam, ctx.foam_state):
                foam.backward(ctx.cams, fwd,
                              z(g_rgb) if g_rgb is not None else torch.zeros_like(rgb),
                              z(g_trans), z(g_depth), grads=grads, eps=ctx.eps,
                              max_steps=ctx.max_steps, d_quantile=z(g_quant) if ctx.quantile else None,
                              effects=ctx.effects, shared_cells=ctx.shared_cells)
        gd = grads.get("density")
        gs = grads.get("sh")
        ctx.walk_record = None
        return (None, None, None, None, None, None, None, None,
                None if gd is None else gd.to(ctx.dtypes[0]),
                None if gs is None else gs.to(ctx.dtypes[1]),
                grads.get("pos"))


def render(foam: Foam, cams, density=None, sh=None, pos=None, eps: float = 1e-4,
           max_steps: int = 0, quantile: bool = False, effects=None, record: int = 256,
           shared_cells: bool = False):
    """Differentiable render of ``cams``: returns (rgb [R,3], trans [R],
    depth [R]) and, with ``quantile``, the per-ray quantile loss of Eq. (6)
    [R]; gradients flow to ``density``, ``sh`` and ``pos`` (defaults: the
    foam's own tensors).  A changed ``pos`` is re-packed first.  ``record``:
    steps per ray of the segment record kept between the passes, 24 bytes per
    step for every ray slot of the cameras' 16x8 tiles (12.7 GB for a
    1920x1080 frame at 256 steps); 0: none, the backward then searches every
    step's exit again and re-reads the attributes.  ``shared_cells``: the
    backward for frames whose rays share cells heavily
    (``RF_RENDER_SHARED_CELLS``)."""
    density = foam.density if density is None else density
    sh = foam.sh if sh is None else sh
    if density is not foam.density or sh is not foam.sh:
        foam.set_attributes(density.detach(), sh.detach())
    if pos is None:
        pos = foam.pos
    return _Render.apply(foam, cams, eps, max_steps, bool(quantile), effects, int(record), bool(shared_cells),
                         density, sh, pos)
