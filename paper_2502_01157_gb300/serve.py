"""Continuous-batching render server (binding of ``rf_serve_*``).

Requests are cameras of any resolution.  :meth:`Server.submit` admits a
request if its output fits in the server's device memory budget (else it is
rejected at once); a native scheduler thread launches admitted requests in
multi-camera batches on several CUDA streams, so requests that arrive while
others are on the GPU run as soon as a stream frees up.  :meth:`Server.poll`
returns the image once it is in host memory.
"""
from __future__ import annotations

import ctypes
import threading
import time
from typing import List, Optional

import numpy as np

from . import rf

BUSY = 4
NOT_FOUND = 8
TIMEOUT = 6


class Server:
    def __init__(self, foam: "rf.Foam", mem_budget_bytes: int = 2 << 30, max_inflight: int = 256,
                 n_streams: int = 4, max_batch: int = 8, eps: float = 1e-4, max_steps: int = 0):
        L = rf.lib()
        self.foam = foam  # the server borrows the packed scene
        cfg = rf.rf_serve_config(int(mem_budget_bytes), int(max_inflight), int(n_streams),
                                 int(max_batch), float(eps), int(max_steps))
        h = ctypes.c_void_p()
        rf._check(L.rf_serve_create(foam.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def submit(self, cam) -> Optional[int]:
        """Request id, or None if the request was not admitted (busy)."""
        c = rf.camera_struct(cam)
        rid = ctypes.c_uint64()
        rc = rf.lib().rf_serve_submit(self._h, ctypes.byref(c), ctypes.byref(rid))
        if rc == BUSY:
            return None
        rf._check(rc)
        return rid.value

    def poll(self, rid: int, out: Optional[np.ndarray] = None):
        """(done, latency_ms); fills ``out`` ([H*W,3] float32) when done."""
        done = ctypes.c_int32()
        lat = ctypes.c_double()
        ptr = None if out is None else out.ctypes.data_as(ctypes.c_void_p)
        rf._check(rf.lib().rf_serve_poll(self._h, ctypes.c_uint64(rid), ptr, ctypes.byref(done),
                                         ctypes.byref(lat)))
        return bool(done.value), lat.value

    def wait(self, rid: int, timeout_ms: int = 10000, out: Optional[np.ndarray] = None) -> float:
        lat = ctypes.c_double()
        ptr = None if out is None else out.ctypes.data_as(ctypes.c_void_p)
        rf._check(rf.lib().rf_serve_wait(self._h, ctypes.c_uint64(rid), int(timeout_ms), ptr,
                                         ctypes.byref(lat)))
        return lat.value

    def stats(self) -> dict:
        m = rf.rf_serve_metrics()
        rf._check(rf.lib().rf_serve_stats(self._h, ctypes.byref(m)))
        return {f: getattr(m, f) for f, _ in m._fields_}

    def reset_stats(self):
        rf._check(rf.lib().rf_serve_reset_stats(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None:
            rf.lib().rf_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_open_loop(server: Server, cams: List, arrivals: np.ndarray, poll_interval_s: float = 2e-4,
                  deadline_s: float = 60.0) -> dict:
    """Open-loop load: request k is submitted at ``arrivals[k]`` seconds
    (rejected if not admitted, never retried); completed requests are
    collected by polling.  Returns the server's latency statistics plus the
    offered and rejected counts."""
    server.reset_stats()
    pending = []
    rejected = 0
    t0 = time.perf_counter()
    k = 0
    n = len(arrivals)
    while k < n or pending:
        now = time.perf_counter() - t0
        while k < n and arrivals[k] <= now:
            rid = server.submit(cams[k])
            if rid is None:
                rejected += 1
            else:
                pending.append(rid)
            k += 1
        still = []
        for rid in pending:
            done, _ = server.poll(rid)
            if not done:
                still.append(rid)
        pending = still
        if now > deadline_s:
            break
        nxt = arrivals[k] - (time.perf_counter() - t0) if k < n else poll_interval_s
        time.sleep(max(0.0, min(poll_interval_s, nxt)))
    st = server.stats()
    st["offered"] = n
    st["rejected_open_loop"] = rejected
    st["wall_s"] = time.perf_counter() - t0
    return st


def run_closed_loop(server: Server, cams: List, inflight: int, duration_s: float,
                    poll_interval_s: float = 1e-4) -> dict:
    """Saturation load: keeps ``inflight`` requests in the server (a new one
    is submitted as soon as one completes), cycling through ``cams``, for
    ``duration_s``; returns the server's statistics (its Mrays/s is the
    saturation throughput)."""
    server.reset_stats()
    pending = []
    k = 0
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        while now < duration_s and len(pending) < inflight:
            rid = server.submit(cams[k % len(cams)])
            if rid is None:
                break
            pending.append(rid)
            k += 1
        pending = [rid for rid in pending if not server.poll(rid)[0]]
        if now >= duration_s and not pending:
            break
        time.sleep(poll_interval_s)
    st = server.stats()
    st["submitted"] = k
    st["wall_s"] = time.perf_counter() - t0
    return st
