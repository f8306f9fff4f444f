"""Helpers for the CUDA-vs-oracle parity tests.

Tolerances:

* visited cells: bit-exact on every ray except those the oracle flags as
  passing within tau of a Voronoi edge or vertex, or as starting within tau
  of a bisector (``tie``); a ray whose transmittance meets eps within a
  relative 1e-3 at a stop test (``stop_tie``) may end one step earlier or
  later, with the shorter cell sequence a prefix of the longer;
* images (rgb, transmittance, depth): RMSE <= 1e-5 over all rays;
* gradients: ||g - g_ref||_2 / ||g_ref||_2 <= 1e-3 per tensor, with the loss
  restricted to rays without any flag (grazing crossings and ill-conditioned
  sphere bounces carry an FP32 conditioning error in the gradient only);
* the flagged fraction of each class is bounded (``check_flag_fractions``),
  so a classifier that flags too much cannot hollow out the comparisons.
"""
import copy

import numpy as np
import torch

import oracle
from paper_2502_01157_gb300 import rf

IMG_RMSE = 1e-5
GRAD_REL = 1e-3
TORCH_DT = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


def rounded_scene(scene, dt: str):
    """The scene with density and SH rounded to the storage dtype (FP32 values)."""
    if dt == "f32":
        return scene
    s = copy.copy(scene)
    s.density = torch.from_numpy(scene.density).to(TORCH_DT[dt]).float().numpy()
    s.sh = torch.from_numpy(scene.sh).to(TORCH_DT[dt]).float().numpy()
    return s


def foam_of(scene, dt="f32"):
    return rf.Foam.from_scene(scene, attr_dtype=TORCH_DT[dt])


def gpu_render(foam, cams, eps=1e-4, max_steps=0):
    out = foam.render(cams, eps=eps, max_steps=max_steps, steps=True, status=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def rmse(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.sqrt(np.mean((a - b) ** 2))) if a.size else 0.0


def image_errors(g, o, rows=None):
    """RMSE / max-abs of rgb, trans, depth; g indexed by ``rows`` if given."""
    sel = (lambda x: x[rows]) if rows is not None else (lambda x: x)
    res = {}
    for k in ("rgb", "trans", "depth"):
        a, b = sel(g[k]), o[k]
        res[k] = (rmse(a, b), float(np.max(np.abs(a - b))) if a.size else 0.0)
    return res


def assert_images_close(g, o, rows=None, tol=IMG_RMSE):
    err = image_errors(g, o, rows)
    for k, (r, m) in err.items():
        assert r <= tol, f"{k}: rmse {r:.3e} > {tol} (max abs {m:.3e})"
    return err


# Upper bounds on the fraction of rays in each near-degenerate class; a
# bound catches a classifier that flags far too much.  An edge tie is a step
# that ends within tau = 1e-6 (scene units) of another face's boundary, about
# 4 tau / (face size) per step: ~1e-4 per step and 0.1-0.5 % of the rays in
# the small scenes (a few thousand sites), 5.5e-4 per step and ~7 % of the
# rays at 3M sites in [-1,1]^3 (faces ~7e-3 across, 128 steps per ray).
FLAG_BOUNDS = {"edge": 0.03, "camera": 0.0, "stop": 0.02, "graze": 0.06, "bend": 0.10, "any": 0.10}
FULL_SIZE_FLAG_BOUNDS = {"edge": 0.10, "any": 0.15}


def check_flag_fractions(flags, bounds=None):
    """Per-class counts of the oracle's flags; asserts each fraction is within
    its bound (``bounds`` overrides entries of FLAG_BOUNDS)."""
    b = dict(FLAG_BOUNDS, **(bounds or {}))
    c = oracle.flag_counts(flags)
    n = max(c["rays"], 1)
    for k, lim in b.items():
        assert c[k] <= lim * n, f"{c[k]} of {n} rays flagged '{k}' (bound {lim:.0%}): {c}"
    return c


def assert_steps_match(steps_gpu, orc, rows=None):
    """Cell-step counts equal on every ray that is not a tie; a stop tie may
    differ by one step."""
    g = np.asarray(steps_gpu if rows is None else steps_gpu[rows])
    keep = ~orc["tie"] & ~orc["stop_tie"]
    np.testing.assert_array_equal(g[keep], orc["steps"][keep])
    st = orc["stop_tie"] & ~orc["tie"]
    assert np.all(np.abs(g[st].astype(np.int64) - orc["steps"][st]) <= 1)


def compare_traces(cells_gpu, counts_gpu, orc, max_per_ray):
    """Number of rays whose visited cells differ from the oracle's where they
    must not, and the number of tie rays left out.  Grazing and bend rays are
    compared bit for bit like any other; a stop tie may end one step apart."""
    tie = orc["tie"]
    stop = orc["stop_tie"]
    bad = 0
    for r in range(len(tie)):
        if tie[r]:
            continue
        n = int(orc["steps"][r])
        ng = int(counts_gpu[r])
        if stop[r]:
            if abs(ng - n) > 1:
                bad += 1
                continue
            m = min(n, ng, max_per_ray)
        else:
            if ng != n:
                bad += 1
                continue
            m = min(n, max_per_ray)
        if not np.array_equal(cells_gpu[r, :m], orc["trace_cells"][r, :m]):
            bad += 1
    return bad, int(tie.sum())


def assert_same_sums(a, b, tag=""):
    """Two GPU gradients that differ only in the order of their float atomics:
    relative L2 within 2e-6, and each element within 1e-5 of the tensor's
    largest magnitude (a sum with cancellation can differ by more than 1e-5
    of its own value, so no element-wise relative bound is used)."""
    a = np.asarray(a.detach().cpu() if hasattr(a, "detach") else a, np.float64)
    b = np.asarray(b.detach().cpu() if hasattr(b, "detach") else b, np.float64)
    e = rel_l2(a, b)
    assert e <= 2e-6, (tag, e)
    scale = float(np.max(np.abs(b))) if b.size else 0.0
    assert np.all(np.abs(a - b) <= 1e-5 * scale + 1e-12), (tag, float(np.max(np.abs(a - b))), scale)


def rel_l2(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))
