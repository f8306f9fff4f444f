"""Helpers for the CUDA-vs-oracle parity tests.

Tolerances:

* visited cells: bit-exact on every ray the oracle does not flag as
  near-degenerate;
* images (rgb, transmittance, depth): RMSE <= 1e-5 over all rays;
* gradients: ||g - g_ref||_2 / ||g_ref||_2 <= 1e-3 per tensor, with the loss
  restricted to non-degenerate rays.
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


def compare_traces(cells_gpu, counts_gpu, orc, max_per_ray):
    """Number of mismatching non-degenerate rays and number of degenerate rays."""
    deg = orc["degen"]
    bad = 0
    for r in range(len(deg)):
        if deg[r]:
            continue
        n = int(orc["steps"][r])
        if int(counts_gpu[r]) != n:
            bad += 1
            continue
        m = min(n, max_per_ray)
        if not np.array_equal(cells_gpu[r, :m], orc["trace_cells"][r, :m]):
            bad += 1
    return bad, int(deg.sum())


def rel_l2(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))
