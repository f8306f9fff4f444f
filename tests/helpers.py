"""Small scene builders shared by the tests (inputs only, no method arithmetic)."""
import dataclasses
import math

import numpy as np

from paper_2502_01157_gb300 import scenes as S


@dataclasses.dataclass
class TinyScene:
    pos: np.ndarray
    adj_off: np.ndarray
    adj_idx: np.ndarray
    density: np.ndarray
    sh: np.ndarray
    sh_degree: int
    aabb_min: np.ndarray
    aabb_max: np.ndarray


def csr_from_lists(nbrs):
    off = np.zeros(len(nbrs) + 1, np.int32)
    off[1:] = np.cumsum([len(x) for x in nbrs])
    idx = np.array([j for x in nbrs for j in sorted(x)], np.int32)
    return off, idx


def random_scene(n, deg, seed, kind="uniform", box=1.0):
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        pos = S.uniform_sites(n, -box, box, rng)
    else:
        pos = S.mixture_sites(n, rng)
    pos = S.dedupe_sites(pos, rng)
    dens = S.lognormal_density(n, rng)
    sh = S.sh_coeffs(n, deg, rng, dc="uniform_colour")
    return S.make_scene(pos, dens, sh, name=f"rand{n}")


def camera_at(eye, target, w=16, h=12, fov=60.0, t_near=0.0, t_far=0.0):
    return S.pinhole(w, h, fov, c2w=S.look_at(eye, target), t_near=t_near, t_far=t_far)
