"""The allocation-free forward render, called through the C ABI.

``rf_render_fwd_noalloc`` serves callers that cannot call cudaMalloc (the
device allocator belongs to another runtime, or allocating would stall a
latency-bound loop): it renders straight from the caller's arrays and keeps
its only scratch in a fixed 64-camera array inside the library.  Its output
must equal ``rf_render_fwd`` on a packed scene bit for bit (the face records
are formed with the packer's own FP32 operations), on two calls in a row (the
second call finds the previous call's keys in the shared array).

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2502_01157_gb300 import rf
from tests.helpers import camera_at, random_scene
from tests.parity import rmse

pytestmark = pytest.mark.gpu


def _inputs(sc, dt=torch.float32):
    t = lambda a, d: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", d)
    return (t(sc.pos, torch.float32), t(sc.adj_off, torch.int32), t(sc.adj_idx, torch.int32),
            t(sc.density, dt), t(sc.sh, dt))


@pytest.mark.parametrize("deg,dt", [(3, torch.float32), (0, torch.float32), (3, torch.bfloat16)])
def test_noalloc_matches_packed_render_twice(deg, dt):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    sc = random_scene(2500, deg, 300 + deg)
    pos, off, idx, dens, sh = _inputs(sc, dt)
    aabb = (sc.aabb_min, sc.aabb_max)
    # 20 cameras: more than one launch of 16, mixed sizes, inside and outside the box
    rng = np.random.default_rng(deg)
    cams = []
    for k in range(20):
        eye = rng.uniform(-0.5, 0.5, 3) if k % 3 else rng.uniform(1.5, 2.5, 3) * rng.choice([-1, 1], 3)
        cams.append(camera_at(eye, rng.uniform(-0.3, 0.3, 3), w=int(rng.integers(1, 40)),
                              h=int(rng.integers(1, 30))))
    foam = rf.Foam(pos, off, idx, dens, sh, aabb=aabb)
    ref = foam.render(cams)
    for call in range(2):
        out = rf.render_noalloc(pos, off, idx, dens, sh, aabb, cams)
        torch.cuda.synchronize()
        for k in ("rgb", "trans", "depth"):
            a = out[k].cpu().numpy()
            b = ref[k].cpu().numpy()
            assert np.array_equal(a, b), f"call {call} {k}: rmse {rmse(a, b):.3e}"
    foam.close()


def test_noalloc_rejects_more_cameras_than_its_scratch_holds():
    sc = random_scene(300, 0, 9)
    pos, off, idx, dens, sh = _inputs(sc)
    cams = [camera_at((0.0, 0.0, 0.0), (0.0, 0.0, 1.0), w=2, h=2)] * 65
    with pytest.raises(rf.RFError) as e:
        rf.render_noalloc(pos, off, idx, dens, sh, (sc.aabb_min, sc.aabb_max), cams)
    assert e.value.code == 1 and "at most 64" in str(e.value)
