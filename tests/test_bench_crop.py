"""bench.py --crop renders the centre window of the workload's frame for
profiler captures: every ray of the window must be the full frame's ray
through the same pixel (checked with the oracle's camera model, FP64)."""
import numpy as np

import bench
import oracle
from paper_2502_01157_gb300 import scenes as S


def test_crop_rays_are_the_full_frames_rays():
    full = S.config_cameras("c3")[0]
    crop = bench.crop_camera(full, "640x360")
    assert (crop.width, crop.height) == (640, 360)
    x0, y0 = (full.width - crop.width) // 2, (full.height - crop.height) // 2
    rng = np.random.default_rng(1)
    us = np.concatenate([[0, crop.width - 1, 0, crop.width - 1], rng.integers(0, crop.width, 60)])
    vs = np.concatenate([[0, 0, crop.height - 1, crop.height - 1], rng.integers(0, crop.height, 60)])
    o_c, d_c = oracle.camera_rays(crop, vs * crop.width + us)
    o_f, d_f = oracle.camera_rays(full, (vs + y0) * full.width + (us + x0))
    assert np.array_equal(o_c, o_f) and np.array_equal(d_c, d_f)


def test_crop_is_clamped_to_the_frame():
    full = S.config_cameras("c1")[0]
    crop = bench.crop_camera(full, "1000x1000")
    assert (crop.width, crop.height, crop.cx, crop.cy) == (full.width, full.height, full.cx, full.cy)
