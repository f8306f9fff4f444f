"""Full-size parity: the workloads' own scenes and cameras, rendered in the
launch configuration the benchmark times, compared with the FP64 oracle on
sampled pixels (which the oracle computes one by one) and on bit-identical
window cameras for the visited-cell sequences."""
import numpy as np
import pytest
import torch

import oracle
from paper_2502_01157_gb300 import rf
from paper_2502_01157_gb300 import scenes as S
from tests.helpers import random_scene
from tests.parity import (FULL_SIZE_FLAG_BOUNDS, GRAD_REL, assert_images_close, assert_steps_match,
                          check_flag_fractions, compare_traces, foam_of, gpu_render, rel_l2, rounded_scene)

pytestmark = pytest.mark.gpu
N_SAMPLE = 1500
RECORD = 384   # walk-record steps of the timed training step


def window(cam, x0, y0, w, h):
    """Camera covering pixels [x0,x0+w) x [y0,y0+h) of ``cam``; its rays are
    bit-identical to the full camera's (cx - x0 and cy - y0 are exact)."""
    return S.Camera(cam.c2w, cam.fx, cam.fy, cam.cx - x0, cam.cy - y0, w, h, cam.t_near, cam.t_far)


def _check_forward_sampled(scene, foam, cams, dt="f32", seed=0):
    g = gpu_render(foam, cams)
    ref = rounded_scene(scene, dt)
    rng = np.random.default_rng(seed)
    base = 0
    flags = []
    for cam in cams:
        px = np.sort(rng.choice(cam.n_rays, size=min(N_SAMPLE, cam.n_rays), replace=False))
        o = oracle.render(ref, cam, pixels=px)
        rows = base + px
        err = assert_images_close(g, o, rows)
        assert_steps_match(g["steps"], o, rows)
        flags.append(o["flags"])
        base += cam.n_rays
    return g, err, check_flag_fractions(np.concatenate(flags), FULL_SIZE_FLAG_BOUNDS)


def _check_traces(scene, foam, cam, dt="f32"):
    ref = rounded_scene(scene, dt)
    bad_total = 0
    flags = []
    for (x0, y0) in [(0, 0), (cam.width // 2 - 16, cam.height // 2 - 8), (cam.width - 32, cam.height - 16)]:
        win = window(cam, max(0, x0), max(0, y0), 32, 16)
        cells, counts = foam.trace(win, max_per_ray=1024)
        o = oracle.render(ref, win, trace=1024)
        bad, _ = compare_traces(cells.cpu().numpy(), counts.cpu().numpy(), o, 1024)
        bad_total += bad
        flags.append(o["flags"])
    return bad_total, check_flag_fractions(np.concatenate(flags), FULL_SIZE_FLAG_BOUNDS)


def _check_backward_sampled(scene, foam, cams, dt="f32", seed=1, record=0, shared_cells=False):
    """Full launch; the loss weights only sampled, unflagged rays, so the
    oracle can compute the reference gradient.  ``record`` > 0: the backward
    replays the forward's walk record, as the timed training step does."""
    ref = rounded_scene(scene, dt)
    fwd = foam.render(cams, record=record)
    R = rf.n_rays_of(cams)
    rng = np.random.default_rng(seed)
    gr = np.zeros((R, 3), np.float32)
    ref_g = dict(density=np.zeros(scene.n_sites), sh=np.zeros(scene.sh.shape),
                 pos=np.zeros((scene.n_sites, 3)))
    base = 0
    for cam in cams:
        px = np.sort(rng.choice(cam.n_rays, size=min(N_SAMPLE // len(cams) + 64, cam.n_rays), replace=False))
        o = oracle.render(ref, cam, pixels=px)
        px = px[~o["degen"]]
        w = rng.normal(size=(len(px), 3)).astype(np.float32)
        gr[base + px] = w
        G = oracle.render_bwd(ref, cam, w, pixels=px)
        for k in ref_g:
            ref_g[k] += G[k]
        base += cam.n_rays
    G = foam.backward(cams, fwd, torch.from_numpy(gr).cuda(), shared_cells=shared_cells)
    torch.cuda.synchronize()
    return {k: rel_l2(G[k].cpu().numpy(), ref_g[k]) for k in ref_g}


@pytest.fixture(scope="module")
def c2():
    return S.config_scene("c2")


@pytest.fixture(scope="module")
def c3():
    return S.config_scene("c3")


@pytest.fixture(scope="module")
def c4():
    return S.config_scene("c4")


def test_c2_full_forward_backward(c2):
    cams = S.config_cameras("c2")
    foam = foam_of(c2)
    g, err, nd = _check_forward_sampled(c2, foam, cams)
    bad, ndeg = _check_traces(c2, foam, cams[0])
    print(f"c2: image err {err}, flags (sampled) {nd}, traces {bad} bad, flags (windows) {ndeg}")
    assert bad == 0
    errs = _check_backward_sampled(c2, foam, cams, record=RECORD)
    print("c2 grads (replayed record)", errs)
    for k, e in errs.items():
        assert e <= GRAD_REL, f"{k}: {e:.2e}"


@pytest.mark.parametrize("dt", ["f32", "bf16", "f16"])
def test_c3_full_forward_backward(c3, dt):
    cams = S.config_cameras("c3")
    foam = foam_of(c3, dt)
    g, err, nd = _check_forward_sampled(c3, foam, cams, dt)
    bad, ndeg = _check_traces(c3, foam, cams[0], dt)
    print(f"c3 {dt}: image err {err}, flags (sampled) {nd}, traces {bad} bad, flags (windows) {ndeg}")
    assert bad == 0
    errs = _check_backward_sampled(c3, foam, cams, dt, record=RECORD)
    print(f"c3 {dt} grads (replayed record)", errs)
    for k, e in errs.items():
        assert e <= GRAD_REL, f"{k}: {e:.2e}"
    if dt != "f32":
        # storage error against the FP32 attributes, reported
        px = np.arange(0, cams[0].n_rays, cams[0].n_rays // 500)
        o32 = oracle.render(c3, cams[0], pixels=px)
        print(f"c3 {dt} storage rmse rgb", float(np.sqrt(np.mean((g["rgb"][px] - o32["rgb"]) ** 2))))


def test_c4_eight_mixed_cameras_one_launch(c4):
    cams = S.config_cameras("c4")
    assert len(cams) == 8 and rf.n_rays_of(cams) == 9_484_800
    foam = foam_of(c4)
    g, err, nd = _check_forward_sampled(c4, foam, cams)
    print(f"c4: image err {err}, flags {nd}")
    errs = _check_backward_sampled(c4, foam, cams, record=RECORD)
    print("c4 grads", errs)
    for k, e in errs.items():
        assert e <= GRAD_REL, f"{k}: {e:.2e}"


def test_c4_gradients_against_finite_differences_512_sites():
    """The C4 recipe on a 512-site copy with 32x24 views: GPU gradients vs
    central finite differences of the FP64 oracle."""
    rng = np.random.default_rng(1004)
    pos = S.dedupe_sites(S.mixture_sites(512, rng), rng)
    sc = S.make_scene(pos, S.lognormal_density(512, rng) * np.float32(0.3),
                      S.sh_coeffs(512, 3, rng))
    cams = [S.pinhole(32, 24, 60.0, c2w=p) for p in S.sphere_poses(8, 12.0, 1004)]
    foam = foam_of(sc)
    fwd = foam.render(cams)
    R = rf.n_rays_of(cams)
    o_all = [oracle.render(sc, c, eps=1e-4) for c in cams]
    degen = np.concatenate([o["degen"] for o in o_all])
    w = rng.normal(size=(R, 3)).astype(np.float32)
    w[degen] = 0
    G = foam.backward(cams, fwd, torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    G = {k: v.cpu().numpy() for k, v in G.items()}

    sc64 = S.Scene(sc.pos.astype(np.float64), sc.adj_off, sc.adj_idx, sc.density.astype(np.float64),
                   sc.sh.astype(np.float64), 3, sc.aabb_min, sc.aabb_max)

    def loss():
        tot = 0.0
        base = 0
        for c in cams:
            o = oracle.render(sc64, c, tau=0.0)
            tot += float(np.sum(w[base:base + c.n_rays] * o["rgb"]))
            base += c.n_rays
        return tot

    def fd(arr, idx, h):
        old = arr[idx]
        arr[idx] = old + h
        lp = loss()
        arr[idx] = old - h
        lm = loss()
        arr[idx] = old
        return (lp - lm) / (2 * h)

    touched = np.nonzero(np.abs(G["density"]) > 1e-6)[0]
    pick = touched[np.argsort(-np.abs(G["density"][touched]))[:6]]
    assert len(pick) >= 3
    num = []
    ana = []
    for i in pick:
        num.append(fd(sc64.density, i, 1e-6)); ana.append(G["density"][i])
        num.append(fd(sc64.sh, (i, 0, 1), 1e-6)); ana.append(G["sh"][i, 0, 1])
        num.append(fd(sc64.sh, (i, 5, 2), 1e-6)); ana.append(G["sh"][i, 5, 2])
        for a in range(3):
            num.append(fd(sc64.pos, (i, a), 1e-6)); ana.append(G["pos"][i, a])
    e = rel_l2(np.array(ana), np.array(num))
    print("c4 512-site FD rel err", e)
    assert e <= GRAD_REL
