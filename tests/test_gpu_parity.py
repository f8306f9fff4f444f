"""CUDA path (through the C ABI) against the FP64 oracle, element by element,
on seeded inputs small enough for the oracle to finish in seconds."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2502_01157_gb300 import rf
from paper_2502_01157_gb300 import scenes as S
from tests.helpers import TinyScene, camera_at, csr_from_lists, random_scene
from tests.parity import (assert_same_sums, GRAD_REL, IMG_RMSE, assert_images_close, assert_steps_match,
                          check_flag_fractions, compare_traces, foam_of, gpu_render, rel_l2,
                          rounded_scene)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    rf.lib()


@pytest.fixture(scope="module")
def c1():
    return S.config_scene("c1")


def test_c1_forward_matches_oracle(c1):
    cam = S.config_cameras("c1")[0]
    foam = foam_of(c1)
    g = gpu_render(foam, [cam])
    o = oracle.render(c1, cam, trace=256)
    err = assert_images_close(g, o)
    assert np.all(g["status"] == 0)
    assert_steps_match(g["steps"], o)
    cnt = check_flag_fractions(o["flags"])
    cells, counts = foam.trace(cam, max_per_ray=256)
    bad, ntie = compare_traces(cells.cpu().numpy(), counts.cpu().numpy(), o, 256)
    print(f"c1: errors {err}, near-degenerate classes {cnt}")
    assert bad == 0
    # grazing rays are in the bit-exact cell comparison: show that they are
    graze = (o["flags"] & oracle.FLAG_GRAZE) != 0
    assert np.any(graze & ~o["tie"])


@pytest.mark.parametrize("dt", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_ragged_multicamera_all_dtypes_and_degrees(dt, deg):
    sc = random_scene(3000, deg, 100 + deg)
    rng = np.random.default_rng(7)
    if deg:
        sc.sh[:, 1:, :] = rng.normal(0, 0.3, sc.sh[:, 1:, :].shape).astype(np.float32)
    cams = [camera_at((0.1, -0.05, 0.02), (0.3, 1.0, 0.2), w=67, h=45),   # ragged tiles
            camera_at((2.2, 1.9, -1.4), (0.0, 0.0, 0.0), w=33, h=17),     # outside the box
            camera_at((-0.4, 0.3, 0.5), (0.0, 0.0, -1.0), w=1, h=1),      # a single ray
            camera_at((3.0, 0.0, 0.0), (6.0, 0.0, 0.0), w=16, h=8)]       # every ray misses
    foam = foam_of(sc, dt)
    g = gpu_render(foam, cams)
    ref = rounded_scene(sc, dt)
    base = 0
    for cam in cams:
        o = oracle.render(ref, cam)
        rows = np.arange(base, base + cam.n_rays)
        assert_images_close(g, o, rows)
        assert_steps_match(g["steps"], o, rows)
        check_flag_fractions(o["flags"])
        base += cam.n_rays
    # the last camera looks away from the box
    miss = slice(base - cams[-1].n_rays, base)
    assert np.all(g["rgb"][miss] == 0) and np.all(g["trans"][miss] == 1)
    assert np.all(g["steps"][miss] == 0)


def test_storage_precision_error_is_reported():
    """BF16/FP16 storage: compute error vs the oracle on the rounded values is
    within the FP32 bound; the storage error vs the FP32 originals is larger
    and reported."""
    sc = random_scene(3000, 3, 5)
    rng = np.random.default_rng(8)
    sc.sh[:, 1:, :] = rng.normal(0, 0.3, sc.sh[:, 1:, :].shape).astype(np.float32)
    cam = camera_at((0.0, 0.0, 0.0), (0.0, 0.0, 1.0), w=48, h=32)
    o32 = oracle.render(sc, cam)
    for dt in ("bf16", "f16"):
        g = gpu_render(foam_of(sc, dt), [cam])
        orr = oracle.render(rounded_scene(sc, dt), cam)
        comp = assert_images_close(g, orr)
        stor = {k: float(np.sqrt(np.mean((g[k] - o32[k]) ** 2))) for k in ("rgb", "trans", "depth")}
        print(f"{dt}: compute rmse {comp}, storage rmse {stor}")
        assert stor["rgb"] > comp["rgb"][0]


def _bwd_compare(sc, cams, dt="f32", seed=0, eps=1e-4, record=0, shared_cells=False):
    """GPU gradients of a random linear loss vs the oracle's; ``record`` > 0:
    the backward replays the forward's walk record of that many steps per
    ray (and searches past it), as a training step does; ``shared_cells``:
    the backward that sums crossing terms over lanes sharing a cell."""
    foam = foam_of(sc, dt)
    ref = rounded_scene(sc, dt)
    fwd = foam.render(cams, eps=eps, record=record)
    R = rf.n_rays_of(cams)
    rng = np.random.default_rng(seed)
    gr = rng.normal(size=(R, 3)).astype(np.float32)
    gt = rng.normal(size=R).astype(np.float32)
    gd = rng.normal(size=R).astype(np.float32)
    # restrict the loss to rays the oracle does not flag
    base = 0
    orc = []
    for cam in cams:
        o = oracle.render(ref, cam, eps=eps)
        check_flag_fractions(o["flags"])
        sl = slice(base, base + cam.n_rays)
        gr[sl][o["degen"]] = 0
        gt[sl][o["degen"]] = 0
        gd[sl][o["degen"]] = 0
        orc.append(o)
        base += cam.n_rays
    t = lambda a: torch.from_numpy(a).cuda()
    G = foam.backward(cams, fwd, t(gr), t(gt), t(gd), eps=eps, shared_cells=shared_cells)
    torch.cuda.synchronize()
    ref_g = dict(density=np.zeros(sc.n_sites), sh=np.zeros(sc.sh.shape), pos=np.zeros((sc.n_sites, 3)))
    base = 0
    for cam in cams:
        sl = slice(base, base + cam.n_rays)
        Go = oracle.render_bwd(ref, cam, gr[sl], gt[sl], gd[sl], eps=eps)
        for k in ref_g:
            ref_g[k] += Go[k]
        base += cam.n_rays
    errs = {k: rel_l2(G[k].cpu().numpy(), ref_g[k]) for k in ref_g}
    return errs


@pytest.mark.parametrize("dt,record", [("f32", 0), ("bf16", 0), ("f32", 384), ("bf16", 384),
                                       ("f16", 384), ("f32", 5)])
def test_backward_matches_oracle(dt, record):
    # record 384: the replayed backward a training step times; record 5: most
    # rays outgrow the record and search again past it
    sc = random_scene(3000, 3, 11)
    rng = np.random.default_rng(12)
    sc.sh[:, 1:, :] = rng.normal(0, 0.3, sc.sh[:, 1:, :].shape).astype(np.float32)
    cams = [camera_at((0.05, 0.1, -0.02), (0.2, -0.3, 1.0), w=40, h=27),
            camera_at((2.5, -1.0, 1.2), (0.0, 0.0, 0.0), w=21, h=19)]
    errs = _bwd_compare(sc, cams, dt, record=record)
    print(dt, record, errs)
    for k, e in errs.items():
        assert e <= GRAD_REL, f"{k}: rel err {e:.2e}"


@pytest.mark.parametrize("record", [0, 256])
def test_backward_with_early_stop(record):
    sc = random_scene(2500, 0, 13)
    sc.density[:] *= 40.0   # T drops below eps inside the foam
    cams = [camera_at((0.0, 0.0, 0.0), (1.0, 0.2, 0.1), w=32, h=24)]
    o = oracle.render(sc, cams[0])
    assert np.mean(o["trans"] <= 1e-4) > 0.5
    errs = _bwd_compare(sc, cams, record=record)
    for k, e in errs.items():
        assert e <= GRAD_REL, f"{k}: rel err {e:.2e}"


def test_autograd_matches_direct_backward():
    sc = random_scene(1500, 2, 21)
    foam = foam_of(sc)
    cam = camera_at((0.1, 0.1, 0.1), (0.0, 1.0, 0.0), w=24, h=16)
    dens = foam.density.clone().requires_grad_(True)
    sh = foam.sh.clone().requires_grad_(True)
    pos = foam.pos.clone().requires_grad_(True)
    rgb, tr, dp = rf.render(foam, [cam], dens, sh, pos)
    (rgb.sum() + 0.5 * tr.sum() + 0.1 * dp.sum()).backward()
    fwd = foam.render([cam])
    ones = torch.ones_like(fwd["rgb"])
    G = foam.backward([cam], fwd, ones, torch.full_like(fwd["trans"], 0.5),
                      torch.full_like(fwd["depth"], 0.1))
    assert_same_sums(dens.grad, G["density"], "density")
    assert_same_sums(sh.grad, G["sh"], "sh")
    assert_same_sums(pos.grad, G["pos"], "pos")


def test_autograd_default_record_matches_oracle():
    """rf.render's default (a 256-step walk record replayed by the backward)
    against the oracle's gradient of the same loss."""
    sc = random_scene(2000, 3, 25)
    rng = np.random.default_rng(26)
    sc.sh[:, 1:, :] = rng.normal(0, 0.3, sc.sh[:, 1:, :].shape).astype(np.float32)
    foam = foam_of(sc)
    cam = camera_at((0.1, -0.05, 0.0), (0.4, 1.0, 0.3), w=36, h=28)
    o = oracle.render(sc, cam)
    check_flag_fractions(o["flags"])
    w_rgb = rng.normal(size=(cam.n_rays, 3)).astype(np.float32)
    w_t = rng.normal(size=cam.n_rays).astype(np.float32)
    w_rgb[o["degen"]] = 0
    w_t[o["degen"]] = 0
    dens = foam.density.clone().requires_grad_(True)
    sh = foam.sh.clone().requires_grad_(True)
    pos = foam.pos.clone().requires_grad_(True)
    rgb, tr, dp = rf.render(foam, [cam], dens, sh, pos)
    ((rgb * torch.from_numpy(w_rgb).cuda()).sum() + (tr * torch.from_numpy(w_t).cuda()).sum()).backward()
    Go = oracle.render_bwd(sc, cam, w_rgb, w_t)
    for k, g in (("density", dens.grad), ("sh", sh.grad), ("pos", pos.grad)):
        e = rel_l2(g.cpu().numpy(), Go[k])
        print(f"autograd record 256 {k}: rel {e:.1e}")
        assert e <= GRAD_REL, k


def test_backward_uses_the_scene_its_forward_rendered():
    """Two renders with different density and positions (gradient
    accumulation), then the two backwards: each gets the gradients of its own
    render, as if it had run right after it; editing an attribute in place
    before the backward raises instead of returning wrong gradients."""
    sc = random_scene(1500, 2, 27)
    foam = foam_of(sc)
    cam = camera_at((0.1, 0.1, 0.1), (0.0, 1.0, 0.0), w=24, h=16)
    base_d = foam.density.clone()
    base_p = foam.pos.clone()
    gen = torch.Generator(device="cuda").manual_seed(5)
    cases = [(base_d, base_p),
             (base_d * 1.7, base_p + 2e-3 * torch.randn(base_p.shape, device="cuda", generator=gen))]

    def run(d0, p0):
        d = d0.clone().requires_grad_(True)
        p = p0.clone().requires_grad_(True)
        rgb, tr, dp = rf.render(foam, [cam], d, None, p)
        return d, p, rgb.sum() + 0.5 * tr.sum() + 0.1 * dp.sum()

    alone = []
    for d0, p0 in cases:
        d, p, L = run(d0, p0)
        L.backward()
        alone.append((d.grad.clone(), p.grad.clone()))
    a = run(*cases[0])
    b = run(*cases[1])
    a[2].backward()   # the foam holds the second render's scene now
    b[2].backward()
    for (d, p, _), (gd, gp) in zip((a, b), alone):
        assert rel_l2(d.grad.cpu().numpy(), gd.cpu().numpy()) <= 2e-6
        assert rel_l2(p.grad.cpu().numpy(), gp.cpu().numpy()) <= 2e-6
    assert torch.equal(foam.pos, b[1].detach())      # the newer scene is back in place
    d, p, L = run(*cases[0])
    with torch.no_grad():
        d.mul_(2.0)
    with pytest.raises(RuntimeError, match="modified in place"):
        L.backward()


def test_partial_gradient_requests_and_accumulation():
    # positions and densities are summed in a per-site workspace that each
    # backward zeroes and then adds into the caller's tensors: a request for
    # one of them, or a second call into the same tensors, must see exactly
    # that call's sums
    sc = random_scene(1800, 3, 23)
    foam = foam_of(sc)
    cam = camera_at((0.05, -0.1, 0.0), (0.3, 1.0, 0.2), w=29, h=21)
    fwd = foam.render([cam])
    gr = torch.randn_like(fwd["rgb"])
    gt = torch.full_like(fwd["trans"], 0.3)
    bytes0 = foam.info()["device_bytes"]
    full = foam.backward([cam], fwd, gr, gt)
    torch.cuda.synchronize()
    assert foam.info()["device_bytes"] - bytes0 == 16 * sc.n_sites
    for k in ("density", "sh", "pos"):
        one = {k: torch.zeros_like(full[k])}
        foam.backward([cam], fwd, gr, gt, grads=one)
        assert rel_l2(one[k].cpu().numpy(), full[k].cpu().numpy()) <= 2e-6, k
    twice = {k: v.clone() for k, v in full.items()}
    foam.backward([cam], fwd, gr, gt, grads=twice)
    for k in full:
        assert rel_l2(twice[k].cpu().numpy(), 2 * full[k].cpu().numpy()) <= 2e-6, k


def test_moved_positions_are_repacked():
    sc = random_scene(1200, 0, 31)
    foam = foam_of(sc)
    cam = camera_at((0.0, 0.0, 0.0), (0.0, 0.0, 1.0), w=20, h=20)
    moved = sc.pos + np.float32(1e-3) * np.random.default_rng(1).normal(size=sc.pos.shape).astype(np.float32)
    foam.update_positions(torch.from_numpy(moved).cuda())
    g = gpu_render(foam, [cam])
    sc2 = TinyScene(moved, sc.adj_off, sc.adj_idx, sc.density, sc.sh, 0, sc.aabb_min, sc.aabb_max)
    o = oracle.render(sc2, cam)
    assert_images_close(g, o)


def test_deterministic_forward():
    sc = random_scene(2000, 3, 41)
    foam = foam_of(sc)
    cam = camera_at((0.0, 0.1, 0.0), (1.0, 0.0, 0.0), w=50, h=30)
    a = gpu_render(foam, [cam])
    b = gpu_render(foam, [cam])
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])


def test_single_site_scene_and_eps_zero():
    box = (np.full(3, -1, np.float32), np.full(3, 1, np.float32))
    sc = TinyScene(np.zeros((1, 3), np.float32), np.array([0, 0], np.int32), np.zeros(0, np.int32),
                   np.array([0.7], np.float32), np.zeros((1, 1, 3), np.float32), 0, box[0], box[1])
    cam = camera_at((-3.0, 0.2, 0.1), (0.0, 0.0, 0.0), w=9, h=9, fov=30.0)
    foam = rf.Foam(torch.zeros(1, 3, device="cuda"), torch.tensor([0, 0], dtype=torch.int32, device="cuda"),
                   torch.zeros(0, dtype=torch.int32, device="cuda"),
                   torch.tensor([0.7], device="cuda"), torch.zeros(1, 1, 3, device="cuda"),
                   aabb=box)
    g = gpu_render(foam, [cam], eps=0.0)
    o = oracle.render(sc, cam, eps=0.0)
    assert_images_close(g, o)


def test_step_cap_sets_ray_status():
    sc = random_scene(2000, 0, 51)
    foam = foam_of(sc)
    cam = camera_at((0.0, 0.0, 0.0), (1.0, 0.0, 0.0), w=8, h=8)
    g = gpu_render(foam, [cam], max_steps=3)
    o = oracle.render(sc, cam, max_steps=3)
    assert np.all(g["steps"] <= 3)
    np.testing.assert_array_equal(g["status"], o["status"])
    assert_images_close(g, o)


def test_invalid_inputs_are_rejected():
    sc = random_scene(500, 0, 61)
    foam = foam_of(sc)
    bad = camera_at((0.0, 0.0, 0.0), (1.0, 0.0, 0.0), w=4, h=4)
    bad.c2w[0, 3] = np.nan
    with pytest.raises(rf.RFError) as e:
        foam.render([bad])
    assert e.value.code == 1
    # no camera, or a camera without pixels: rejected before anything runs
    for cams in ([], [camera_at((0.0, 0.0, 0.0), (1.0, 0.0, 0.0), w=0, h=4)],
                 [camera_at((0.0, 0.0, 0.0), (1.0, 0.0, 0.0), w=4, h=0)]):
        with pytest.raises(rf.RFError) as e:
            foam.render(cams)
        assert e.value.code == 1
    # asymmetric adjacency
    off, idx = csr_from_lists([[1], [], [0]])
    with pytest.raises(rf.RFError) as e:
        rf.Foam(torch.rand(3, 3, device="cuda"), torch.from_numpy(off).cuda(),
                torch.from_numpy(idx).cuda(), torch.rand(3, device="cuda"),
                torch.rand(3, 1, 3, device="cuda"))
    assert e.value.code == 7
