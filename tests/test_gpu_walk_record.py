"""Walk record: the forward stores each step's segment (exit neighbour, exit
parameter, density, colour before the clamp) so that the backward rebuilds
the walk instead of reading the faces and attributes again.  The forward
outputs must not change, and the gradients must equal those of the
searching backward (the same exits, the same arithmetic; only the order of
the floating-point atomics may differ)."""
import numpy as np
import pytest
import torch

from paper_2502_01157_gb300 import rf
from paper_2502_01157_gb300 import scenes as S
from tests.helpers import camera_at, random_scene
from tests.parity import foam_of, rel_l2

pytestmark = pytest.mark.gpu
SAME = 2e-6   # float atomics summed in another order


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    rf.lib()


def _cams():
    return [camera_at((0.05, 0.1, -0.02), (0.2, -0.3, 1.0), w=67, h=45),
            camera_at((2.5, -1.0, 1.2), (0.0, 0.0, 0.0), w=33, h=17),
            camera_at((-0.3, 0.2, 0.1), (1.0, 0.0, 0.2), w=1, h=1)]


def _grads(foam, cams, out, gr, **kw):
    G = foam.backward(cams, out, gr, torch.ones_like(out["trans"]) * 0.3, torch.ones_like(out["depth"]) * 0.1, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in G.items()}


@pytest.mark.parametrize("dt,deg,steps", [("f32", 3, 512), ("bf16", 2, 512), ("f32", 1, 3), ("f16", 0, 17)])
def test_replayed_backward_equals_searching_backward(dt, deg, steps):
    sc = random_scene(3000, deg, 40 + deg)
    foam = foam_of(sc, dt)
    cams = _cams()
    plain = foam.render(cams)
    rec = foam.render(cams, record=steps)
    torch.cuda.synchronize()
    for k in ("rgb", "trans", "depth"):
        assert torch.equal(plain[k], rec[k]), k
    gr = torch.randn_like(plain["rgb"])
    a = _grads(foam, cams, plain, gr)
    b = _grads(foam, cams, rec, gr)
    for k in a:
        e = rel_l2(b[k], a[k])
        print(f"{dt} deg {deg} record {steps}: {k} rel {e:.1e}")
        assert e <= SAME, k


def test_record_with_quantile_and_effects():
    sc = random_scene(2500, 3, 51)
    foam = foam_of(sc)
    cams = [S.fisheye(31, 23, 200.0, c2w=S.look_at((-0.85, 0.3, 0.2), (0.1, 0.0, 0.05))),
            S.Camera(**{**camera_at((0.1, 0.8, -0.6), (0.1, 0.0, 0.05), w=18, h=14).__dict__,
                        "shutter": (0.1, 0.0, 0.2)})]
    sph = S.Sphere((0.1, 0.0, 0.05), 0.35, ior=1.5, max_bounces=4)
    plain = foam.render(cams, quantile=True, effects=sph)
    rec = foam.render(cams, quantile=True, effects=sph, record=64)
    torch.cuda.synchronize()
    for k in ("rgb", "trans", "depth", "quantile"):
        assert torch.equal(plain[k], rec[k]), k
    gr = torch.randn_like(plain["rgb"])
    gq = torch.randn_like(plain["quantile"])
    a = _grads(foam, cams, plain, gr, d_quantile=gq, effects=sph)
    b = _grads(foam, cams, rec, gr, d_quantile=gq, effects=sph)
    for k in a:
        assert rel_l2(b[k], a[k]) <= SAME, k


def test_record_over_several_launches():
    # more than 16 cameras: several launches, each with its own part of the record
    sc = random_scene(2000, 1, 52)
    foam = foam_of(sc)
    cams = [camera_at((0.1 * k, 0.05, -0.1), (1.0, 0.2 * k, 0.3), w=9 + k, h=7 + (k % 3)) for k in range(19)]
    plain = foam.render(cams)
    rec = foam.render(cams, record=40)
    gr = torch.randn_like(plain["rgb"])
    a = _grads(foam, cams, plain, gr)
    b = _grads(foam, cams, rec, gr)
    for k in a:
        assert rel_l2(b[k], a[k]) <= SAME, k


def test_autograd_uses_the_record():
    sc = random_scene(1500, 2, 53)
    foam = foam_of(sc)
    cam = camera_at((0.1, 0.1, 0.1), (0.0, 1.0, 0.0), w=24, h=16)
    res = []
    for record in (0, 256):
        dens = foam.density.clone().requires_grad_(True)
        pos = foam.pos.clone().requires_grad_(True)
        rgb, tr, dp = rf.render(foam, [cam], dens, None, pos, record=record)
        (rgb.sum() + tr.sum()).backward()
        res.append((dens.grad.cpu().numpy(), pos.grad.cpu().numpy()))
    assert rel_l2(res[1][0], res[0][0]) <= SAME and rel_l2(res[1][1], res[0][1]) <= SAME


def test_short_record_buffer_is_rejected():
    sc = random_scene(800, 0, 54)
    foam = foam_of(sc)
    cam = camera_at((0.0, 0.0, 0.0), (1.0, 0.0, 0.0), w=20, h=10)
    out = foam.render([cam], record=8)
    buf, steps = out["walk_record"]
    out["walk_record"] = (buf[: buf.numel() // 2], steps)
    with pytest.raises(rf.RFError, match="walk_record"):
        foam.render([cam], out=out)


def test_unaligned_record_buffer_is_rejected():
    sc = random_scene(800, 0, 54)
    foam = foam_of(sc)
    cam = camera_at((0.0, 0.0, 0.0), (1.0, 0.0, 0.0), w=20, h=10)
    out = foam.render([cam], record=8)
    buf, steps = out["walk_record"]
    out["walk_record"] = (buf[4:], steps)   # 4 bytes past a 16-byte boundary
    with pytest.raises(rf.RFError, match="aligned"):
        foam.render([cam], out=out)


def test_record_of_another_scene_stays_in_bounds():
    """A record made on a larger scene holds exit ids beyond the smaller
    scene's sites: the backward ends those walks instead of following them
    (the gradients are not meaningful, but every access stays in bounds and
    the call succeeds)."""
    big = foam_of(random_scene(3000, 1, 61))
    small = foam_of(random_scene(500, 1, 62))
    cam = camera_at((0.05, 0.1, -0.02), (0.2, -0.3, 1.0), w=40, h=24)
    out = big.render([cam], record=64)
    ids = out["walk_record"][0].view(torch.int32).view(-1, 6, 32)[:, 0, :]
    assert int(ids.max()) >= 500   # the record does name sites the small scene lacks
    gr = torch.randn_like(out["rgb"])
    G = small.backward([cam], out, gr)
    torch.cuda.synchronize()   # the launch completed without a fault
    assert G["density"].shape == (500,) and G["pos"].shape == (500, 3)


def test_full_size_c3_replay():
    sc = S.config_scene("c3")
    cam = S.config_cameras("c3")[0]
    foam = foam_of(sc)
    plain = foam.render([cam])
    rec = foam.render([cam], record=384)
    gr = torch.randn_like(plain["rgb"]) * 1e-3
    a = _grads(foam, [cam], plain, gr)
    b = _grads(foam, [cam], rec, gr)
    for k in a:
        e = rel_l2(b[k], a[k])
        print(f"c3 record: {k} rel {e:.1e}")
        assert e <= SAME, k
