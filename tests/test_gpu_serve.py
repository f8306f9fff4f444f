"""Continuous-batching server: admission by memory, overlap of batches on the
device, and identical images alone and in a mix of concurrent requests."""
import numpy as np
import pytest
import torch

from paper_2502_01157_gb300 import rf
from paper_2502_01157_gb300 import scenes as S
from paper_2502_01157_gb300.serve import Server, run_open_loop
from tests.helpers import camera_at, random_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def foam():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    sc = random_scene(4000, 3, 77)
    rng = np.random.default_rng(78)
    sc.sh[:, 1:, :] = rng.normal(0, 0.3, sc.sh[:, 1:, :].shape).astype(np.float32)
    f = rf.Foam.from_scene(sc, attr_dtype=torch.bfloat16)
    yield f
    f.close()


def _cams(n, seed):
    rng = np.random.default_rng(seed)
    sizes = [(32, 24), (64, 48), (128, 72), (192, 108)]
    out = []
    for k in range(n):
        w, h = sizes[rng.integers(0, len(sizes))]
        v = rng.normal(size=3)
        out.append(S.pinhole(w, h, 60.0, c2w=S.look_at(2.4 * v / np.linalg.norm(v))))
    return out


def _image(foam, cam):
    out = foam.render([cam])
    torch.cuda.synchronize()
    return out["rgb"].cpu().numpy()


def test_result_is_the_same_alone_and_in_the_mix(foam):
    target = S.pinhole(96, 64, 60.0, c2w=S.look_at((1.5, -1.8, 0.9)))
    ref = _image(foam, target)
    srv = Server(foam, mem_budget_bytes=64 << 20, max_inflight=64, n_streams=3, max_batch=4)
    alone = np.zeros((target.n_rays, 3), np.float32)
    srv.wait(srv.submit(target), out=alone)
    np.testing.assert_array_equal(alone, ref)
    # the same request again, submitted in the middle of a burst of others
    others = _cams(40, 1)
    ids = [srv.submit(c) for c in others[:20]]
    mine = srv.submit(target)
    ids += [srv.submit(c) for c in others[20:]]
    mixed = np.zeros_like(alone)
    srv.wait(mine, out=mixed)
    for rid, cam in zip(ids, others):
        if rid is not None:
            img = np.zeros((cam.n_rays, 3), np.float32)
            srv.wait(rid, out=img)
            np.testing.assert_array_equal(img, _image(foam, cam))
    np.testing.assert_array_equal(mixed, ref)
    st = srv.stats()
    assert st["mean_batch"] > 1.0, st          # requests were batched together
    assert st["max_busy_streams"] > 1, st      # batches overlapped on the device
    srv.close()


def test_admission_by_memory(foam):
    cam = S.pinhole(40, 30, 60.0, c2w=S.look_at((2.0, 1.0, 0.5)))
    srv = Server(foam, mem_budget_bytes=2 * cam.n_rays * 20, max_inflight=8, n_streams=1, max_batch=1)
    a = srv.submit(cam)
    b = srv.submit(cam)
    assert a is not None and b is not None
    assert srv.submit(cam) is None            # no memory left: rejected at once
    srv.wait(a)                               # collecting a frees its memory
    c = srv.submit(cam)
    assert c is not None
    srv.wait(b)
    srv.wait(c)
    big = S.pinhole(400, 300, 60.0, c2w=S.look_at((2.0, 1.0, 0.5)))
    with pytest.raises(rf.RFError) as e:
        srv.submit(big)                       # can never fit
    assert e.value.code == 1
    assert srv.stats()["rejected"] >= 2
    srv.close()


def test_slot_limit_and_invalid_requests(foam):
    cam = S.pinhole(16, 16, 60.0, c2w=S.look_at((2.0, 0.0, 0.0)))
    srv = Server(foam, mem_budget_bytes=16 << 20, max_inflight=2, n_streams=2, max_batch=2)
    ids = [srv.submit(cam), srv.submit(cam)]
    assert srv.submit(cam) is None
    bad = S.pinhole(16, 16, 60.0, c2w=S.look_at((2.0, 0.0, 0.0)))
    bad.c2w[1, 3] = np.inf
    with pytest.raises(rf.RFError):
        srv.submit(bad)
    for rid in ids:
        srv.wait(rid)
    with pytest.raises(rf.RFError) as e:
        srv.poll(ids[0])                      # already collected
    assert e.value.code == 8
    srv.close()


def test_open_loop_poisson_stream(foam):
    cams = _cams(300, 5)
    arrivals = S.poisson_arrivals(600.0, len(cams), 9)
    srv = Server(foam, mem_budget_bytes=256 << 20, max_inflight=128, n_streams=4, max_batch=8)
    st = run_open_loop(srv, cams, arrivals)
    assert st["completed"] + st["rejected_open_loop"] == len(cams)
    assert st["completed"] > 0.9 * len(cams)
    assert 0 < st["p50_ms"] <= st["p99_ms"]
    print("serve", {k: st[k] for k in ("completed", "rejected_open_loop", "p50_ms", "p99_ms",
                                         "mrays_s", "mean_batch", "max_busy_streams")})
    srv.close()


def test_fisheye_and_rolling_shutter_requests(foam):
    # non-pinhole cameras go through the same batches (effects kernels)
    fish = S.fisheye(48, 40, 190.0, c2w=S.look_at((1.2, 0.9, -0.4)))
    roll = S.Camera(**{**S.pinhole(40, 30, 60.0, c2w=S.look_at((-1.5, 0.5, 1.0))).__dict__,
                       "shutter": (0.1, 0.05, 0.0)})
    srv = Server(foam, mem_budget_bytes=64 << 20, max_inflight=16, n_streams=2, max_batch=4)
    pins = [S.pinhole(32, 24, 60.0, c2w=S.look_at((2.0, -1.0, 0.3))) for _ in range(3)]
    ids = [(srv.submit(c), c) for c in pins[:2] + [fish, roll] + pins[2:]]
    for rid, cam in ids:
        img = np.zeros((cam.n_rays, 3), np.float32)
        srv.wait(rid, out=img)
        np.testing.assert_array_equal(img, _image(foam, cam))
    srv.close()


def test_served_images_match_the_oracle(foam):
    """Requests of mixed sizes served concurrently: each image against the
    FP64 oracle (on the BF16-rounded attributes the server renders) on
    sampled pixels, within the image tolerance."""
    import oracle
    from tests.parity import IMG_RMSE

    sc = random_scene(4000, 3, 77)
    rng = np.random.default_rng(78)
    sc.sh[:, 1:, :] = rng.normal(0, 0.3, sc.sh[:, 1:, :].shape).astype(np.float32)
    sc.density = torch.from_numpy(sc.density).bfloat16().float().numpy()
    sc.sh = torch.from_numpy(sc.sh).bfloat16().float().numpy()
    P = oracle.prepare(sc)
    cams = _cams(12, 5)
    srv = Server(foam, mem_budget_bytes=64 << 20, max_inflight=64, n_streams=3, max_batch=4)
    ids = [srv.submit(c) for c in cams]
    assert all(r is not None for r in ids)
    for rid, cam in zip(ids, cams):
        img = np.zeros((cam.n_rays, 3), np.float32)
        srv.wait(rid, out=img)
        px = np.sort(rng.choice(cam.n_rays, size=min(256, cam.n_rays), replace=False))
        o = oracle.render(P, cam, pixels=px)
        err = float(np.sqrt(np.mean((img[px].astype(np.float64) - o["rgb"]) ** 2)))
        assert err <= IMG_RMSE, f"{cam.width}x{cam.height}: rmse {err:.2e}"
    srv.close()
