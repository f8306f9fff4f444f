"""Stored FP64 oracle values (``tests/golden/c1_oracle_sample.txt``, written
by ``tests/golden/make_golden.py`` from ``oracle/`` alone) on 48 pixels of
the 4,096-site, 64x64 workload: the oracle must still produce them, and the
CUDA path must match them within the parity tolerances."""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "c1_oracle_sample.txt")


def load():
    px, g_in, fwd, sites, grads = [], [], [], [], []
    for line in open(GOLDEN):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "px":
            bar = f.index("|")
            px.append(int(f[1]))
            g_in.append([float(v) for v in f[2:bar]])
            fwd.append([float(v) for v in f[bar + 1:]])
        elif f[0] == "site":
            sites.append(int(f[1]))
            grads.append([float(v) for v in f[2:]])
    g_in, fwd, grads = np.array(g_in), np.array(fwd), np.array(grads)
    return dict(px=np.array(px, np.int64), g_rgb=g_in[:, :3], g_trans=g_in[:, 3], g_depth=g_in[:, 4],
                rgb=fwd[:, :3], trans=fwd[:, 3], depth=fwd[:, 4], steps=fwd[:, 5].astype(int),
                flags=fwd[:, 6].astype(np.uint8), sites=np.array(sites, np.int64), grads=grads)


def test_fixture_is_well_formed():
    G = load()
    assert len(G["px"]) == 48 and len(np.unique(G["px"])) == 48
    assert np.all((G["px"] >= 0) & (G["px"] < 64 * 64))
    assert np.all((G["trans"] >= 0) & (G["trans"] <= 1)) and np.all(G["rgb"] >= 0)
    assert len(G["sites"]) == 24 and G["grads"].shape == (24, 7)


def test_oracle_reproduces_the_fixture():
    import oracle
    from paper_2502_01157_gb300 import scenes as S

    G = load()
    scene = S.config_scene("c1")
    cam = S.config_cameras("c1")[0]
    f = oracle.render(scene, cam, pixels=G["px"])
    for k in ("rgb", "trans", "depth"):
        np.testing.assert_allclose(f[k], G[k], rtol=1e-12, atol=1e-14, err_msg=k)
    np.testing.assert_array_equal(f["steps"], G["steps"])
    np.testing.assert_array_equal(f["flags"], G["flags"])
    g = oracle.render_bwd(scene, cam, G["g_rgb"], G["g_trans"], G["g_depth"], pixels=G["px"])
    got = np.concatenate([g["density"][G["sites"], None], g["sh"][G["sites"], 0], g["pos"][G["sites"]]], 1)
    # gradients are sums over rays in thread order: equal up to rounding
    np.testing.assert_allclose(got, G["grads"], rtol=1e-9, atol=1e-13)


@pytest.mark.gpu
def test_cuda_matches_the_fixture():
    import torch

    from paper_2502_01157_gb300 import rf
    from paper_2502_01157_gb300 import scenes as S

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    G = load()
    scene = S.config_scene("c1")
    cam = S.config_cameras("c1")[0]
    foam = rf.Foam.from_scene(scene)
    out = foam.render([cam], steps=True)
    px = torch.from_numpy(G["px"]).cuda()
    # equal step counts wherever the oracle sees no tie of cells or stop
    keep = (G["flags"] & 7) == 0
    for k in ("rgb", "trans", "depth"):
        a = out[k][px].double().cpu().numpy()
        err = float(np.sqrt(np.mean((a - G[k]) ** 2)))
        assert err <= 1e-5, f"{k}: rmse {err:.3e}"
    np.testing.assert_array_equal(out["steps"][px].cpu().numpy()[keep], G["steps"][keep])
    # the same upstream gradients on the sampled pixels, zero elsewhere
    R = cam.n_rays
    d_rgb = torch.zeros(R, 3, device="cuda")
    d_t = torch.zeros(R, device="cuda")
    d_d = torch.zeros(R, device="cuda")
    d_rgb[px] = torch.from_numpy(G["g_rgb"]).float().cuda()
    d_t[px] = torch.from_numpy(G["g_trans"]).float().cuda()
    d_d[px] = torch.from_numpy(G["g_depth"]).float().cuda()
    g = foam.backward([cam], out, d_rgb, d_t, d_d)
    s = torch.from_numpy(G["sites"]).cuda()
    got = torch.cat([g["density"][s, None], g["sh"][s, 0], g["pos"][s]], 1).double().cpu().numpy()
    rel = np.linalg.norm(got - G["grads"]) / np.linalg.norm(G["grads"])
    assert rel <= 1e-3, f"gradient rel err {rel:.3e}"
