"""GPU Voronoi adjacency (the neighbour lists of Alg. 1, rebuilt when the
sites move) against the FP64 face-polygon oracle: identical lists, through
the C ABI, on uniform and clustered sites, incremental rebuilds, cells with
many faces, small closed-form sets and the 3M-site scene (sampled)."""
import numpy as np
import pytest
import torch

import oracle  # noqa: F401  (builds the oracle library)
from oracle import adjacency as A
from paper_2502_01157_gb300 import rf
from paper_2502_01157_gb300 import scenes as S
from tests.helpers import random_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    rf.lib()


@pytest.fixture(scope="module")
def builder():
    b = rf.Adjacency()
    yield b
    b.close()


def _gpu_rows(builder, pos, domain=None, incremental=False):
    off, idx = builder.build(torch.from_numpy(np.ascontiguousarray(pos, np.float32)).cuda(), domain=domain,
                             incremental=incremental)
    torch.cuda.synchronize()
    off, idx = off.cpu().numpy(), idx.cpu().numpy()
    return [idx[off[i]:off[i + 1]] for i in range(len(off) - 1)], off, idx


def _compare(gpu_rows, pos, domain, sites=None):
    sites = np.arange(len(pos)) if sites is None else np.asarray(sites)
    nb, areas = A.voronoi_neighbors(np.asarray(pos, np.float64), sites=sites, domain=np.asarray(domain, np.float64))
    bad = [(int(s), sorted(set(gpu_rows[s]) ^ set(nb[q].tolist())))
           for q, s in enumerate(sites) if not np.array_equal(gpu_rows[s], nb[q])]
    return bad, areas


def _domain(lo, hi):
    return np.array([lo, lo, lo, hi, hi, hi], np.float32)


@pytest.mark.parametrize("kind,n,seed", [("uniform", 5000, 1), ("uniform", 20000, 2), ("mixture", 20000, 3)])
def test_matches_oracle(builder, kind, n, seed):
    rng = np.random.default_rng(seed)
    pos = S.uniform_sites(n, -1, 1, rng) if kind == "uniform" else S.mixture_sites(n, rng)
    pos = S.dedupe_sites(pos, rng)
    dom = _domain(-1.1, 1.1) if kind == "uniform" else _domain(-10.5, 10.5)
    rows, off, idx = _gpu_rows(builder, pos, dom)
    st = builder.stats
    print(f"{kind} {n}: edges {st['n_edges']} (mean degree {st['n_edges'] / n:.2f}), max degree "
          f"{st['max_degree']}, asym added {st['asym_added']}, wide {st['wide_sites']}, "
          f"failed {st['failed_sites']}, fp64 tests {st['fp64_tests']}")
    bad, _ = _compare(rows, pos, dom)
    assert not bad, bad[:5]
    assert st["failed_sites"] == 0 and st["asym_added"] == 0
    # symmetric, sorted, no self loops
    src = np.repeat(np.arange(n), np.diff(off))
    assert np.all(idx != src)
    key = np.sort(src.astype(np.int64) * n + idx)
    rkey = np.sort(idx.astype(np.int64) * n + src)
    assert np.array_equal(key, rkey)
    assert all(np.all(np.diff(r) > 0) for r in rows)


def test_default_domain_is_the_grown_box(builder):
    rng = np.random.default_rng(9)
    pos = S.uniform_sites(3000, -0.5, 2.0, rng)
    rows, _, _ = _gpu_rows(builder, pos)
    lo, hi = pos.min(0).astype(np.float64), pos.max(0).astype(np.float64)
    m = np.maximum(0.05 * (hi - lo), 1e-3)
    expect = np.concatenate([lo - m, hi + m]).astype(np.float32)
    np.testing.assert_array_equal(np.asarray(builder.stats["domain"], np.float32), expect)
    bad, _ = _compare(rows, pos, expect)
    assert not bad, bad[:5]


def test_incremental_rebuild_equals_full_build(builder):
    rng = np.random.default_rng(12)
    pos = S.dedupe_sites(S.uniform_sites(20000, -1, 1, rng), rng)
    dom = _domain(-1.2, 1.2)
    _gpu_rows(builder, pos, dom)
    moved = (pos + rng.normal(0, 0.01, pos.shape)).astype(np.float32)   # ~1/4 of the spacing
    inc, off_i, idx_i = _gpu_rows(builder, moved, dom, incremental=True)
    full, off_f, idx_f = _gpu_rows(builder, moved, dom)
    assert np.array_equal(off_i, off_f) and np.array_equal(idx_i, idx_f)
    sample = rng.choice(len(pos), 2000, replace=False)
    bad, _ = _compare(inc, moved, dom, sample)
    assert not bad, bad[:5]


def test_cell_with_many_faces_takes_the_wide_pass(builder):
    # a site at the centre of 90 sites spread over a sphere: 90 faces
    k = np.arange(90) + 0.5
    phi = np.arccos(1 - 2 * k / 90)
    th = np.pi * (1 + 5 ** 0.5) * k
    ring = np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)
    rng = np.random.default_rng(5)
    pos = np.concatenate([[[0.0, 0.0, 0.0]], ring * (1 + 0.01 * rng.normal(size=(90, 1)))]).astype(np.float32)
    dom = _domain(-2, 2)
    rows, _, _ = _gpu_rows(builder, pos, dom)
    assert len(rows[0]) == 90 and builder.stats["wide_sites"] >= 1
    bad, _ = _compare(rows, pos, dom)
    assert not bad, bad[:5]


def test_small_closed_form_sets(builder):
    one, _, _ = _gpu_rows(builder, np.zeros((1, 3), np.float32), _domain(-1, 1))
    assert len(one[0]) == 0
    two, _, _ = _gpu_rows(builder, np.array([[-0.5, 0, 0], [0.5, 0, 0]], np.float32), _domain(-1, 1))
    assert [list(r) for r in two] == [[1], [0]]
    t = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1], [0, 0, 0]], np.float32) * 0.4
    # an asymmetric box: in a box centred on the tetrahedron the bisectors run
    # exactly through box corners (four planes through one point)
    dom = np.array([-50, -47, -53, 51, 49, 46], np.float32)
    tet, _, _ = _gpu_rows(builder, t, dom)
    print("tetrahedron", [list(r) for r in tet], builder.stats)
    assert all(list(tet[i]) == [j for j in range(5) if j != i] for i in range(5))
    x = np.array([0.0, 0.3, 1.1, 1.5, 2.6], np.float32)
    line = np.stack([x, np.full(5, 0.1, np.float32), np.full(5, -0.2, np.float32)], 1)
    lr, _, _ = _gpu_rows(builder, line, np.array([-1, -1, -1, 4, 1, 1], np.float32))
    assert [list(r) for r in lr] == [[1], [0, 2], [1, 3], [2, 4], [3]]


def test_renders_like_the_qhull_adjacency():
    # Qhull's lists also hold faces far outside any finite domain (between
    # nearly coplanar hull sites); the walk inside the box never uses them
    sc = random_scene(4000, 2, 31)
    foam_q = rf.Foam.from_scene(sc)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float32)
    dom = np.array([-3, -3, -3, 3, 3, 3], np.float32)
    foam_g = rf.Foam.from_sites(t(sc.pos), t(sc.density), t(sc.sh), domain=dom,
                                aabb=(sc.aabb_min, sc.aabb_max))
    og, ig = foam_g.adj_off.cpu().numpy(), foam_g.adj_idx.cpu().numpy()
    differ = 0
    for i in range(sc.n_sites):
        g = set(ig[og[i]:og[i + 1]].tolist())
        q = set(sc.adj_idx[sc.adj_off[i]:sc.adj_off[i + 1]].tolist())
        assert g <= q
        differ += g != q
    print(f"sites whose Qhull list has faces beyond the domain: {differ}")
    assert differ < sc.n_sites // 20
    for cam in (S.pinhole(48, 32, 60.0, c2w=S.look_at((0.1, 0.05, -0.02), (1.0, 0.3, 0.2))),
                S.pinhole(40, 30, 50.0, c2w=S.look_at((2.5, 1.0, -1.5), (0.0, 0.0, 0.0)))):
        a, b = foam_q.render([cam]), foam_g.render([cam])
        torch.cuda.synchronize()
        for k in ("rgb", "trans", "depth"):
            assert torch.equal(a[k], b[k])


def test_invalid_inputs_are_rejected(builder):
    pos = torch.zeros(4, 3, device="cuda")
    pos[1, 0] = 1.0
    pos[2, 1] = 1.0
    pos[3, 2] = float("nan")
    with pytest.raises(rf.RFError, match="finite"):
        builder.build(pos)
    pos[3, 2] = 5.0
    with pytest.raises(rf.RFError, match="inside the domain"):
        builder.build(pos, domain=[-1, -1, -1, 2, 2, 2])
    with pytest.raises(rf.RFError):
        builder.build(pos, domain=[1, -1, -1, -2, 2, 2])


def test_full_size_3m_sites_sampled(builder):
    sc = S.config_scene("c3")
    pos = torch.from_numpy(sc.pos).cuda()
    dom = _domain(-1.05, 1.05)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    builder.build(pos, domain=dom)    # warm-up (allocations)
    torch.cuda.synchronize()
    ev[0].record()
    off, idx = builder.build(pos, domain=dom)
    ev[1].record()
    torch.cuda.synchronize()
    st = builder.stats
    print(f"3M sites: {ev[0].elapsed_time(ev[1]):.1f} ms, edges {st['n_edges']}, max degree {st['max_degree']}, "
          f"wide {st['wide_sites']}, failed {st['failed_sites']}, asym {st['asym_added']}, fp64 {st['fp64_tests']}")
    off, idx = off.cpu().numpy(), idx.cpu().numpy()
    rows = [None] * sc.n_sites
    rng = np.random.default_rng(8)
    sample = rng.choice(sc.n_sites, 1500, replace=False)
    for s in sample:
        rows[s] = idx[off[s]:off[s + 1]]
    bad, _ = _compare(rows, sc.pos, dom, sample)
    assert not bad, bad[:5]
    assert st["failed_sites"] == 0


def test_training_loop_rebuild_matches_a_fresh_foam():
    # sites move (a position step), the foam re-packs, the lists are rebuilt
    # incrementally: the renders equal those of a foam built from scratch
    rng = np.random.default_rng(21)
    sc = random_scene(5000, 1, 22)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float32)
    dom = np.array([-1.3, -1.3, -1.3, 1.3, 1.3, 1.3], np.float32)
    box = (np.full(3, -1.2, np.float32), np.full(3, 1.2, np.float32))
    foam = rf.Foam.from_sites(t(sc.pos), t(sc.density), t(sc.sh), domain=dom, aabb=box)
    cam = S.pinhole(40, 30, 60.0, c2w=S.look_at((0.1, -0.05, 0.02), (1.0, 0.4, 0.2)))
    for step in range(3):
        moved = (foam.pos + 0.004 * torch.from_numpy(rng.normal(size=sc.pos.shape).astype(np.float32)).cuda())
        foam.update_positions(moved.clamp(-1.15, 1.15))
        st = foam.rebuild_adjacency(domain=dom, incremental=True)
        fresh = rf.Foam.from_sites(foam.pos.clone(), t(sc.density), t(sc.sh), domain=dom, aabb=box)
        assert torch.equal(foam.adj_off, fresh.adj_off) and torch.equal(foam.adj_idx, fresh.adj_idx)
        a, b = foam.render([cam]), fresh.render([cam])
        torch.cuda.synchronize()
        for k in ("rgb", "trans", "depth"):
            assert torch.equal(a[k], b[k]), (step, k)
        assert st["failed_sites"] == 0
        fresh.close()
    foam.close()
