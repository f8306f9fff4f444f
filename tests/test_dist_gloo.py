"""The multi-rank path on CPU (gloo, world size 2): cameras sharded across
ranks, per-rank gradients summed by the all-reduce, timing maximum over ranks.
The per-rank gradients come from the FP64 oracle, so the test checks the
host-side partition and reduction logic without a GPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2502_01157_gb300 import dist as D
from tests.helpers import camera_at, random_scene


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _cams():
    return [camera_at((0.1 * k, 0.05, -0.02), (0.3, 1.0 - 0.2 * k, 0.2), w=7, h=5) for k in range(5)]


def _worker(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = random_scene(400, 1, 3)
    mine = D.shard(_cams(), rank, world)
    g = dict(density=torch.zeros(sc.n_sites, dtype=torch.float64),
             sh=torch.zeros(sc.sh.shape, dtype=torch.float64),
             pos=torch.zeros(sc.n_sites, 3, dtype=torch.float64))
    for cam in mine:
        o = oracle.render(sc, cam)
        G = oracle.render_bwd(sc, cam, np.ones_like(o["rgb"]), threads=1)
        for k in g:
            g[k] += torch.from_numpy(G[k])
    D.allreduce_grads(g)
    slow = D.max_over_ranks(float(rank + 1))
    if rank == 0:
        torch.save(dict(g={k: v.numpy() for k, v in g.items()}, slow=slow,
                        n_mine=len(mine)), out_path)
    dist.destroy_process_group()


def test_shard_is_a_partition():
    items = list(range(11))
    parts = [D.shard(items, r, 3) for r in range(3)]
    assert sum(parts, []) == items
    assert max(map(len, parts)) - min(map(len, parts)) <= 1


def test_two_rank_gradient_allreduce(tmp_path):
    out = str(tmp_path / "r0.pt")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    res = torch.load(out, weights_only=False)
    sc = random_scene(400, 1, 3)
    ref = dict(density=0, sh=0, pos=0)
    for cam in _cams():
        o = oracle.render(sc, cam)
        G = oracle.render_bwd(sc, cam, np.ones_like(o["rgb"]), threads=1)
        for k in ref:
            ref[k] = ref[k] + G[k]
    for k in ref:
        np.testing.assert_allclose(res["g"][k], ref[k], rtol=1e-12, atol=1e-14)
    assert res["slow"] == 2.0
    assert res["n_mine"] == 2
