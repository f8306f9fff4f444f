"""Writes ``c1_oracle_sample.txt``: FP64 oracle values on a fixed sample of
the 4,096-site, 64x64 workload, kept as a fixture so that a later change to
the oracle's arithmetic, or to the CUDA path, shows up against stored numbers.

Everything here comes from ``oracle/`` (the forward of Alg. 1 with the
compositing of Eq. 3-4, and its analytic backward of Sec. 3.1) and from the
seeded input generators; nothing comes from the CUDA path.

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "c1_oracle_sample.txt")
N_PIXELS = 48
N_SITES_KEPT = 24


def sample():
    """The pixels and upstream gradients of the fixture (seeded)."""
    rng = np.random.default_rng(20250201)
    px = np.sort(rng.choice(64 * 64, size=N_PIXELS, replace=False)).astype(np.int64)
    g_rgb = rng.uniform(-1.0, 1.0, size=(N_PIXELS, 3))
    g_trans = np.full(N_PIXELS, 0.25)
    g_depth = np.full(N_PIXELS, 0.1)
    return px, g_rgb, g_trans, g_depth


def compute():
    import oracle
    from paper_2502_01157_gb300 import scenes as S

    scene = S.config_scene("c1")
    cam = S.config_cameras("c1")[0]
    px, g_rgb, g_trans, g_depth = sample()
    f = oracle.render(scene, cam, pixels=px)
    g = oracle.render_bwd(scene, cam, g_rgb, g_trans, g_depth, pixels=px)
    # the sites with the largest density gradients, ties broken by id
    order = np.lexsort((np.arange(scene.n_sites), -np.abs(g["density"])))[:N_SITES_KEPT]
    sites = np.sort(order)
    return px, g_rgb, g_trans, g_depth, f, g, sites


def main():
    px, g_rgb, g_trans, g_depth, f, g, sites = compute()
    lines = [
        "# FP64 oracle on the 4,096-site workload (sites uniform in [-1,1]^3, seed 1001, SH degree 0,",
        "# one 64x64 pinhole camera at the origin, 60 degree field of view, eps 1e-4).",
        "# Forward: Alg. 1 walk with the compositing of Eq. 3-4.  Backward: the analytic gradient",
        "# of Sec. 3.1 (density, SH, and positions through the segment widths) of",
        "# sum(g_rgb * rgb) + sum(g_trans * T) + sum(g_depth * depth) over the sampled pixels.",
        "# Written by tests/golden/make_golden.py, which calls only oracle/ and the input generators.",
        "# pixel  g_r  g_g  g_b  g_T  g_depth  |  r  g  b  T  depth  steps  flags",
        "# (flags: near-degenerate classes, 1 edge/vertex tie, 2 camera tie, 4 stop tie, 8 grazing, 16 bend)",
    ]
    for k in range(len(px)):
        lines.append("px %d %r %r %r %r %r | %r %r %r %r %r %d %d" % (
            px[k], *map(float, g_rgb[k]), float(g_trans[k]), float(g_depth[k]),
            *map(float, f["rgb"][k]), float(f["trans"][k]), float(f["depth"][k]),
            int(f["steps"][k]), int(f["flags"][k])))
    lines.append("# site  d_sigma  d_sh(r, g, b)  d_pos(x, y, z)")
    for i in sites:
        lines.append("site %d %r %r %r %r %r %r %r" % (
            i, float(g["density"][i]), *map(float, g["sh"][i, 0]), *map(float, g["pos"][i])))
    with open(OUT, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print(f"wrote {OUT}: {len(px)} pixels, {len(sites)} sites")


if __name__ == "__main__":
    main()
