"""The roofline accounting in bench.py: algorithmic bytes per cell step (what
a step reads with no reuse: CSR offsets, one 16-byte record per face,
density and the SH row; the backward adds the gradient read-modify-write),
the counters file, the L1 ceiling, and the clock-record parser."""
import bench


def test_bytes_per_cell_step():
    # offsets 8 + 15.5 faces x 16 + density + SH
    assert bench.bytes_per_step(15.5, 3, 4) == 8 + 248 + 4 + 192 == 452
    assert bench.bytes_per_step(15.5, 3, 2) == 8 + 248 + 2 + 96 == 354
    assert bench.bytes_per_step(15.5, 0, 4) == 8 + 248 + 4 + 12 == 272
    # gradient read-modify-write: density, SH row, two site positions
    assert bench.bwd_extra_bytes_per_step(3) == 2 * (4 + 192 + 24) == 440
    # fwd + bwd (re-walk) per step: 452 + 452 + 440
    assert 2 * bench.bytes_per_step(15.5, 3, 4) + bench.bwd_extra_bytes_per_step(3) == 1344


def test_kernel_counters_follow_the_sources(tmp_path, monkeypatch):
    path = tmp_path / "kernel_counters.txt"
    src = bench.kernel_source_hash()
    path.write_text("# kernel workload sources steps dram lts l1_wavefronts lsu_pct occupancy\n"
                    f"bwd_kernel<float,3> c3 {src} 1000 2000 30000 500000 76.5 35.5\n"
                    "bwd_kernel<float,3> c3 0123456789ab 1000 9 9 9 9 9\n")
    monkeypatch.setattr(bench, "COUNTERS", str(path))
    c = bench.kernel_counters("bwd_kernel<float,3>", "c3")
    assert c["dram_bytes_per_step"] == 2.0 and c["lts_bytes_per_step"] == 30.0
    assert c["l1_wavefronts_per_step"] == 500.0 and c["l1_lsu_pct"] == 76.5
    assert bench.kernel_counters("fwd_kernel<float,3>", "c3") is None
    path.write_text(f"bwd_kernel<float,3> c3 0123456789ab 1000 9 9 9 9 9\n")
    assert bench.kernel_counters("bwd_kernel<float,3>", "c3") is None   # other kernel sources


def test_clock_record_parser(tmp_path, monkeypatch):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("2070, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c.proc = Done()
    c.f = open(str(tmp_path / "unused"), "w")
    r = c.stop()
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
