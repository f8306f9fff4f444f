"""The roofline accounting in bench.py: algorithmic bytes per cell step as
stated for the forward (no reuse), the replayed backward and the gradient
read-modify-write, and the clock-record parser."""
import bench


def test_bytes_per_cell_step():
    # header 16 + 15.5 faces x 12 + neighbour id 4 + density + SH
    assert bench.bytes_per_step(15.5, 3, 4) == 16 + 186 + 4 + 4 + 192 == 402
    assert bench.bytes_per_step(15.5, 3, 2) == 16 + 186 + 4 + 2 + 96 == 304
    assert bench.bytes_per_step(15.5, 0, 4) == 16 + 186 + 4 + 4 + 12
    # replayed backward: record byte, header, one exit face, its id, density, SH
    assert bench.replay_bytes_per_step(3, 4) == 1 + 16 + 12 + 4 + 4 + 192 == 229
    # gradient read-modify-write: density, SH row, two site positions
    assert bench.bwd_extra_bytes_per_step(3) == 2 * (4 + 192 + 24) == 440
    assert bench.replay_bytes_per_step(3, 4) + bench.bwd_extra_bytes_per_step(3) == 669


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
