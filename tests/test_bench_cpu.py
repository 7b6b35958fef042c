"""Host logic of the benchmark's measurement (no GPU): the clock record that
decides whether a timed run is kept, the DRAM-traffic record that is only
reported for the kernel source it was measured on, and the byte counts the
roofline fractions divide by."""
import hashlib
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampled(bench, rows):
    cs = bench.ClockSampler(0)
    cs.p = _Done()                      # the nvidia-smi process: already finished
    cs.f.write("\n".join(rows) + "\n")
    cs.f.flush()
    return cs.stop()


def test_clock_record_median_and_no_reasons():
    b = _bench()
    rows = [f"0, {mhz}, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active"
            for mhz in (2070, 2070, 1995, 2070, 2055)]
    rec = _sampled(b, rows)
    assert rec["sm_mhz"] == 2070 and rec["sm_max_mhz"] == 2070 and rec["samples"] == 5
    assert rec["reasons"] == []


def test_clock_record_flags_each_throttle_reason():
    b = _bench()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for k, name in enumerate(names):
        flags = ["Active" if i == k else "Not Active" for i in range(4)]
        rows = ["0, 1800, 2070, 1380.0, 0x4, " + ", ".join(flags),
                "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
        assert _sampled(b, rows)["reasons"] == [name]


def test_clock_record_skips_malformed_rows():
    b = _bench()
    rows = ["garbage", "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2000, 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    rec = _sampled(b, rows)
    assert rec["samples"] == 1 and rec["sm_mhz"] == 2000


def test_traffic_reported_only_for_the_measured_source(monkeypatch):
    b = _bench()
    src = "paper_1905_12154_gb300/csrc/ctransform.cu"
    h = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()
    monkeypatch.setitem(b.TRAFFIC, "probe_kind", {"bytes": 123.0, "source": src, "sha256": h})
    assert b.traffic_of("probe_kind") == 123.0
    monkeypatch.setitem(b.TRAFFIC, "probe_kind", {"bytes": 123.0, "source": src, "sha256": "0" * 64})
    assert b.traffic_of("probe_kind") is None
    monkeypatch.setitem(b.TRAFFIC, "probe_kind", {"bytes": 1.0, "source": "no/such/file.cu",
                                                  "sha256": h})
    assert b.traffic_of("probe_kind") is None
    assert b.traffic_of("kind_without_a_record") is None


def test_algorithmic_bytes_per_iteration():
    b = _bench()
    # 4 c-transforms of two 12-byte sweeps, 2 Poisson solves (12 + 8 + 12), 2
    # pushforwards of 16 bytes per cell
    assert b.METHOD_BYTES_PER_CELL_ITER == 192
    # of L transposes per iteration, L - 8 also read a weight (12 bytes), the
    # others read and write (8 bytes)
    assert abs(b.transpose_bytes_per_cell(10) - (2 * 12 + 8 * 8) / 10) < 1e-12
    assert b.transpose_bytes_per_cell(8) == 8
    assert b.BYTES_PER_CELL_2D_TRANSPOSED["ct_pass_axis1"] == 8


def test_map_difference_separates_split_points():
    """A map that jumps by 10 cells along one column (mass split between two
    targets): an FP32 map that sends the cells beside the jump to the other
    side differs by 10 cells there, but by 0.01 cells off the split points."""
    import torch
    b = _bench()
    n = 16
    x = (torch.arange(n, dtype=torch.float64) + 0.5) / n
    X, Y = x[None, :].expand(n, n), x[:, None].expand(n, n)
    m64 = torch.stack([X.clone(), Y.clone()])
    m64[0, :, 8:] += 10.0 / n                     # the jump between columns 7 and 8
    m32 = m64.clone()
    m32[0] += 0.01 / n
    m32[0, :, 8] -= 10.0 / n                      # column 8 lands on the other side
    mu = torch.ones(n, n, dtype=torch.float64)
    r = b.map_difference(m32, m64, mu, n)
    assert abs(r["map_linf_cells_on_mu_support"] - 9.99) < 1e-9
    assert abs(r["map_linf_cells_off_split_points"] - 0.01) < 1e-9
    assert abs(r["split_points_mass_share"] - 4.0 / n) < 1e-12   # columns 6-9
