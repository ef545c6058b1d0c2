"""Host logic of the measurement (bench.py), on the CPU: the FP32 work counted per pair of the
linear-chirp statistic, the choice of the roofline's bound for a gather launch, and the rule that
the DRAM traffic committed under profiles/ is used only while the statistic kernel's sources are
the ones it was captured on."""
import ctypes
import math
import re

import pytest

import bench


def test_chirp_flops_per_pair():
    # 5 M log2 M for the template's M-point FFT, 6 per windowed sample, 12 per bin of 2P + 1
    assert bench.chirp_flops_pair(256, 100) == 5 * 256 * 8 + 6 * 256 + 12 * 201 == 14188
    assert bench.chirp_flops_pair(256, 0) == 5 * 256 * 8 + 6 * 256 + 12


class _FakeLib:
    """Stands in for libtfstat's L2 read probe (no GPU here)."""

    def __init__(self, gbs, rc=0):
        self.gbs, self.rc = gbs, rc

    def tfs_measure_l2_read(self, nbytes, passes, out):
        ctypes.cast(out, ctypes.POINTER(ctypes.c_double))[0] = self.gbs
        return self.rc


def test_gather_roofline_bound_follows_the_resident_bytes():
    hbm, _ = bench.measured_peaks()
    alg, ms = 4432 * 10**7, 2.68  # one-year FP32 launch: algorithmic bytes, kernel time
    achieved = alg / (ms / 1e3) / 1e9
    # a table and window sums that stay in L2 (25 MB): bounded by the L2 read rate measured now
    r = bench.gather_roofline(alg, ms, 25e6, _FakeLib(18000.0), "k")
    assert r["bound"] == "l2" and r["unit"] == "GB/s" and r["peak"] == 18000.0
    assert r["achieved"] == pytest.approx(achieved) and r["frac"] == pytest.approx(achieved / 18000.0)
    assert r["frac_of_hbm"] == pytest.approx(achieved / hbm)
    # larger than L2 (1.9 GB of tables): bounded by the HBM copy rate
    r = bench.gather_roofline(alg, ms, 1.9e9, _FakeLib(18000.0), "k")
    assert r["bound"] == "hbm" and r["peak"] == hbm and r["frac"] == pytest.approx(achieved / hbm)
    # no L2 figure (the probe failed): HBM, whatever the size
    r = bench.gather_roofline(alg, ms, 25e6, _FakeLib(0.0, rc=1), "k")
    assert r["bound"] == "hbm" and r["frac_of_l2"] is None


def test_profiled_traffic_only_for_the_captured_sources(monkeypatch):
    txt = open(bench.os.path.join(bench.ROOT, "profiles", "eval_stat_kernel_oneyear_daily_fp32_f32.md")).read()
    h = re.search(r"kernel source hash:\s*([0-9a-f]+)", txt).group(1)
    dram = float(re.search(r"dram bytes per full launch:\s*([0-9.e+]+)", txt).group(1))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.profiled_traffic("oneyear_daily_fp32", "f32") == dram
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.profiled_traffic("oneyear_daily_fp32", "f32") is None
    assert bench.profiled_traffic("no_such_workload", "f32") is None
    assert math.isfinite(dram) and dram > 0
