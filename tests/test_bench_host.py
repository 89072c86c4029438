"""Host logic of bench.py that feeds its JSON line: the algorithmic bytes of
one SpMV launch (the roofline numerator) and the clock/throttle summary taken
from nvidia-smi samples.  CPU only; nothing here launches a kernel."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

N128, NNZ128 = 128 ** 3, 14_581_760


@pytest.mark.parametrize("k,mb", [(1, 130.3), (2, 159.5), (3, 196.0)])
def test_gse_bytes_per_launch_128cube(k, mb):
    """nnz (4 B column + the live segments 2 / 4 / 6.5 B + 2/32 B group
    exponent) + 4 (n + 1) row pointers + 8 n for x read once + 8 n for y."""
    assert bench.algorithmic_bytes(NNZ128, N128, N128, k) / 1e6 == pytest.approx(mb, abs=0.05)


def test_baseline_and_table_bytes():
    assert bench.csr_bytes(NNZ128, N128, N128, 8) / 1e6 == pytest.approx(216.9, abs=0.05)   # FP64 CSR
    assert bench.csr_bytes(NNZ128, N128, N128, 4) / 1e6 == pytest.approx(158.6, abs=0.05)   # FP32 CSR
    # the table format has no per-group exponent: 2/32 B per nonzero less
    d = bench.algorithmic_bytes(NNZ128, N128, N128, 1) - bench.algorithmic_bytes(NNZ128, N128, N128, 1, G=0)
    assert d == pytest.approx(NNZ128 * 2 / 32)
    # the power-law matrix at 16.0M nonzeros, n = 10^6
    for k, mb in ((1, 117.0), (2, 149.0), (3, 189.0)):
        assert bench.algorithmic_bytes(16_000_000, 10 ** 6, 10 ** 6, k) / 1e6 == pytest.approx(mb, abs=0.05)


def _line(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", pcap="Not Active"):
    return f"0, {sm}, {mx}, 900.5, 0x0, {hw}, {hwt}, {swt}, {pcap}"


def test_clock_summary_median_max_and_reasons():
    c = bench.Clocks(0)
    c.lines = [_line(2070, 2070), _line(1965, 2070, pcap="Active"), _line(2070, 2070), "garbage",
               _line(1800, 2070, hwt="Active")]
    s = c.summary()
    assert s["sm_mhz"] == pytest.approx((1965 + 2070) / 2) and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"] and s["samples"] == 4


def test_clock_summary_without_samples():
    c = bench.Clocks(0)
    c.lines = []
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}


def test_peak_comes_from_the_measured_file_when_present():
    peak, kind = bench.load_peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        import json
        assert kind == "measured" and peak == json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    else:
        assert kind == "fallback"


def test_kernels_per_spmv_call():
    """The row schedule is one kernel; the nonzero split adds the split-row
    pass once the matrix spans more than one chunk of 256 * schedule nonzeros
    (the bench's kernel count in the timed region)."""
    assert bench.spmv_kernels_per_call(8, NNZ128) == 1
    assert bench.spmv_kernels_per_call(1, 16_140_000) == 2
    assert bench.spmv_kernels_per_call(4, 1024) == 1 and bench.spmv_kernels_per_call(4, 1025) == 2
    assert bench.spmv_kernels_per_call(1, 256) == 1


def test_iters_per_level_from_switch_iterations():
    assert bench.iters_per_level({"switch_iter": [0, 50, 80], "iters": 517}) == {"k1": 50, "k2": 30, "k3": 437}
    assert bench.iters_per_level({"switch_iter": [0, 3000, -1], "iters": 5000}) == {"k1": 3000, "k2": 2000}
    assert bench.iters_per_level({"switch_iter": [-1, -1, -1], "iters": 471}) == {}
