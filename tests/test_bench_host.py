"""Host-side pieces of bench.py checked on the CPU: the clock record taken during the timed
region, and the DRAM traffic that the roofline object quotes from the committed ncu summary."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_summary_takes_the_median_and_the_active_reasons():
    bench = _bench()
    cs = bench.ClockSampler(0)
    cs.out = "\n".join([
        "2070, 2070, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1965, 2070, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "[N/A], 2070, 0x0, Not Active, Not Active, Not Active, Not Active",     # skipped
        "garbage",
    ])
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    cs.out = "2000, 2070, 0x0, Active, Not Active, Not Active, Not Active\n"
    assert cs.summary()["reasons"] == ["hw_slowdown"]
    cs.out = ""
    assert cs.summary()["reasons"] == ["unavailable"] and cs.summary()["samples"] == 0


def test_committed_traffic_of_the_roofline_kernel_is_its_algorithmic_bytes():
    """The A^T(y) pass reads the m n(n+1)/2 integer-digit copy of A once: 2000 * 20100 * 8 bytes
    = 321.6 MB per launch.  The ncu summary it quotes must be within 1% of that (no re-reads)."""
    bench = _bench()
    t = bench.read_traffic()
    algorithmic = 2000 * (200 * 201 // 2) * 8
    assert t is not None and abs(t - algorithmic) <= 0.01 * algorithmic
    assert bench.read_traffic("does_not_exist.txt") is None
