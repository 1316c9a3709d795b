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
        "2026/12/04 10:00:00.000, 2070, 2070, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2026/12/04 10:00:00.050, 1965, 2070, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2026/12/04 10:00:00.100, 2070, 2070, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2026/12/04 10:00:00.150, [N/A], 2070, 0x0, Not Active, Not Active, Not Active, Not Active",   # skipped
        "garbage",
    ])
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"] and s["window"] == "sampler span"
    cs.out = "2026/12/04 10:00:00.000, 2000, 2070, 0x0, Active, Not Active, Not Active, Not Active\n"
    assert cs.summary()["reasons"] == ["hw_slowdown"]
    cs.out = ""
    assert cs.summary()["reasons"] == ["unavailable"] and cs.summary()["samples"] == 0


def test_clock_summary_keeps_the_samples_of_the_timed_window():
    """Only the samples stamped inside the timed steps (one interval of slack) count; a
    throttle reason seen before the window does not, and with no sample inside the window the
    whole span is reported and says so."""
    import datetime
    bench = _bench()
    cs = bench.ClockSampler(0, interval_ms=50)
    cs.used_ms = 50
    base = datetime.datetime(2026, 12, 4, 10, 0, 0)
    rows = []
    for k in range(20):                                   # one sample every 50 ms over 1 s
        t = base + datetime.timedelta(milliseconds=50 * k)
        sm, thermal = (1500, "Active") if k < 5 else (2070, "Not Active")
        rows.append(f"{t.strftime('%Y/%m/%d %H:%M:%S.%f')[:-3]}, {sm}, 2070, 0x0, Not Active, {thermal}, Not Active, Not Active")
    cs.out = "\n".join(rows)
    t0 = (base + datetime.timedelta(milliseconds=410)).timestamp()
    t1 = (base + datetime.timedelta(milliseconds=690)).timestamp()
    s = cs.summary(window=(t0, t1))
    assert s["window"] == "timed steps" and s["samples"] == 7          # 400 .. 700 ms
    assert s["sm_mhz"] == 2070.0 and s["reasons"] == []
    whole = cs.summary()
    assert whole["samples"] == 20 and whole["reasons"] == ["hw_thermal_slowdown"]
    late = (base + datetime.timedelta(seconds=5)).timestamp()
    s = cs.summary(window=(late, late + 0.1))
    assert s["samples"] == 20 and s["window"].startswith("sampler span (no sample")


FAKE_SMI = """#!/usr/bin/env python3
import datetime, sys, time
ms = int(sys.argv[sys.argv.index("-lms") + 1])
if ms < {min_ms}:
    sys.exit(2)                      # an interval this tool refuses
for _ in range(1000):
    now = datetime.datetime.now().strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    print(now + ", 2070, 2070, 0x0, Not Active, Not Active, Not Active, Not Active", flush=True)
    time.sleep(ms / 1000.0)
"""


def _fake_smi(tmp_path, min_ms):
    p = tmp_path / "fake-smi"
    p.write_text(FAKE_SMI.replace("{min_ms}", str(min_ms)))
    p.chmod(0o755)
    return str(p)


def test_clock_sampler_samples_during_the_region_and_falls_back_to_200_ms(tmp_path):
    import time
    bench = _bench()
    with bench.ClockSampler(0, interval_ms=50, cmd=_fake_smi(tmp_path, 0)) as cs:
        assert cs.lines, "the first sample arrives before the region starts"
        t0 = time.time()
        time.sleep(0.5)
        t1 = time.time()
    s = cs.summary(window=(t0, t1))
    assert s["window"] == "timed steps" and s["interval_ms"] == 50 and 8 <= s["samples"] <= 13
    assert s["sm_mhz"] == 2070.0 and s["reasons"] == []
    # a tool that refuses 50 ms: restarted at 200 ms
    with bench.ClockSampler(0, interval_ms=50, cmd=_fake_smi(tmp_path, 100)) as cs:
        time.sleep(0.45)
    s = cs.summary()
    assert s["interval_ms"] == 200 and 2 <= s["samples"] <= 4
    # no such tool: unavailable, and the region still runs
    with bench.ClockSampler(0, cmd=str(tmp_path / "missing")) as cs:
        pass
    assert cs.summary()["reasons"] == ["unavailable"]


def test_committed_traffic_of_the_roofline_kernel_is_its_algorithmic_bytes():
    """The A^T(y) pass reads the m n(n+1)/2 integer-digit copy of A once: 2000 * 20100 * 8 bytes
    = 321.6 MB per launch.  The ncu summary it quotes must be within 1% of that (no re-reads)."""
    bench = _bench()
    t = bench.read_traffic()
    algorithmic = 2000 * (200 * 201 // 2) * 8
    assert t is not None and abs(t - algorithmic) <= 0.01 * algorithmic
    assert bench.read_traffic("does_not_exist.txt") is None
