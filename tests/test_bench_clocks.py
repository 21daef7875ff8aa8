"""The bench's summary of the clocks sampled during the timed steps
(bench._clock_summary): median SM clock, maximum, and the throttle reasons
seen, parsed from records in the format nvidia-smi writes (no GPU needed)."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _write(tmp_path, lines):
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(lines) + "\n")
    return str(p)


def test_clock_summary_quiet_run(tmp_path):
    b = _bench()
    rec = "0, 2070, 2070, 189.84, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    s = b._clock_summary(_write(tmp_path, [rec, rec.replace("2070, 2070", "2055, 2070"), rec]))
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == [] and s["samples"] == 3


def test_clock_summary_reports_throttle_reasons(tmp_path):
    b = _bench()
    lines = ["0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "0, 1650, 2070, 1400.0, 0x0000000000000008, Active, Not Active, Not Active, Active",
             "garbage line", "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = b._clock_summary(_write(tmp_path, lines))
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert s["samples"] == 2 and s["sm_mhz"] == 1815.0


def test_clock_summary_without_records(tmp_path):
    b = _bench()
    s = b._clock_summary(str(tmp_path / "missing.csv"))
    assert s["reasons"] == ["unavailable"] and s["sm_mhz"] is None
