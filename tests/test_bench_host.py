"""Host logic of bench.py that decides what a benchmark line reports, on CPU.

- The clock record: nvidia-smi rows sampled during the timed region reduce to the median SM clock
  under load (power above 200 W; all rows when none is), the maximum clock, and the throttle
  reasons seen Active in any row (what makes a run rejected or noted).
- The DRAM traffic lookup: a committed ncu figure is used only while the kernel source it was
  captured on is unchanged (its SHA-256 prefix matches), and only for its own workload.
"""
import hashlib
import importlib.util
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load_bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _DoneProc:
    """Stands in for the nvidia-smi process: already finished."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _clocks_from(bench, tmp_path, lines):
    c = bench.Clocks(None, enabled=False)
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(lines) + "\n")
    c.proc, c.path = _DoneProc(), str(path)
    return c.stop()


def test_clock_record_median_under_load_and_reasons(tmp_path):
    bench = _load_bench()
    idle = "0, 345, 2070, 95.10, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    busy = [f"0, {mhz}, 2070, {w}, 0x0000000000000004, Not Active, Not Active, Not Active, {cap}"
            for mhz, w, cap in [(1980, 900.5, "Not Active"), (2010, 1010.0, "Active"), (1995, 950.2, "Not Active"),
                                (2040, 870.0, "Not Active")]]
    rec = _clocks_from(bench, tmp_path, [idle] + busy + [idle, "garbage line", ""])
    assert rec["samples"] == 6
    assert rec["sm_mhz"] == 2002.5  # median of the four rows under load; the idle rows are left out
    assert rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(tmp_path / "clocks.csv")


def test_clock_record_flags_thermal_slowdown_and_handles_missing_power(tmp_path):
    bench = _load_bench()
    rows = ["0, 1500, 2070, [N/A], 0x0000000000000040, Not Active, Active, Not Active, Not Active",
            "0, 1600, 2070, [N/A], 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"]
    rec = _clocks_from(bench, tmp_path, rows)
    assert rec["sm_mhz"] == 1550.0  # no row above 200 W: the median of all rows
    assert rec["reasons"] == ["hw_thermal_slowdown"]


def test_clock_record_empty_is_none(tmp_path):
    bench = _load_bench()
    assert _clocks_from(bench, tmp_path, ["not, a, clock, row"]) is None


def test_traffic_only_for_the_source_it_was_captured_on():
    bench = _load_bench()
    table = open(os.path.join(ROOT, "profiles", "dram_traffic.md")).read()
    rows = re.findall(r"^\|\s*`?([\w@/]+)`?\s*\|\s*([0-9.eE+]+)\s*\|\s*([0-9a-f]{16})\s*\|", table, re.M)
    assert rows, "the traffic table has no keyed rows"
    for key, value, sha in rows:
        workload, kernel_class = key.split("/")[0], key.split("/")[1].split("@")[0]
        level = int(key.split("@")[1]) if "@" in key else None
        src = os.path.join(ROOT, "paper_2102_07417_gb300", "csrc",
                           bench.KERNEL_SOURCE.get(kernel_class, "solve.cu"))
        current = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        got = bench.traffic_for(workload, kernel_class, level)
        if current == sha:
            assert got == float(value)
        else:
            assert got is None
        assert bench.traffic_for(workload + "_other", kernel_class, level) is None
