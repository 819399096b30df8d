"""Host-side logic of bench.py (no GPU): parsing of the nvidia-smi clock
samples and the choice of the samples inside the timed region, and the DRAM
traffic taken from the committed ncu summary only while the march source
matches the one it was captured on."""
import os

import bench


def _csv(tmp_path, lines):
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(lines) + "\n")
    return str(p)


def test_clock_rows_and_window(tmp_path):
    lines = [
        "2026/12/03 10:00:00.000, 0, 1980, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2026/12/03 10:00:00.100, 0, 2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2026/12/03 10:00:00.200, 0, 2070, 2070, 1200.0, 0x4, Not Active, Not Active, Not Active, Active",
        "2026/12/03 10:00:00.300, 0, 2055, 2070, 1300.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "2026/12/03 10:00:00.400, 0, [N/A], 2070, 1300.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    rows = bench._parse_clock_rows(_csv(tmp_path, lines))
    assert len(rows) == 4
    t0 = rows[1][0]
    s = bench.clock_summary(rows, (t0 - 1e-3, rows[3][0] + 1e-3))
    assert s["span"] == "timed region" and s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    # a window with fewer than three samples falls back to all of them
    s2 = bench.clock_summary(rows, (t0, t0))
    assert s2["samples"] == 4 and s2["span"].startswith("whole benchmark")
    assert bench.clock_summary([], (0, 1)) is None


def test_traffic_only_for_the_captured_source(tmp_path):
    h = bench.march_source_hash()
    assert len(h) == 16 and h == bench.march_source_hash()
    good = tmp_path / "good.md"
    good.write_text("x\n" f"march source sha256/16: `{h}`\n" "dram bytes per launch: 123456 (mean)\n")
    assert bench.march_traffic(str(good)) == 123456.0
    stale = tmp_path / "stale.md"
    stale.write_text("march source sha256/16: `0000000000000000`\ndram bytes per launch: 99\n")
    assert bench.march_traffic(str(stale)) is None
    assert bench.march_traffic(str(tmp_path / "missing.md")) is None
