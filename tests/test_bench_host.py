"""Host logic of bench.py that needs no GPU: the clock record taken during the timed region
(the field a run is accepted or rejected on) and the iteration counts that scale the
oracle's sampled per-step costs."""
import os

import bench


class _Running:  # stands for the nvidia-smi process of a sampler that started
    pass


def _sampler(tmp_path, lines):
    os.environ["BENCH_CLOCKS_DIR"] = str(tmp_path)
    try:
        cs = bench.ClockSampler(0)
    finally:
        del os.environ["BENCH_CLOCKS_DIR"]
    with open(cs.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    cs.proc = _Running()
    return cs


def test_clock_summary_median_max_and_reasons(tmp_path):
    row = "0, {sm}, 2070, 900.5, 0x0, {hw}, Not Active, Not Active, {pc}"
    lines = [row.format(sm=s, hw="Not Active", pc="Not Active") for s in (2070, 2055, 2070, 1980, 2070)]
    lines.append(row.format(sm=2070, hw="Not Active", pc="Active"))
    lines.append("garbage line")
    lines.append("0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active")
    s = _sampler(tmp_path, lines).summary()
    assert s["samples"] == 6 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    lines.append(row.format(sm=1200, hw="Active", pc="Not Active"))
    s = _sampler(tmp_path, lines).summary()
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_summary_without_nvidia_smi(tmp_path):
    s = bench.ClockSampler(0)
    s.proc = None
    assert s.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_fp64_counts_prefer_the_solve_of_this_run():
    c = bench.fp64_counts({"inner_total": 123, "lanczos_matvecs": 45, "rank": 7})
    assert (c["inner_total"], c["lanczos_matvecs"], c["rank"]) == (123, 45, 7)
    assert c["source"] == "FP64 GPU solve of this run"
    c = bench.fp64_counts(None)
    assert c["inner_total"] == bench.FP64_RECORD["inner_total"] and "committed record" in c["source"]
