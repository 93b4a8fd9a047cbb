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


def test_batch_work_rate_counts_per_instance():
    class Inst:
        def __init__(self, n, ci, cj):
            self.n, self.c_i, self.c_j = n, ci, cj

    # a triangle (3 strict-upper entries plus the diagonal) and a 2-path (1 plus diagonal)
    insts = [Inst(3, [0, 0, 1, 0, 1, 2], [1, 2, 2, 0, 1, 2]), Inst(2, [0, 0, 1], [1, 0, 1])]
    per = [{"inner_total": 10, "lanczos_matvecs": 4}, {"inner_total": 5, "lanczos_matvecs": 2}]
    w = bench.batch_work_rate(insts, per, 2.0)
    step = lambda n, e: 12 * n * 32 * 4 + 2 * (2 * e) * 8
    prod = lambda n, e: (2 * e + n) * 8 + 4 * (n + 1) + 2 * n * 4
    want = 10 * step(3, 3) + 4 * prod(3, 3) + 5 * step(2, 1) + 2 * prod(2, 1)
    assert w["bytes_est"] == want
    assert w["inner_steps_per_s"] == 7.5 and w["lanczos_products_per_s"] == 3.0
    assert w["gbs_est"] == want / 2.0 / 1e9
