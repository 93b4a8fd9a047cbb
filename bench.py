"""Benchmark: time to relative KKT <= 1e-6 of rank-adaptive ALM-BM (ALORA) on the
MaxCut SDP of a 1000 x 1000 toroidal grid with Rademacher +-1 weights (n = 1e6,
2e6 edges, r0 = r_max = 32, sigma0 = 10, cold start y = 0), FP32 bulk / FP64 dual,
plus the HBM throughput of the two inner-step kernels (the fused step + gradient SpMM,
and the fused direction + line-search SDDMM) measured live inside the timed solves.

One step = one full solve (all hot-path kernels: constraint-map SDDMM, dual and
slack update, gradient SpMM, CG direction, line-search SDDMM with the exact
quartic step, Lanczos smallest eigenpair, rank growth test) on inputs resident in
HBM.  Beside it, in the same clock record: the plain FP64 solve of the same instance
(`fp64_cold`, median of --fp64-reps).  After it: the learned warm start on the same
torus (`warm_start`), the 4096-instance batch cold and warm (`batch`), the ER(800)
FP64 configuration with the oracle's own full solve (`config1`), and the oracle's
CPU baseline for the torus (`cpu_baseline`).

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference] [--no-fp64]

--impl reference times the FP64 CPU oracle on the host cores (a bounded sample of
the same workload, extrapolated to a full solve; see `cpu_baseline.sample`).
Multi-GPU: the path has no exchange step, so N ranks run N independent replicas
(one instance each), value = the slowest replica's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-6 rel KKT (s) + SDDMM/SpMM HBM GB/s; mixed+warm-start vs plain FP64"
WORKLOAD = ("maxcut-sdp torus 1000x1000 (n=1e6, |E|=2e6, weights +-1, seed 2), r0=32, r<=32, sigma0=10, y0=0, "
            "Lanczos started from the previous Ritz vector, "
            "PR+ CG with row-block Jacobi preconditioning, exact quartic line search")
N1, N2, SEED, R0, RMAX, EPS, SIGMA0 = 1000, 1000, 2, 32, 32, 1e-6, 10.0


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples (one CSV line every 200 ms); BENCH_CLOCKS_DIR overrides the directory
        out_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"alm_bench_clocks_rank{gpu_index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax = float(p[2])
                except ValueError:
                    continue
                for k, nm in enumerate(names):
                    if p[5 + k].lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# Other MaxCut workloads the solver can be timed on (not the default line): graphs shaped
# like the paper's DIMACS10 families at n = 2^20, and the two n = 1e7 graphs.
OTHER_WORKLOADS = {
    "rgg20": "maxcut-sdp random geometric graph n=2^20 (radius 0.55 sqrt(ln n / n)), unit weights",
    "delaunay20": "maxcut-sdp Delaunay triangulation of 2^20 uniform points, unit weights",
    "kron20": "maxcut-sdp Kronecker (R-MAT a,b,c = 0.57,0.19,0.19, edge factor 16) graph on 2^20 vertices",
    "regular3-1e7": "maxcut-sdp random 3-regular graph n=1e7, unit weights (seed 4), adaptive sigma rule",
    "torus-1e7": "maxcut-sdp torus 2500x4000 (n=1e7), weights +-1 (seed 5)",
}


def make_workload(name: str, seed: int):
    """(instance, description) of a named workload; "torus" is the benchmark's own."""
    import sdp_instances as si

    if name == "torus":
        return si.torus_maxcut(N1, N2, seed=seed), WORKLOAD
    suffix = (f", r0=32, r<=32, sigma0=10, y0=0, same solver options as the torus line (seed offset "
              f"{seed - SEED})")
    if name == "rgg20":
        return si.rgg_maxcut(1 << 20, seed=7 + seed - SEED), OTHER_WORKLOADS[name] + suffix
    if name == "delaunay20":
        return si.delaunay_maxcut(1 << 20, seed=8 + seed - SEED), OTHER_WORKLOADS[name] + suffix
    if name == "kron20":
        return si.kron_maxcut(20, seed=9 + seed - SEED), OTHER_WORKLOADS[name] + suffix
    if name == "regular3-1e7":
        return si.regular3_maxcut(10 ** 7, seed=4 + seed - SEED), OTHER_WORKLOADS[name] + suffix
    if name == "torus-1e7":
        return si.torus_maxcut(2500, 4000, seed=5 + seed - SEED, weights="pm1"), OTHER_WORKLOADS[name] + suffix
    raise ValueError(f"unknown workload {name}")


def max_over_ranks(value: float, world: int, device: str = "cpu") -> float:
    """The slowest replica's time (the job's time) over the ranks of the process group."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _flush_l2(torch, buf):
    buf.add_(1.0)  # 256 MiB write, larger than the 129 MB L2


def gpu_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import sdp_instances as si
    from paper_2505_15775_gb300 import alm

    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    seed = SEED + 1000 * rank                       # replicas: one instance per rank
    inst, workload = make_workload(args.workload, seed)
    R0 = si.factor_init(inst.n, R0_RANK, (seed, 7))
    opts = dict(eps=EPS, r_max=RMAX, sigma0=SIGMA0, profile=1, lanczos_warm=1)
    if args.workload == "regular3-1e7":
        # with sigma fixed the primal term stalls near 6e-4 (each inner solve at max_inner);
        # the adaptive rule doubles sigma when the primal term falls by less than 4x
        opts["sigma_rule"] = alm.ALM_SIGMA_ADAPTIVE
    h32 = alm.alm_create(inst, precision=alm.ALM_FP32, **opts)
    # launch shape of the two inner-step kernels: chosen by the autotuner on this instance
    # before anything is timed (32 inner steps per candidate shape)
    shape, tune, _ = alm.alm_autotune(h32, alm.factor_tensor(h32, R0), R0_RANK, None, steps=32)
    h64 = alm.alm_create(inst, precision=alm.ALM_FP64, **opts) if args.fp64 else None
    flush = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = h32.stream
    R0_dev = {alm.ALM_FP32: torch.as_tensor(R0, dtype=torch.float32, device="cuda"),
              alm.ALM_FP64: torch.as_tensor(R0, dtype=torch.float64, device="cuda")}  # resident before timing

    def solve(h, R_init=None, y_init=None):
        _flush_l2(torch, flush)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        R, r, y, st = alm.alm_solve(h, R0_dev[h.precision] if R_init is None else R_init, y_init)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, st

    for _ in range(args.warmup):
        solve(h32)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    times, stats = [], []
    fp64_runs = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            t, st = solve(h32)
            times.append(t)
            stats.append(st)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        step_s = statistics.mean(times)
        # plain FP64 cold start, same instance and options, inside the same clock record
        if h64 is not None:
            for _ in range(args.fp64_reps):
                fp64_runs.append(solve(h64))
    step_s = max_over_ranks(step_s, world, device="cuda")
    fp64 = None
    if fp64_runs:
        t64s = [t for t, _ in fp64_runs]
        st64 = fp64_runs[-1][1]
        fp64 = {"value": statistics.median(t64s), "all_s": t64s, "status": st64["status"], "outer": st64["outer"],
                "inner_total": st64["inner_total"], "rank": st64["rank"], "kkt": st64["kkt"],
                "objective": st64["objective"], "lanczos_matvecs": st64["lanczos_matvecs"],
                "speedup_of_fp32_form": statistics.median(t64s) / step_s}
    # e2e: through the public API from host buffers (create from host arrays, pinned R0 in, R and y out)
    R0_pinned = torch.from_numpy(np.ascontiguousarray(R0)).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = alm.alm_create(inst, precision=alm.ALM_FP32, **opts)
    alm.alm_set_inner_shape(h, **shape)
    R, r, y, st = alm.alm_solve(h, R0_pinned)
    Rh = R.cpu()
    yh = y.cpu()
    alm.alm_destroy(h)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h2d = sum(a.nbytes for a in (inst.c_i, inst.c_j, inst.c_v, inst.a_k, inst.a_i, inst.a_j, inst.a_v, inst.b)) \
        + R0_pinned.numel() * 8
    d2h = Rh.numel() * Rh.element_size() + yh.numel() * 8
    last = stats[-1]
    peak, peak_kind = _peaks()
    nl = max(1, last["spmm_launches"])
    step_ms = last["spmm_ms"] / nl
    spmm_gbs = last["spmm_bytes"] / (last["spmm_ms"] * 1e-3) / 1e9 if last["spmm_ms"] > 0 else None
    ls_ms = last["step_ms"][3] / nl
    ls_gbs = last["ls_bytes"] / (last["step_ms"][3] * 1e-3) / 1e9 if last["step_ms"][3] > 0 else None
    ncu_shape = shape == NCU_SHAPE and args.workload == "torus"
    roofline = {"bound": "hbm", "kernel": "k_spmm_step_pipe (R += alpha D, diag(S), G = 2 S R, preconditioner, "
                                          "CG inner products)",
                "achieved": spmm_gbs, "peak": peak, "unit": "GB/s",
                "frac": (spmm_gbs / peak) if spmm_gbs else None, "peak_kind": f"{peak_kind} (hbm_gbs)",
                "traffic": STEP_DRAM_BYTES_PER_LAUNCH if ncu_shape else None,
                "traffic_source": TRAFFIC_SOURCE if ncu_shape else None,
                "bytes_per_launch": last["spmm_bytes"] / nl, "avg_launch_ms": step_ms,
                "timed_launches": last["spmm_launches"], "rank_pad_last": last["spmm_rank_pad"]}
    roofline_sddmm = {"bound": "hbm", "kernel": "k_ls_dir_pipe (D = -Z + beta D_old, line-search SDDMM "
                                                "<S, D D^T> and A(R D^T), A(D D^T), FP64 quartic)",
                      "achieved": ls_gbs, "peak": peak, "unit": "GB/s",
                      "frac": (ls_gbs / peak) if ls_gbs else None, "peak_kind": f"{peak_kind} (hbm_gbs)",
                      "traffic": LS_DRAM_BYTES_PER_LAUNCH if ncu_shape else None,
                      "bytes_per_launch": last["ls_bytes"] / nl, "avg_launch_ms": ls_ms}
    clocks = clk.summary()
    out = {
        "metric": METRIC, "value": step_s, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "precision": "fp32-bulk/fp64-dual", "warm_start": False,
                   "eps": EPS, "l2": "flushed (256 MiB write) before each timed solve; R and S exceed L2 at r>=32",
                   "parallelism": "replicas" if world > 1 else "single", "inner_shape": shape},
        "solve": {"status": last["status"], "outer": last["outer"], "inner_total": last["inner_total"],
                  "rank": last["rank"], "kkt": last["kkt"], "objective": last["objective"],
                  "maxcut_value": -last["objective"], "lanczos_matvecs": last["lanczos_matvecs"],
                  "growth_steps": last["growth_steps"], "all_step_s": times},
        "fp64_cold": fp64,
        "autotune": {"chosen": shape, "candidates_ms_per_32_steps": [[s_, t_] for s_, t_ in tune]},
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "includes": "alm_create from host arrays + solve + R, y to host"},
        "roofline": roofline,
        "roofline_sddmm": roofline_sddmm,
        "gpu_launches": int(last["kernel_launches"]),
        "clocks": clocks,
    }
    if rank == 0 and not args.no_warm and args.workload == "torus":
        out["warm_start"] = torus_warm_leg(inst, R0, h32, solve, step_s)
    alm.alm_destroy(h32)
    if h64 is not None:
        alm.alm_destroy(h64)
    if rank == 0:
        if not args.no_batch:
            out["batch"] = batch_leg()
        if not args.no_config1:
            out["config1"] = config1_leg(args.no_cpu_baseline)
        if not args.no_cpu_baseline and args.workload == "torus":
            out["cpu_baseline"] = cpu_baseline(fp64 or {}, budget_s=args.cpu_budget)
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


# the inner shape the committed ncu capture of the two inner-step kernels used, and the DRAM
# bytes (read + write) per launch it measured on the torus at r = 32; the roofline lines
# carry them only when the bench ran the same shape
NCU_SHAPE = {"variant": 1, "stages": 2, "threads": 128}
STEP_DRAM_BYTES_PER_LAUNCH = 465.436416e6 + 246.724096e6
LS_DRAM_BYTES_PER_LAUNCH = 288.493824e6 + 105.090560e6
TRAFFIC_SOURCE = "ncu --set full of bench.py --case inner30 (dram__bytes_read.sum + dram__bytes_write.sum)"

TORUS_TRAIN = 24                      # warm-start training set: 48 x 48 tori, +-1 weights, seeds 1000..


def torus_warm_leg(inst, R0, h32, solve, cold_s):
    """Learned warm start on the benchmark torus: the network is trained on the solver's own
    solutions of 24 small tori of the same family (48 x 48, +-1 weights, seeds 1000..1023;
    never the benchmark instance), then predicts (R0, y0) for the 1e6-row torus (mixed with
    a seeded full-rank factor, mix = 1); the FP32 solve from that start is timed like the
    cold one.  Training is reported, not amortised into the solve time."""
    import torch

    import sdp_instances as si
    from paper_2505_15775_gb300 import alm, warm

    train = [si.torus_maxcut(48, 48, seed=1000 + k, weights="pm1") for k in range(TORUS_TRAIN)]
    g, rep = warm.train_warm_start(train, [si.factor_init(x.n, R0_RANK, (b, 7)) for b, x in enumerate(train)],
                                   lr=1e-3, eps=EPS, sigma0=SIGMA0, r_max=RMAX)
    hb = alm.alm_batch_create([inst], eps=EPS, sigma0=SIGMA0, r_max=RMAX)  # the network reads C through it
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(g.stream)
    Rw, rw, yw = alm.alm_gnn_warm_start(g, hb, mix=1.0)
    e1.record(g.stream)
    torch.cuda.synchronize()
    infer_s = e0.elapsed_time(e1) / 1e3
    runs = [solve(h32, Rw, yw) for _ in range(2)]
    t = statistics.median([x for x, _ in runs])
    st = runs[-1][1]
    alm.alm_gnn_destroy(g)
    alm.alm_batch_destroy(hb)
    return {"value": t + infer_s, "solve_s": t, "network_s": infer_s, "cold_s": cold_s,
            "ratio_to_cold": (t + infer_s) / cold_s, "status": st["status"], "outer": st["outer"],
            "inner_total": st["inner_total"], "kkt": st["kkt"], "objective": st["objective"],
            "training": rep, "train_set": f"{TORUS_TRAIN} tori 48x48, +-1 weights, seeds 1000..{1000 + TORUS_TRAIN - 1}"}


def config1_leg(skip_oracle: bool):
    """The small configuration: MaxCut SDP on ER(800, 0.06) (seed 1), plain FP64, r0 = 8,
    rank-adaptive, sigma0 = 1: GPU time to KKT <= 1e-6 (median of 3; the FP32-bulk form
    beside it), and the FP64 oracle's own full solve of the same instance on one host core
    (not extrapolated).  At n = 800 the solve is latency-bound and, in FP64, bound by this
    GPU's FP64 rate: most of it is the Lanczos eigensolves."""
    import torch

    import sdp_instances as si
    from paper_2505_15775_gb300 import alm

    inst = si.er_maxcut(800, 0.06, seed=1)
    R0 = si.factor_init(inst.n, 8, (1, 7))

    def timed(prec, growth_k=1):
        h = alm.alm_create(inst, precision=prec, eps=EPS, r_max=32, sigma0=1.0, lanczos_warm=1, growth_k=growth_k)
        ts, st = [], None
        for _ in range(4):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(h.stream)
            R, r, y, st = alm.alm_solve(h, R0)
            e1.record(h.stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        alm.alm_destroy(h)
        return statistics.median(ts[1:]), st

    t64, st = timed(alm.ALM_FP64)
    t32, st32 = timed(alm.ALM_FP32)
    t64b, stb = timed(alm.ALM_FP64, growth_k=4)
    out = {"workload": "maxcut-sdp ER(800, 0.06) seed 1, FP64, r0=8, sigma0=1 (Lanczos warm-started)",
           "gpu_s": t64, "status": st["status"], "outer": st["outer"], "inner_total": st["inner_total"],
           "rank": st["rank"], "kkt": st["kkt"], "objective": st["objective"],
           "lanczos_matvecs": st["lanczos_matvecs"],
           "fp32_form": {"gpu_s": t32, "status": st32["status"], "kkt": st32["kkt"], "objective": st32["objective"]},
           "block_growth": {"growth_k": 4, "gpu_s": t64b, "status": stb["status"], "outer": stb["outer"],
                            "growth_steps": stb["growth_steps"], "inner_total": stb["inner_total"],
                            "rank": stb["rank"], "kkt": stb["kkt"], "objective": stb["objective"],
                            "lanczos_matvecs": stb["lanczos_matvecs"]},
           "growth_steps": st["growth_steps"]}
    if not skip_oracle:
        code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import oracle as O, sdp_instances as si
inst = si.er_maxcut(800, 0.06, seed=1)
t = time.perf_counter()
P = O.OracleProblem(inst)
res = O.solve(P, si.factor_init(800, 8, (1, 7)), opts=O.SolveOptions(eps={EPS}, sigma=1.0, r_max=32))
print(json.dumps(dict(s=time.perf_counter() - t, objective=res.objective, kkt=[float(x) for x in res.kkt],
                      outer=res.outer, inner=res.inner_total, rank=int(res.R.shape[1]))))
"""
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
                   CUDA_VISIBLE_DEVICES="")
        rr = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
        if rr.returncode == 0:
            o = json.loads(rr.stdout.strip().splitlines()[-1])
            out["oracle"] = {"value": o["s"], "unit": "s", "cores": 1, "kind": "oracle", "objective": o["objective"],
                             "kkt": o["kkt"], "outer": o["outer"], "inner_total": o["inner"], "rank": o["rank"],
                             "sample": "full FP64 oracle solve of the same instance, one thread"}
            out["objective_rel_diff"] = abs(o["objective"] - st["objective"]) / abs(o["objective"])
        else:
            out["oracle"] = {"error": rr.stderr[-500:]}
    return out


R0_RANK = R0

BATCH_COUNT, BATCH_SEED, BATCH_TRAIN, BATCH_TRAIN_SEED = 4096, 6, 512, 1_000_000


def batch_work_rate(insts, per, device_s, s=4, ldr=32):
    """Work rate of the batched solve: inner steps and Lanczos products per second, and the
    bytes they move by the per-instance counts of the kernel (an inner step ~12 n_b ldr s
    from the factor-sized vectors plus 2 nnz_b (4 + s) for the two passes over the pattern;
    a Lanczos SpMV (nnz_b + n_b)(4 + s) + 4 (n_b + 1) + 2 n_b s, reorthogonalisation not
    counted) per second of the launch.  The instances' working sets stay in L1/L2, so this
    is a work rate for comparing runs, not a fraction of an HBM roofline."""
    import numpy as np

    steps = prods = 0
    nbytes = 0.0
    for x, p in zip(insts, per):
        n = int(x.n)
        e = int(np.count_nonzero(np.asarray(x.c_i) < np.asarray(x.c_j)))  # strict upper entries
        nnz = 2 * e
        nbytes += p["inner_total"] * (12.0 * n * ldr * s + 2.0 * nnz * (4 + s))
        nbytes += p["lanczos_matvecs"] * ((nnz + n) * (4.0 + s) + 4.0 * (n + 1) + 2.0 * n * s)
        steps += int(p["inner_total"])
        prods += int(p["lanczos_matvecs"])
    return {"inner_steps_per_s": steps / device_s, "lanczos_products_per_s": prods / device_s,
            "bytes_est": nbytes, "gbs_est": nbytes / device_s / 1e9,
            "bound": "L1/L2 and latency (per-instance working sets stay on chip): no HBM roofline"}


def batch_leg():
    """The 4096-instance batch of ER MaxCut SDPs (n ~ U{64..4096}, average degree ~ U[3,30],
    seed 6) in one persistent launch: cold start, and with the warm-start network trained
    on the solver's own solutions of 512 instances of the same generator (seeds >= 1e6).
    Times are CUDA-event times of the persistent launch (the inputs are resident)."""
    import numpy as np
    import torch

    import sdp_instances as si
    from paper_2505_15775_gb300 import alm, warm

    t0 = time.perf_counter()
    specs = si.batch_specs(BATCH_COUNT, seed=BATCH_SEED)
    insts = [si.er_maxcut(n, p, seed=sub) for n, p, sub in specs]
    opts = dict(eps=EPS, sigma0=SIGMA0, r_max=RMAX)
    hb = alm.alm_batch_create(insts, **opts)
    R0, rank0 = alm.batch_factor(hb, [si.factor_init(x.n, R0_RANK, (b, 7)) for b, x in enumerate(insts)])
    y0 = torch.zeros(hb.rows, dtype=torch.float64, device="cuda")
    t_setup = time.perf_counter() - t0
    threads, tune_ms = alm.alm_batch_autotune(hb, R0, rank0, y0)

    def run(handle, R, rank, y):
        stats, per = alm.alm_batch_solve(handle, R, rank, y)
        torch.cuda.synchronize()
        return {"device_s": stats["device_ms"] / 1e3, "converged": stats["converged"],
                "fell_back": int(sum(p["fell_back"] for p in per)),
                "inner_total": stats["inner_total"], "lanczos_matvecs": stats["lanczos_matvecs"],
                "outer_total": int(sum(p["outer"] for p in per)),
                "sum_instance_s": float(sum(p["device_ms"] for p in per)) / 1e3,
                "max_kkt": float(max(max(p["kkt"]) for p in per)),
                "objective_sum": float(sum(p["objective"] for p in per)),
                "work_rate": batch_work_rate(insts, per, stats["device_ms"] / 1e3)}

    cold = run(hb, R0.clone(), rank0.clone(), y0.clone())
    train = [si.er_maxcut(n, p, seed=sub) for n, p, sub in si.batch_specs(BATCH_TRAIN, seed=BATCH_TRAIN_SEED)]
    g, rep = warm.train_warm_start(train, [si.factor_init(x.n, R0_RANK, (b, 7)) for b, x in enumerate(train)],
                                   lr=1e-3, **opts)
    # the warm-started solve runs with the cold-start fallback (an instance that has taken
    # more than 2000 inner steps restarts once from a seeded cold start)
    hbw = alm.alm_batch_create(insts, fallback_inner=2000, **opts)
    alm.alm_batch_set_threads(hbw, threads)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(g.stream)
    Rw, rw, yw = alm.alm_gnn_warm_start(g, hbw, mix=1.0)
    e1.record(g.stream)
    torch.cuda.synchronize()
    infer_s = e0.elapsed_time(e1) / 1e3
    warm_res = run(hbw, Rw, rw, yw)
    warm_res["network_s"] = infer_s
    warm_res["device_plus_network_s"] = warm_res["device_s"] + infer_s
    alm.alm_gnn_destroy(g)
    alm.alm_batch_destroy(hbw)
    alm.alm_batch_destroy(hb)
    return {"workload": f"{BATCH_COUNT} ER MaxCut SDPs, n ~ U{{64..4096}}, d ~ U[3,30], seed {BATCH_SEED}; "
                        f"r0=32, sigma0=10, eps=1e-6, FP32 form, one persistent launch",
            "rows": int(sum(x.n for x in insts)), "threads": threads, "autotune_ms": tune_ms,
            "setup_s": t_setup, "cold": cold, "warm": warm_res, "training": rep,
            "kernel_launches_per_solve": 1}


# Tab. 2 of the paper (matrix completion, Sec. 6.2; A100, KKT <= 1e-5, context only):
# (rank, n) -> (seconds from the true rank, seconds from rank 1)
MC_PAPER_A100 = {(3, 10000): (0.379, 0.562), (3, 20000): (0.726, 1.040), (3, 50000): (1.409, 2.344),
                 (5, 10000): (0.504, 1.894), (5, 20000): (0.969, 3.349)}


def mc_leg(sizes=((3, 10000), (3, 20000), (3, 50000), (5, 10000))):
    """Matrix completion (Sec. 6.2, the nuclear-norm SDP) at Tab. 2's sizes: n1 = n2 = n/2,
    m = ceil(rank log(n) rank (n - rank)) observed entries (the paper's m for these n), M =
    U V^T Gaussian (seeded).  FP32-bulk form, eps = 1e-6, sigma0 = 1 with the adaptive rule,
    r_max = 32, from the true rank and from rank 1 (the paper's two columns); the paper's A100
    times (at KKT <= 1e-5) are quoted as context."""
    import torch

    import sdp_instances as si
    from paper_2505_15775_gb300 import alm

    rows = []
    for rank, n in sizes:
        inst = si.matrix_completion(n // 2, n // 2, rank, seed=(10, rank, n))
        h = alm.alm_create(inst, precision=alm.ALM_FP32, eps=EPS, sigma0=1.0, sigma_rule=alm.ALM_SIGMA_ADAPTIVE,
                           r_max=32, lanczos_warm=1)
        row = {"rank": rank, "n": n, "m": int(inst.m), "paper_a100_s": MC_PAPER_A100.get((rank, n))}
        for tag, r0 in (("from_true_rank", rank), ("from_rank_1", 1)):
            R0 = si.factor_init(inst.n, r0, (11, r0), scale=0.3)
            ts, st = [], None
            for _ in range(2):  # the first run also loads and captures
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(h.stream)
                _, _, _, st = alm.alm_solve(h, R0)
                e1.record(h.stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1) / 1e3)
            U, V, _ = inst.graph
            row[tag] = {"s": ts[-1], "status": st["status"], "outer": st["outer"], "inner_total": st["inner_total"],
                        "rank": st["rank"], "kkt": st["kkt"], "objective": st["objective"]}
        alm.alm_destroy(h)
        rows.append(row)
    return {"workload": "matrix completion, Tab. 2 sizes (n1 = n2 = n/2), FP32 form, eps=1e-6", "rows": rows}


def _oracle_sample(budget_s, rank_hint):
    """Time the FP64 oracle on the full-size instance: inner CG steps (gradient,
    preconditioner, direction, quartic coefficients, exact step) for about 0.7 of budget_s,
    and the oracle's own Lanczos (lanczos_min, one cycle of 32 products with CGS2
    reorthogonalisation) on the slack matrix.  Runs in a fresh single-threaded process."""
    code = f"""
import json, os, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
import oracle as O, sdp_instances as si
inst = si.torus_maxcut({N1}, {N2}, seed={SEED})
t0 = time.perf_counter()
P = O.OracleProblem(inst)
t_setup = time.perf_counter() - t0
r = {int(rank_hint)}
R = si.factor_init(inst.n, r, ({SEED}, 7))
y = np.zeros(inst.m)
budget = {float(budget_s)}
steps, t_in = 0, 0.0
Gp = Zp = Dp = None
while t_in < 0.7 * budget or steps < 2:
    t = time.perf_counter()
    G = O.gradient(P, R, y, {SIGMA0})
    Z = O.precondition(P, R, y, {SIGMA0}, G)
    D = -Z if Gp is None else -Z + max(0.0, (float(np.sum(Z * G)) - float(np.sum(G * Zp))) / float(np.sum(Zp * Gp))) * Dp
    a = O.exact_step(O.quartic_coeffs(P, R, D, y, {SIGMA0}))
    R = R + a * D
    Gp, Zp, Dp = G, Z, D
    t_in += time.perf_counter() - t
    steps += 1
S = O.slack_sparse(P, O.dual_candidate(P, R, y, {SIGMA0}))
t = time.perf_counter()
theta, v, res, nmv = O.lanczos_min(lambda x: O.slack_matvec(P, S, x), inst.n, k=32, max_restarts=1, seed=0)
t_lz = time.perf_counter() - t
print(json.dumps(dict(inner_s=t_in / steps, inner_steps=steps, lz_product_s=t_lz / nmv, lz_products=nmv,
                      setup_s=t_setup, rank=r)))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def fp64_counts(fp64: dict | None) -> dict:
    """Inner CG steps, Lanczos products and final rank of the plain FP64 solve of the
    benchmark instance: the same iteration the oracle runs (a deterministic function of the
    seeded instance), taken from a GPU FP64 solve; the committed record of that solve when
    no GPU solve ran in this process."""
    if fp64 and fp64.get("inner_total"):
        return {"inner_total": fp64["inner_total"], "lanczos_matvecs": fp64["lanczos_matvecs"],
                "rank": fp64["rank"], "source": "FP64 GPU solve of this run"}
    return dict(FP64_RECORD, source="committed record of an FP64 GPU solve of this instance")


def cpu_baseline(fp64: dict | None, budget_s=20.0):
    counts = fp64_counts(fp64)
    inner, mvs, rank = counts["inner_total"], counts["lanczos_matvecs"], counts["rank"]
    s = _oracle_sample(budget_s, rank)
    est = s["setup_s"] + inner * s["inner_s"] + mvs * s["lz_product_s"]
    return {"value": est, "unit": "s", "cores": 1, "kind": "oracle",
            "sample": (f"FP64 numpy/scipy oracle, 1 thread, full n=1e6 instance: {s['inner_steps']} inner CG steps "
                       f"at r={s['rank']} ({s['inner_s']:.3f} s each) and one cycle of its own lanczos_min "
                       f"({s['lz_products']} products with CGS2, {s['lz_product_s']:.4f} s each), extrapolated to "
                       f"the {inner} inner steps and {mvs} Lanczos products of the plain FP64 solve "
                       f"({counts['source']}; that solve skips eigensolves that cannot change the outcome, so the "
                       f"oracle, which computes one every outer iteration, would need more), plus setup "
                       f"{s['setup_s']:.1f} s"),
            "per_inner_step_s": s["inner_s"], "per_lanczos_product_s": s["lz_product_s"], "counts": counts}


def reference_arm(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    if args.workload != "torus":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle's CPU baseline is sampled on the torus "
                                                            "workload only"}))
        return
    # the iteration counts: from the plain FP64 GPU solve of the same instance, as in the
    # repo arm (one set of counts for both arms)
    fp64 = None
    try:
        import torch

        if torch.cuda.is_available():
            import sdp_instances as si
            from paper_2505_15775_gb300 import alm

            inst, _ = make_workload("torus", SEED)
            h64 = alm.alm_create(inst, precision=alm.ALM_FP64, eps=EPS, r_max=RMAX, sigma0=SIGMA0,
                                 lanczos_warm=1)
            _, _, _, st = alm.alm_solve(h64, si.factor_init(inst.n, R0_RANK, (SEED, 7)))
            torch.cuda.synchronize()
            alm.alm_destroy(h64)
            fp64 = {"inner_total": st["inner_total"], "lanczos_matvecs": st["lanczos_matvecs"], "rank": st["rank"]}
    except Exception:
        fp64 = None
    vals, last = [], None
    budget = max(5.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for i in range(args.warmup + args.steps):
        b = cpu_baseline(fp64, budget_s=budget)
        if i >= args.warmup:
            vals.append(b["value"])
            last = b
    v = statistics.mean(vals)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "precision": "fp64 (CPU oracle)"},
           "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": last["sample"], "value": v, "unit": "s"},
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# Plain FP64 solve of the benchmark instance (same options) recorded on a GB300: used for the
# oracle's iteration counts only when no GPU solve runs in the process.
FP64_RECORD = {"inner_total": 23284, "lanczos_matvecs": 1153, "rank": 32}


def profile_case(args):
    """Short runs for ncu.  inner30: one outer iteration of the bench workload capped at 30
    inner steps (FP32, r = 32, kernels launched one by one, the default inner shape:
    variant 1, 2 stages, 128 threads) and one Lanczos cycle.  batch64:
    the first 64 instances of the 4096-instance generator in one persistent launch."""
    import torch

    import sdp_instances as si
    from paper_2505_15775_gb300 import alm

    if args.case == "batch64":
        insts = [si.er_maxcut(n, p, seed=sub) for n, p, sub in si.batch_specs(BATCH_COUNT, seed=BATCH_SEED)[:64]]
        hb = alm.alm_batch_create(insts, eps=EPS, sigma0=SIGMA0, r_max=RMAX)
        R, rank = alm.batch_factor(hb, [si.factor_init(x.n, R0_RANK, (b, 7)) for b, x in enumerate(insts)])
        y = torch.zeros(hb.rows, dtype=torch.float64, device="cuda")
        stats, per = alm.alm_batch_solve(hb, R, rank, y)
        torch.cuda.synchronize()
        alm.alm_batch_destroy(hb)
        print(json.dumps({"case": args.case, "rows": int(sum(x.n for x in insts)), **stats}))
        return

    inst = si.torus_maxcut(N1, N2, seed=SEED)
    h = alm.alm_create(inst, precision=alm.ALM_FP32, eps=EPS, r_max=RMAX, sigma0=SIGMA0, max_outer=1, max_inner=30,
                       use_graph=0, lanczos_max_restarts=1)
    R, r, y, st = alm.alm_solve(h, si.factor_init(inst.n, R0_RANK, (SEED, 7)))
    torch.cuda.synchronize()
    alm.alm_destroy(h)
    print(json.dumps({"case": args.case, "inner": st["inner_total"], "kernel_launches": st["kernel_launches"]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64", action="store_true", default=True,
                    help="also time the plain FP64 cold-start solve (the default; --no-fp64 skips it)")
    ap.add_argument("--no-fp64", dest="fp64", action="store_false")
    ap.add_argument("--case", default=None, choices=["inner30", "batch64"],
                    help="small profiling case: inner30 (30 inner steps of the bench workload, no graphs) or "
                         "batch64 (64 instances of the batch generator, one persistent launch)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 4096-instance batch (config 5) leg")
    ap.add_argument("--no-warm", action="store_true", help="skip the learned warm start on the torus")
    ap.add_argument("--no-config1", action="store_true", help="skip the ER(800) FP64 leg and its oracle solve")
    ap.add_argument("--fp64-reps", type=int, default=3, help="timed plain FP64 solves (inside the clock record)")
    ap.add_argument("--mc", action="store_true", help="only the matrix-completion leg (Tab. 2 sizes); one JSON line")
    ap.add_argument("--workload", default="torus", choices=["torus", *OTHER_WORKLOADS],
                    help="the MaxCut instance of the timed solve (default: the 1000x1000 torus)")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    args = ap.parse_args()
    if args.mc:
        print(json.dumps({"mc": mc_leg()}))
    elif args.case:
        profile_case(args)
    elif args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
