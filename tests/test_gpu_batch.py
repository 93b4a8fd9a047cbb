"""The batched persistent solver (alm_batch_*) against closed-form MaxCut SDP values,
the FP64 oracle's solves and the single-instance solver: every instance of a ragged
batch (1 to a few hundred rows, degree 0 to 30, instances with no edges) converges,
reaches the oracle's objective within 1e-6 relative, and its (R, y) passes the oracle's
relative KKT check (dense eigendecomposition) at 1e-6."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import sdp_instances as si  # noqa: E402
from gpu_common import as_np  # noqa: E402

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2505_15775_gb300 import alm  # noqa: E402

EPS = 5e-7
R0 = 32
SIGMA0 = 10.0


def _closed_form_instances():
    """(instance, MaxCut SDP value) pairs with known values."""
    out = []
    for n in (9, 12):
        out.append((si.maxcut(n, *si.complete_edges(n), np.ones(n * (n - 1) // 2)), n * n / 4))
    for n in (10, 9, 31):
        expect = float(n) if n % 2 == 0 else n / 2 * (1 + math.cos(math.pi / n))
        out.append((si.maxcut(n, *si.cycle_edges(n), np.ones(n)), expect))
    z = np.zeros(0, np.int64)
    out.append((si.maxcut(1, z, z, np.zeros(0)), 0.0))             # one vertex
    out.append((si.maxcut(6, z, z, np.zeros(0)), 0.0))             # no edges
    out.append((si.maxcut(2, np.array([0]), np.array([1]), np.ones(1)), 1.0))
    return out


def _random_instances(count, n_hi, seed=60):
    return [si.er_maxcut(n, p, seed=sub) for n, p, sub in si.batch_specs(count, seed=seed, n_lo=16, n_hi=n_hi)]


def _solve_batch(instances, threads=None, **opt):
    hb = alm.alm_batch_create(instances, eps=EPS, sigma0=SIGMA0, **opt)
    try:
        if threads:
            alm.alm_batch_set_threads(hb, threads)
        R, rank = alm.batch_factor(hb, [si.factor_init(x.n, R0, (b, 7)) for b, x in enumerate(instances)])
        y = torch.zeros(hb.rows, dtype=torch.float64, device="cuda")
        stats, per = alm.alm_batch_solve(hb, R, rank, y)
        torch.cuda.synchronize()
        return hb.row_off.copy(), as_np(R), rank.cpu().numpy(), as_np(y), stats, per
    finally:
        alm.alm_batch_destroy(hb)


def _slice(row_off, R, rank, y, b):
    s, e = int(row_off[b]), int(row_off[b + 1])
    return R[s:e, : int(rank[b])], y[s:e]


def _oracle_kkt(inst, Rb, yb):
    P = O.OracleProblem(inst)
    lam = float(np.linalg.eigvalsh(O.slack_dense(P, yb))[0])
    return P, O.kkt(P, Rb, yb, lam)


def test_batch_closed_forms():
    cases = _closed_form_instances()
    insts = [c[0] for c in cases]
    row_off, R, rank, y, stats, per = _solve_batch(insts)
    assert stats["converged"] == len(insts), per
    assert stats["kernel_launches"] == 1
    for b, (inst, value) in enumerate(cases):
        assert per[b]["status"] == 0, (b, per[b])
        assert -per[b]["objective"] == pytest.approx(value, rel=1e-6, abs=1e-9), (b, per[b])
        Rb, yb = _slice(row_off, R, rank, y, b)
        assert np.all(R[int(row_off[b]):int(row_off[b + 1]), int(rank[b]):] == 0.0)
        P, k = _oracle_kkt(inst, Rb, yb)
        assert max(k) <= 1e-6, (b, k)
        assert -O.cost(P, Rb) == pytest.approx(value, rel=1e-6, abs=1e-9)


def test_batch_matches_oracle_solves():
    """A ragged ER batch (n 16..300, average degree 3..30, seeded like the 4096-instance
    workload): the same objective as the oracle's own solve within 1e-6 relative, and the
    oracle's KKT of the GPU's (R, y) within 1e-6."""
    insts = _random_instances(24, 300)
    row_off, R, rank, y, stats, per = _solve_batch(insts)
    assert stats["converged"] == len(insts), [p["status"] for p in per]
    for b, inst in enumerate(insts):
        Rb, yb = _slice(row_off, R, rank, y, b)
        P, k = _oracle_kkt(inst, Rb, yb)
        assert max(k) <= 1e-6, (b, k, per[b])
        ref = O.solve(P, si.factor_init(inst.n, R0, (b, 7)),
                      opts=O.SolveOptions(eps=1e-7, sigma=SIGMA0, r_max=32))
        assert max(ref.kkt) <= 1e-7
        assert per[b]["objective"] == pytest.approx(ref.objective, rel=1e-6), (b, per[b], ref.objective)
        assert O.cost(P, Rb) == pytest.approx(ref.objective, rel=1e-6)


def test_batch_matches_single_instance_solver():
    """The batch and alm_solve (FP32 form, same options and R0) reach the same objective."""
    insts = _random_instances(6, 400, seed=61)
    row_off, R, rank, y, stats, per = _solve_batch(insts)
    for b, inst in enumerate(insts):
        h = alm.alm_create(inst, precision=alm.ALM_FP32, eps=EPS, sigma0=SIGMA0)
        try:
            _, _, _, st = alm.alm_solve(h, si.factor_init(inst.n, R0, (b, 7)))
        finally:
            alm.alm_destroy(h)
        assert st["status"] == 0 and per[b]["status"] == 0
        assert per[b]["objective"] == pytest.approx(st["objective"], rel=1e-6)


@pytest.mark.parametrize("threads", [256, 1024])
def test_batch_block_sizes_and_determinism(threads):
    """Each CTA size converges to the same objectives; at a fixed CTA size two runs give
    bit-identical factors (no result depends on which CTA took an instance)."""
    insts = _random_instances(40, 200, seed=62)
    a = _solve_batch(insts, threads=threads)
    b = _solve_batch(insts, threads=threads)
    ref = _solve_batch(insts, threads=512)
    assert a[4]["threads"] == threads
    assert a[4]["converged"] == len(insts)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[3], b[3])
    for k in range(len(insts)):
        assert a[5][k]["objective"] == pytest.approx(ref[5][k]["objective"], rel=1e-6)


def test_batch_autotune_leaves_inputs_unchanged():
    insts = _random_instances(64, 300, seed=63)
    hb = alm.alm_batch_create(insts, eps=EPS, sigma0=SIGMA0)
    try:
        R, rank = alm.batch_factor(hb, [si.factor_init(x.n, R0, (b, 7)) for b, x in enumerate(insts)])
        y = torch.zeros(hb.rows, dtype=torch.float64, device="cuda")
        R0c, r0c, y0c = R.clone(), rank.clone(), y.clone()
        t, times = alm.alm_batch_autotune(hb, R, rank, y)
        torch.cuda.synchronize()
        assert t in (256, 512, 1024)
        assert all(math.isfinite(v) and v > 0 for v in times.values())
        assert torch.equal(R, R0c) and torch.equal(rank, r0c) and torch.equal(y, y0c)
        stats, per = alm.alm_batch_solve(hb, R, rank, y)
        assert stats["threads"] == t and stats["converged"] == len(insts)
    finally:
        alm.alm_batch_destroy(hb)


def test_batch_solve_after_autotune_reuses_no_stale_graph():
    """solve -> autotune -> solve on the same tensors at the same CTA size: the autotuner
    grows the per-CTA scratch, and the second solve must not replay a graph that still
    points at the freed scratch (its result equals the first solve's, bit for bit)."""
    insts = _random_instances(200, 64, seed=64)
    hb = alm.alm_batch_create(insts, eps=EPS, sigma0=SIGMA0)
    try:
        alm.alm_batch_set_threads(hb, 1024)
        R, rank = alm.batch_factor(hb, [si.factor_init(x.n, R0, (b, 7)) for b, x in enumerate(insts)])
        y = torch.zeros(hb.rows, dtype=torch.float64, device="cuda")
        R0c, r0c, y0c = R.clone(), rank.clone(), y.clone()
        st1, per1 = alm.alm_batch_solve(hb, R, rank, y)
        R1, y1 = R.clone(), y.clone()
        alm.alm_batch_autotune(hb, R0c, r0c, y0c)
        alm.alm_batch_set_threads(hb, 1024)
        R.copy_(R0c)
        rank.copy_(r0c)
        y.copy_(y0c)
        st2, per2 = alm.alm_batch_solve(hb, R, rank, y)
        torch.cuda.synchronize()
        assert st1["converged"] == st2["converged"] == len(insts)
        assert torch.equal(R, R1) and torch.equal(y, y1)
        assert [p["objective"] for p in per1] == [p["objective"] for p in per2]
    finally:
        alm.alm_batch_destroy(hb)


def test_batch_rejects_bad_input():
    with pytest.raises(alm.AlmError) as e:
        alm.alm_batch_create([si.er_maxcut(20, 0.2, seed=1)], precision=alm.ALM_FP64)
    assert e.value.status == alm.ALM_ERR_INVALID_ARG
    bad = si.er_maxcut(20, 0.2, seed=1)
    bad.c_i = bad.c_i.copy()
    bad.c_i[-1] = 25  # row index beyond n
    with pytest.raises(alm.AlmError) as e:
        alm.alm_batch_create([si.er_maxcut(20, 0.2, seed=2), bad])
    assert "instance 1" in str(e.value)
