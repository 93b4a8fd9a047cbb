"""GPU ALORA solves (through the C-ABI) against closed-form SDP values and the FP64
oracle: same objective within 1e-6 relative, and the GPU's final (R, y) re-checked
by the oracle (dense eigendecomposition) to satisfy relative KKT <= 1e-6."""
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


def _gpu_solve(inst, r0, prec, eps=1e-7, seed=0, **opt):
    scale = None if inst.kind == "maxcut" else 1.0 / math.sqrt(inst.n * r0)
    R0 = si.factor_init(inst.n, r0, seed, scale=scale)
    h = alm.alm_create(inst, precision=prec, eps=eps, **opt)
    try:
        R, r, y, st = alm.alm_solve(h, R0)
    finally:
        alm.alm_destroy(h)
    return as_np(R), as_np(y), st, R0


def _oracle_kkt(inst, R, y):
    P = O.OracleProblem(inst)
    lam = float(np.linalg.eigvalsh(O.slack_dense(P, y))[0])
    return P, O.kkt(P, R, y, lam)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [8, 9, 10])
def test_maxcut_closed_forms(prec, n):
    inst = si.maxcut(n, *si.cycle_edges(n), np.ones(n))
    R, y, st, _ = _gpu_solve(inst, 2, prec)
    expect = float(n) if n % 2 == 0 else n / 2 * (1 + math.cos(math.pi / n))
    assert st["status"] == 0
    assert -st["objective"] == pytest.approx(expect, rel=1e-6)
    P, k = _oracle_kkt(inst, R, y)
    assert max(k) <= 1e-6


@pytest.mark.parametrize("prec", [0, 1])
def test_maxcut_complete_graph(prec):
    n = 9
    inst = si.maxcut(n, *si.complete_edges(n), np.ones(n * (n - 1) // 2))
    R, y, st, _ = _gpu_solve(inst, 2, prec)
    assert -st["objective"] == pytest.approx(n * n / 4, rel=1e-6)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [5, 7])
def test_theta_odd_cycles(prec, n):
    inst = si.lovasz_theta(n, *si.cycle_edges(n))
    R, y, st, _ = _gpu_solve(inst, 2, prec, sigma_rule=alm.ALM_SIGMA_ADAPTIVE)
    expect = n * math.cos(math.pi / n) / (1 + math.cos(math.pi / n))
    assert st["status"] == 0
    assert -st["objective"] == pytest.approx(expect, rel=1e-6)
    P, k = _oracle_kkt(inst, R, y)
    assert max(k) <= 1e-6


@pytest.mark.parametrize("lanczos_warm", [0, 1])
@pytest.mark.parametrize("prec", [0, 1])
def test_er800_matches_oracle_solve(prec, lanczos_warm):
    """MaxCut on G(800, 0.06), r0 = 8, sigma = 1: GPU (FP64, or FP32 bulk with FP64
    dual; Lanczos from a fresh vector or from the previous Ritz vector) and the oracle
    reach the same objective, and the oracle confirms the GPU's KKT residual."""
    inst = si.er_maxcut(800, 0.06, seed=1)
    R, y, st, R0 = _gpu_solve(inst, 8, prec, lanczos_warm=lanczos_warm)
    assert st["status"] == 0, st
    P = O.OracleProblem(inst)
    ref = O.solve(P, R0, opts=O.SolveOptions(eps=1e-7))
    assert max(ref.kkt) <= 1e-7
    assert st["objective"] == pytest.approx(ref.objective, rel=1e-6)
    _, k = _oracle_kkt(inst, R, y)
    assert max(k) <= 1e-6
    assert O.cost(P, R) == pytest.approx(st["objective"], rel=1e-9 if prec == 0 else 1e-6)


def test_solve_reports_not_converged_at_cap():
    inst = si.er_maxcut(200, 0.1, seed=3)
    R, y, st, _ = _gpu_solve(inst, 2, 0, max_outer=2)
    assert st["status"] == alm.ALM_ERR_NOT_CONVERGED
    assert st["outer"] == 2


def test_solve_rank_grows_from_one():
    inst = si.er_maxcut(120, 0.1, seed=9, weights="pm1")
    R, y, st, _ = _gpu_solve(inst, 1, 0)
    assert st["status"] == 0
    assert st["rank"] > 1 and st["growth_steps"] == st["rank"] - 1


def test_profile_mode_times_spmm():
    inst = si.torus_maxcut(64, 64, seed=2)
    R, y, st, _ = _gpu_solve(inst, 8, 1, eps=1e-5, profile=1)
    assert st["spmm_launches"] > 0 and st["spmm_ms"] > 0 and st["spmm_bytes"] > 0
    assert st["kernel_launches"] > st["spmm_launches"]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("which", ["torus-40x50-pm1", "regular3-1500"])
def test_ell_inner_loop_matches_oracle_solve(which, prec):
    """Instances with short rows take the ELL inner loop (the pending step, the slack
    diagonal and the SpMM in one kernel with ping-pong factor buffers; the direction fused
    into the line search), with r0 = r_max = 32 and sigma0 = 10 as in the benchmark: same
    objective as the oracle's solve, and the oracle confirms the KKT residual."""
    inst = si.torus_maxcut(40, 50, seed=3, weights="pm1") if which.startswith("torus") else \
        si.regular3_maxcut(1500, seed=12)
    R, y, st, R0 = _gpu_solve(inst, 32, prec, eps=1e-7, sigma0=10.0, lanczos_warm=1)
    assert st["status"] == 0, st
    P = O.OracleProblem(inst)
    ref = O.solve(P, R0, opts=O.SolveOptions(eps=1e-7, sigma=10.0))
    assert max(ref.kkt) <= 1e-7
    assert st["objective"] == pytest.approx(ref.objective, rel=1e-6)
    P, k = _oracle_kkt(inst, R, y)
    assert max(k) <= 1e-6
    assert O.cost(P, R) == pytest.approx(st["objective"], rel=1e-9 if prec == 0 else 1e-6)


@pytest.mark.parametrize("prec", [0, 1])
def test_checkpoint_resume_reproduces_the_trajectory(tmp_path, prec):
    """Stop a solve after 3 outer iterations, save it, resume it on a fresh handle: the
    result is bit for bit that of the uninterrupted solve (same rank, counters, R, y)."""
    inst = si.er_maxcut(400, 0.03, seed=21)
    R0 = si.factor_init(inst.n, 8, 5)
    opts = dict(precision=prec, eps=1e-7)
    hs = [alm.alm_create(inst, **opts), alm.alm_create(inst, max_outer=3, **opts), alm.alm_create(inst, **opts)]
    try:
        Ra, ra, ya, sa = alm.alm_solve(hs[0], R0)
        Rb, rb, yb, sb = alm.alm_solve(hs[1], R0)
        assert sa["status"] == 0 and sa["outer"] > 3
        assert sb["status"] == alm.ALM_ERR_NOT_CONVERGED and sb["outer"] == 3
        path = str(tmp_path / "alm.ckpt")
        alm.alm_checkpoint(hs[1], path)
        Rc, rc, yc, sc = alm.alm_resume(hs[2], path)
        assert sc["status"] == 0 and rc == ra
        for k in ("outer", "inner_total", "lanczos_matvecs", "growth_steps"):
            assert sc[k] == sa[k], k
        assert torch.equal(Rc, Ra) and torch.equal(yc, ya)
        assert sc["objective"] == sa["objective"]
    finally:
        for h in hs:
            alm.alm_destroy(h)


def test_checkpoint_needs_a_solve_and_a_matching_problem(tmp_path):
    a = alm.alm_create(si.er_maxcut(60, 0.1, seed=1), precision=0)
    b = alm.alm_create(si.er_maxcut(70, 0.1, seed=1), precision=0)
    try:
        with pytest.raises(alm.AlmError):
            alm.alm_checkpoint(a, str(tmp_path / "none.ckpt"))
        alm.alm_solve(a, si.factor_init(60, 4, 1))
        alm.alm_checkpoint(a, str(tmp_path / "a.ckpt"))
        with pytest.raises(alm.AlmError) as e:
            alm.alm_resume(b, str(tmp_path / "a.ckpt"))
        assert "another problem" in str(e.value)
        # same n, m and precision but different edges: rejected by the problem fingerprint
        c = alm.alm_create(si.er_maxcut(60, 0.1, seed=2), precision=0)
        try:
            with pytest.raises(alm.AlmError) as e:
                alm.alm_resume(c, str(tmp_path / "a.ckpt"))
            assert e.value.status == alm.ALM_ERR_INVALID_ARG
            assert "C, A or b differ" in str(e.value)
        finally:
            alm.alm_destroy(c)
        # the same problem built again resumes
        d = alm.alm_create(si.er_maxcut(60, 0.1, seed=1), precision=0)
        try:
            alm.alm_resume(d, str(tmp_path / "a.ckpt"))
        finally:
            alm.alm_destroy(d)
    finally:
        alm.alm_destroy(a)
        alm.alm_destroy(b)


@pytest.mark.parametrize("prec", [0, 1])
def test_block_growth_matches_the_oracle_and_needs_fewer_outer_iterations(prec):
    """Alg. 1's growth along several eigenvectors (growth_k = 4: up to four eigenpairs below
    -tau_lambda, deflated Lanczos, the 4 x 4 SDP on the device, R <- [R, V S^{1/2}]) from a
    rank-1 start: the oracle's solve with the same growth rule reaches the same objective,
    the oracle confirms the KKT residual, and the solve takes fewer outer iterations and
    growth steps than growing one direction at a time."""
    inst = si.er_maxcut(120, 0.08, seed=7)
    R0 = si.factor_init(inst.n, 1, 2)
    P = O.OracleProblem(inst)
    ref = O.solve(P, R0, opts=O.SolveOptions(eps=1e-7, growth_k=4))
    assert max(ref.kkt) <= 1e-7
    out = {}
    for k in (1, 4):
        h = alm.alm_create(inst, precision=prec, eps=1e-7, growth_k=k)
        try:
            R, r, y, st = alm.alm_solve(h, R0)
            out[k] = (as_np(R), as_np(y), st)
        finally:
            alm.alm_destroy(h)
    R, y, st = out[4]
    assert st["status"] == 0, st
    assert st["objective"] == pytest.approx(ref.objective, rel=1e-6)
    _, k = _oracle_kkt(inst, R, y)
    assert max(k) <= 1e-6
    assert st["outer"] < out[1][2]["outer"]
    assert st["growth_steps"] < out[1][2]["growth_steps"]


def test_growth_k_is_validated():
    with pytest.raises(alm.AlmError) as e:
        alm.alm_create(si.er_maxcut(30, 0.2, seed=1), growth_k=5)
    assert e.value.status == alm.ALM_ERR_INVALID_ARG
