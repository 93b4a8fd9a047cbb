"""The matrix-completion workload of Sec. 6.2 on the GPU (nuclear-norm SDP: C = I/2,
off-diagonal selector constraints X_{i, n1+j} = M_ij, so S's off-diagonal values move with
y): solves in FP64 and in the FP32-bulk form against the closed forms the oracle is pinned
by (the nuclear norm when every entry is observed; exact recovery of a sampled rank-1
matrix) and against the oracle's own solve on a sampled rank-2 instance, with the oracle's
KKT check of the GPU's (R, y) at 1e-6."""
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

# FP64 solves to 1e-7; the FP32-bulk form to the solver's target 1e-6 (its general-constraint
# path moves S's off-diagonal values with y in FP32, which puts 1e-7 out of reach here)
EPS = {alm.ALM_FP64: 1e-7, alm.ALM_FP32: 1e-6}
OPTS = dict(sigma0=1.0, sigma_rule=alm.ALM_SIGMA_ADAPTIVE)


def _gpu(inst, prec, r0=4):
    R0 = si.factor_init(inst.n, r0, 1, scale=0.3)
    h = alm.alm_create(inst, precision=prec, eps=EPS[prec], **OPTS)
    try:
        R, r, y, st = alm.alm_solve(h, R0)
        return as_np(R), as_np(y), st
    finally:
        alm.alm_destroy(h)


def _kkt(inst, R, y):
    P = O.OracleProblem(inst)
    lam = float(np.linalg.eigvalsh(O.slack_dense(P, y))[0])
    return P, O.kkt(P, R, y, lam)


def _nuclear(inst):
    U, V, _ = inst.graph
    return float(np.linalg.svd(U @ V.T, compute_uv=False).sum())


@pytest.mark.parametrize("prec", [alm.ALM_FP64, alm.ALM_FP32])
@pytest.mark.parametrize("rank", [1, 2])
def test_fully_observed_value_is_the_nuclear_norm(prec, rank):
    inst = si.matrix_completion(6, 5, rank, seed=(9, rank), m=30)
    R, y, st = _gpu(inst, prec)
    assert st["status"] == 0, st
    assert st["objective"] == pytest.approx(_nuclear(inst), rel=2e-6)
    P, k = _kkt(inst, R, y)
    assert max(k) <= 1e-6


@pytest.mark.parametrize("prec", [alm.ALM_FP64, alm.ALM_FP32])
def test_sampled_rank_one_is_recovered(prec):
    n1 = n2 = 20
    inst = si.matrix_completion(n1, n2, 1, seed=(9, 20, 1))
    R, y, st = _gpu(inst, prec)
    U, V, _ = inst.graph
    M = U @ V.T
    assert inst.m < n1 * n2 and st["status"] == 0, st
    assert st["objective"] == pytest.approx(_nuclear(inst), rel=2e-6)
    Y = (R @ R.T)[:n1, n1:]
    # the completion error follows the KKT residual the solve stops at (1e-7 / 1e-6)
    assert np.max(np.abs(Y - M)) <= (1e-4 if prec == alm.ALM_FP64 else 1e-3) * np.max(np.abs(M))
    P, k = _kkt(inst, R, y)
    assert max(k) <= 1e-6


@pytest.mark.parametrize("prec", [alm.ALM_FP64, alm.ALM_FP32])
def test_sampled_rank_two_matches_the_oracle_solve(prec):
    inst = si.matrix_completion(60, 50, 2, seed=(9, 60, 2))
    R, y, st = _gpu(inst, prec)
    assert st["status"] == 0, st
    P = O.OracleProblem(inst)
    ref = O.solve(P, si.factor_init(inst.n, 4, 1, scale=0.3),
                  opts=O.SolveOptions(eps=1e-7, sigma=1.0, sigma_rule="adaptive"))
    assert max(ref.kkt) <= 1e-7
    assert st["objective"] == pytest.approx(ref.objective, rel=2e-6)
    P, k = _kkt(inst, R, y)
    assert max(k) <= 1e-6
