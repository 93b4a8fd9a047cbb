"""The matrix-completion workload of Sec. 6.2 (nuclear-norm SDP) in the oracle: the
generator's sampling rule, and solves pinned by the closed form min tr(X)/2 = ||M||_*
(sum of singular values) when every entry is observed, and by exact recovery of a
sufficiently sampled rank-1 matrix (the completion is M itself)."""
import math

import numpy as np
import pytest

import oracle as O
import sdp_instances as si


def _solve(inst):
    P = O.OracleProblem(inst)
    res = O.solve(P, si.factor_init(inst.n, 4, 1, scale=0.3),
                  opts=O.SolveOptions(eps=1e-7, sigma=1.0, sigma_rule="adaptive"))
    return P, res


def test_generator_sampling_rule():
    n1, n2, r = 40, 35, 2
    inst = si.matrix_completion(n1, n2, r, seed=3)
    n = n1 + n2
    assert inst.m == min(math.ceil(r * math.log(n) * r * (n - r)), n1 * n2)
    pos = inst.a_i.astype(np.int64) * n2 + (inst.a_j.astype(np.int64) - n1)
    assert np.unique(pos).size == inst.m                     # distinct positions
    assert np.all(inst.a_j >= n1) and np.all(inst.a_i < n1)   # the off-diagonal block
    U, V, _ = inst.graph
    assert np.allclose(inst.b, np.einsum("ij,ij->i", U[inst.a_i], V[inst.a_j - n1]))
    assert np.all(inst.c_v == 0.5) and inst.c_i.size == n    # C = I/2


@pytest.mark.parametrize("rank", [1, 2])
def test_fully_observed_value_is_the_nuclear_norm(rank):
    n1, n2 = 6, 5
    inst = si.matrix_completion(n1, n2, rank, seed=(9, rank), m=n1 * n2)
    P, res = _solve(inst)
    U, V, _ = inst.graph
    nuc = float(np.linalg.svd(U @ V.T, compute_uv=False).sum())
    assert max(res.kkt) <= 1e-7
    assert res.objective == pytest.approx(nuc, rel=1e-6)


def test_sampled_rank_one_is_recovered_exactly():
    n1 = n2 = 20
    inst = si.matrix_completion(n1, n2, 1, seed=(9, 20, 1))
    P, res = _solve(inst)
    U, V, _ = inst.graph
    M = U @ V.T
    assert inst.m < n1 * n2
    assert max(res.kkt) <= 1e-7
    assert res.objective == pytest.approx(float(np.linalg.svd(M, compute_uv=False).sum()), rel=1e-6)
    Y = (res.R @ res.R.T)[:n1, n1:]
    assert np.max(np.abs(Y - M)) <= 1e-4 * np.max(np.abs(M))
