"""Full ALORA solves of the oracle against closed-form SDP optimal values and a
dense duality certificate.  CPU only.

Closed forms (textbook):
* MaxCut SDP of the complete graph K_n (unit weights): n^2/4 (X = (nI - J)/(n-1)).
* MaxCut SDP of the cycle C_n: n for even n, (n/2)(1 + cos(pi/n)) for odd n
  (unit vectors at angle pi(n-1)/n around a circle; Goemans-Williamson / Delorme-Poljak).
* Lovasz theta (Lovasz 1979): theta(C_n) = n cos(pi/n)/(1 + cos(pi/n)) for odd n
  (theta(C_5) = sqrt 5), theta(K_n) = 1, theta of the empty graph = n.
"""
import math

import numpy as np
import pytest

import oracle as O
import sdp_instances as si

EPS = 1e-7


def _solve(inst, r0, seed=0, **kw):
    P = O.OracleProblem(inst)
    scale = 1.0 / math.sqrt(r0) if inst.kind == "maxcut" else 1.0 / math.sqrt(inst.n * r0)
    R0 = si.factor_init(P.n, r0, seed, scale=scale)
    if inst.kind == "theta":
        kw.setdefault("sigma_rule", "adaptive")   # the theta SDPs need a growing penalty
    res = O.solve(P, R0, opts=O.SolveOptions(eps=EPS, **kw))
    return P, res


def _certificate(P, res, tol):
    """Dense check: dual feasibility of y (lambda_min(C - A^* y) >= -tol(1+||C||))
    and a small duality gap."""
    Z = O.slack_dense(P, res.y)
    lam = np.linalg.eigvalsh(Z)[0]
    assert lam >= -tol * (1 + P.norm_C)
    cx, by = res.objective, float(P.b @ res.y)
    assert abs(cx - by) <= tol * (1 + abs(cx) + abs(by))
    assert max(res.kkt) <= EPS


@pytest.mark.parametrize("n", [6, 9])
def test_maxcut_complete_graph(n):
    inst = si.maxcut(n, *si.complete_edges(n), np.ones(n * (n - 1) // 2))
    P, res = _solve(inst, 2)
    assert -res.objective == pytest.approx(n * n / 4, rel=1e-6)
    _certificate(P, res, 1e-6)


@pytest.mark.parametrize("n", [5, 7, 8, 12])
def test_maxcut_cycle(n):
    inst = si.maxcut(n, *si.cycle_edges(n), np.ones(n))
    P, res = _solve(inst, 2)
    expect = float(n) if n % 2 == 0 else n / 2 * (1 + math.cos(math.pi / n))
    assert -res.objective == pytest.approx(expect, rel=1e-6)
    _certificate(P, res, 1e-6)


@pytest.mark.parametrize("n", [5, 7, 9])
def test_theta_odd_cycle(n):
    inst = si.lovasz_theta(n, *si.cycle_edges(n))
    P, res = _solve(inst, 2)
    expect = n * math.cos(math.pi / n) / (1 + math.cos(math.pi / n))
    if n == 5:
        assert expect == pytest.approx(math.sqrt(5), rel=1e-15)
    assert -res.objective == pytest.approx(expect, rel=1e-6)
    _certificate(P, res, 1e-6)


def test_theta_complete_and_empty():
    n = 6
    P, res = _solve(si.lovasz_theta(n, *si.complete_edges(n)), 2)
    assert -res.objective == pytest.approx(1.0, rel=1e-6)
    P, res = _solve(si.lovasz_theta(n, np.zeros(0, np.int64), np.zeros(0, np.int64)), 2)
    assert -res.objective == pytest.approx(float(n), rel=1e-6)


def test_maxcut_er_certificate_and_growth():
    """ER MaxCut from rank 1: the rank grows (Alg. 1's escape) and the dense
    certificate holds at the end."""
    inst = si.er_maxcut(60, 0.15, seed=7, weights="pm1")
    P, res = _solve(inst, 1)
    assert res.rank > 1
    _certificate(P, res, 1e-6)


@pytest.mark.parametrize("method", ["gd", "cg"])
def test_al_minimizers_share_constraint_image(method):
    """All minimisers of (AL-P) at a fixed y share A(X) (Sec. 2.3 lemma): inner
    solves from different random starts agree on A(RR^T) and on L."""
    inst = si.er_maxcut(30, 0.3, seed=2)
    P = O.OracleProblem(inst)
    rng = np.random.default_rng(0)
    y = rng.uniform(-1.0, 0.5, P.m)
    outs = []
    for seed in range(2):
        R = si.factor_init(P.n, 12, seed)
        Gp = Dp = None
        for _ in range(20000):
            G = O.gradient(P, R, y, 1.0)
            if np.linalg.norm(G) < 1e-10:
                break
            D = -G
            if method == "cg" and Gp is not None:
                beta = max(0.0, float(np.sum(G * (G - Gp)) / np.sum(Gp * Gp)))
                D = -G + beta * Dp
                if np.sum(D * G) >= 0:
                    D = -G
            a = O.exact_step(O.quartic_coeffs(P, R, D, y, 1.0))
            if a == 0:
                break
            R = R + a * D
            Gp, Dp = G, D
        outs.append((O.amap(P, R), O.aug_lagrangian(P, R, y, 1.0)))
    assert np.allclose(outs[0][0], outs[1][0], atol=1e-7)
    assert outs[0][1] == pytest.approx(outs[1][1], rel=1e-10)
