"""Pins of the L-BFGS inner direction of the oracle (oracle.lbfgs_direction, option
inner_method="lbfgs"): the two-loop recursion equals the explicit BFGS inverse-Hessian
product built pair by pair from the scaled identity, it satisfies the secant equation of
the newest pair, and ALORA with it reaches the same optimal value as with CG."""
import numpy as np
import pytest

import oracle as O
import sdp_instances as si


def _pairs(d=6, k=3, seed=0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((d, d))
    A = A @ A.T + d * np.eye(d)           # SPD: y = A s gives s.y > 0
    pairs = []
    for _ in range(k):
        s = rng.standard_normal(d)
        pairs.append((s, A @ s))
    return pairs, rng.standard_normal(d)


def _explicit(pairs, g):
    s, y = pairs[-1]
    H = (s @ y) / (y @ y) * np.eye(g.size)
    for s, y in pairs:
        rho = 1.0 / (y @ s)
        V = np.eye(g.size) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return H @ g


def test_two_loop_equals_explicit_bfgs():
    pairs, g = _pairs()
    assert np.allclose(O.lbfgs_direction(g, pairs), _explicit(pairs, g), rtol=1e-12, atol=1e-12)


def test_secant_equation_of_the_newest_pair():
    pairs, _ = _pairs(seed=3)
    s, y = pairs[-1]
    assert np.allclose(O.lbfgs_direction(y, pairs), s, rtol=1e-10, atol=1e-12)


def test_no_pairs_gives_the_gradient():
    g = np.arange(5.0)
    assert np.array_equal(O.lbfgs_direction(g, []), g)


def test_alora_with_lbfgs_reaches_the_same_value():
    inst = si.er_maxcut(150, 0.06, seed=5)
    P = O.OracleProblem(inst)
    R0 = si.factor_init(inst.n, 8, 3)
    a = O.solve(P, R0, opts=O.SolveOptions(eps=1e-7))
    b = O.solve(P, R0, opts=O.SolveOptions(eps=1e-7, inner_method="lbfgs"))
    assert max(a.kkt) <= 1e-7 and max(b.kkt) <= 1e-7
    assert b.objective == pytest.approx(a.objective, rel=1e-6)
