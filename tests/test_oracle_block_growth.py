"""Pins of Alg. 1's rank-growth step with several directions (oracle.block_growth_step):
it reduces to the closed form s* = -lambda / (sigma ||A(vv^T)||^2) for one direction; its
S satisfies the optimality conditions of the small SDP (S >= 0, W = Lambda + sigma
A_V^*(A_V(S)) >= 0, <S, W> = 0); the decrease it predicts is the augmented Lagrangian's
own decrease at the grown factor [R, V S^{1/2}]; and ALORA with several directions per
growth reaches the same optimal value."""
import math

import numpy as np
import pytest

import oracle as O
import sdp_instances as si


def _setup(k=3, seed=4):
    inst = si.er_maxcut(60, 0.2, seed=seed, weights="pm1")
    P = O.OracleProblem(inst)
    R = si.factor_init(inst.n, 2, 1)
    y = np.random.default_rng(seed).uniform(-2.0, 0.0, inst.m)
    sigma = 1.5
    w = O.dual_candidate(P, R, y, sigma)
    ev, Q = np.linalg.eigh(O.slack_dense(P, w))
    assert np.all(ev[:k] < 0)
    return P, R, y, sigma, ev[:k], Q[:, :k]


def test_one_direction_is_the_closed_form():
    P, R, y, sigma, lams, V = _setup(k=1)
    S = O.block_growth_step(P, lams, V, sigma)
    assert S.shape == (1, 1)
    assert S[0, 0] == pytest.approx(O.growth_step(P, lams[0], V[:, 0], sigma), rel=1e-9)


def test_small_sdp_optimality_conditions():
    P, R, y, sigma, lams, V = _setup(k=3)
    S = O.block_growth_step(P, lams, V, sigma)
    M = O.block_growth_map(P, V)
    W = np.diag(lams) + sigma * (M.T @ (M @ S.reshape(-1))).reshape(3, 3)
    W = 0.5 * (W + W.T)
    scale = float(np.abs(lams).max())
    assert np.linalg.eigvalsh(S).min() >= -1e-12
    assert np.linalg.eigvalsh(W).min() >= -1e-8 * scale
    assert abs(float(np.sum(S * W))) <= 1e-8 * scale * max(1.0, float(np.trace(S)))


def test_predicted_decrease_is_the_augmented_lagrangian_decrease():
    P, R, y, sigma, lams, V = _setup(k=3)
    S = O.block_growth_step(P, lams, V, sigma)
    M = O.block_growth_map(P, V)
    pred = float(np.sum(lams * np.diag(S))) + 0.5 * sigma * float(np.sum((M @ S.reshape(-1)) ** 2))
    R2 = np.hstack([R, V @ O.psd_sqrt(S)])
    actual = O.aug_lagrangian(P, R2, y, sigma) - O.aug_lagrangian(P, R, y, sigma)
    assert pred < 0
    assert actual == pytest.approx(pred, rel=1e-9, abs=1e-12)
    # more directions decrease L at least as much as the best single one
    s1 = O.growth_step(P, lams[0], V[:, 0], sigma)
    R1 = np.hstack([R, math.sqrt(s1) * V[:, [0]]])
    assert O.aug_lagrangian(P, R2, y, sigma) <= O.aug_lagrangian(P, R1, y, sigma) + 1e-12


def test_alora_with_block_growth_reaches_the_same_value():
    inst = si.er_maxcut(120, 0.08, seed=7)
    P = O.OracleProblem(inst)
    R0 = si.factor_init(inst.n, 1, 2)
    a = O.solve(P, R0, opts=O.SolveOptions(eps=1e-7, growth_k=1))
    b = O.solve(P, R0, opts=O.SolveOptions(eps=1e-7, growth_k=4))
    assert max(a.kkt) <= 1e-7 and max(b.kkt) <= 1e-7
    assert b.objective == pytest.approx(a.objective, rel=1e-6)
    assert any(h.get("grew") for h in b.history)
