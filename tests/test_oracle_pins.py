"""Pins of the FP64 oracle against what the paper and the mathematics fix
(closed forms, the paper's worked examples, finite differences, interpolation,
brute force, dense eigendecompositions).  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import sdp_instances as si

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _factor_of(X):
    """A factor R with RR^T = X for a PSD X (test helper, via eigh)."""
    ev, V = np.linalg.eigh(np.asarray(X, float))
    ev = np.clip(ev, 0, None)
    return V * np.sqrt(ev)


# ------------------------------------------------------------------------------
# eval: the quadratic-growth example of Sec. 3.2 (exact differences)
# ------------------------------------------------------------------------------
def test_eval_qg_example():
    g = _load("al_example_qg.json")
    P = O.OracleProblem(si.t11_instance())
    Rstar = np.array([[0.0], [1.0]])
    for c in g["cases"]:
        rho, eps, delta = c["rho"], c["eps"], c["delta"]
        y = np.array([-eps, 0.0])
        Rd = np.array([[math.sqrt(delta)], [1.0]])   # R R^T = [[d, sqrt d], [sqrt d, 1]]
        diff = O.aug_lagrangian(P, Rd, y, rho) - O.aug_lagrangian(P, Rstar, y, rho)
        assert diff == pytest.approx(eps * delta + rho / 2 * delta ** 2, rel=1e-13, abs=1e-15)


# ------------------------------------------------------------------------------
# the rank-2 example of Sec. 3.2 (n = 2, m = 3)
# ------------------------------------------------------------------------------
def test_rank2_example_value_gradient_dual():
    g = _load("al_example_rank2.json")
    P = O.OracleProblem(si.t8_instance())
    y = np.array(g["y"])
    rho = g["rho"]
    R = _factor_of(g["X_y_rho"])
    assert O.aug_lagrangian(P, R, y, rho) == pytest.approx(-13.0 / 32.0, abs=1e-15)
    assert np.allclose(O.gradient(P, R, y, rho), 0.0, atol=1e-15)
    z = O.dual_candidate(P, R, y, rho)
    assert np.allclose(z, 0.0, atol=1e-15)
    # Z(y) as printed
    assert np.allclose(O.slack_dense(P, y), np.array(g["Z_y"]), atol=1e-15)
    # (X*, y*) optimal for (P): zero gap, dual feasible, complementary
    Xs = np.array(g["X_star"])
    ys = np.array(g["y_star"])
    Rs = _factor_of(Xs)
    assert np.allclose(O.amap(P, Rs), P.b)
    Zs = O.slack_dense(P, ys)
    assert np.linalg.eigvalsh(Zs).min() >= -1e-15
    assert np.allclose(Zs @ Xs, 0.0)
    assert O.cost(P, Rs) == pytest.approx(float(P.b @ ys), abs=1e-15)


@pytest.mark.parametrize("method", ["cg", "gd"])
def test_rank2_example_inner_solve_reaches_unique_minimizer(method):
    """The unique minimiser X_{y,rho} = diag(1/4, 1/4) is reached from random
    starts by the inner solver (gradient + quartic line search)."""
    g = _load("al_example_rank2.json")
    P = O.OracleProblem(si.t8_instance())
    y = np.array(g["y"])
    for seed in range(3):
        R = si.factor_init(2, 3, seed)
        R = _inner(P, R, y, g["rho"], method, tol=1e-12, max_it=20000)
        assert np.allclose(R @ R.T, np.array(g["X_y_rho"]), atol=1e-8)


def _inner(P, R, y, sigma, method, tol, max_it):
    Gp = Dp = None
    for _ in range(max_it):
        G = O.gradient(P, R, y, sigma)
        if np.linalg.norm(G) <= tol:
            break
        D = -G
        if method == "cg" and Gp is not None:
            beta = max(0.0, float(np.sum(G * (G - Gp)) / np.sum(Gp * Gp)))
            D = -G + beta * Dp
            if np.sum(D * G) >= 0:
                D = -G
        a = O.exact_step(O.quartic_coeffs(P, R, D, y, sigma))
        if a == 0:
            break
        R = R + a * D
        Gp, Dp = G, D
    return R


# ------------------------------------------------------------------------------
# the generalised rank-r example of Sec. 3.2: X_{y,1} = diag(1_r/(2r), 0)
# ------------------------------------------------------------------------------
def _rank_r_example(n, r):
    """C = diag(0_r, 1_{n-r}); A_ij = (e_i e_j^T + e_j e_i^T)/2 (i < j <= r);
    A_ii = e_i e_i^T (i < r); A_rr = diag(I_r, 0); b_11 = b_rr = 1, else 0;
    y_11 = 1/(2r) - 1, y_ii = 1/(2r) (1 < i < r), y_rr = -1/2, off-diagonal 0."""
    ks, is_, js, vs, b, y = [], [], [], [], [], []
    k = 0
    for i in range(r):
        for j in range(i, r):
            if i == j and i < r - 1:
                ks.append(k); is_.append(i); js.append(i); vs.append(1.0)
                b.append(1.0 if i == 0 else 0.0)
                y.append(1 / (2 * r) - 1 if i == 0 else 1 / (2 * r))
            elif i == j:
                for t in range(r):
                    ks.append(k); is_.append(t); js.append(t); vs.append(1.0)
                b.append(1.0)
                y.append(-0.5)
            else:
                ks.append(k); is_.append(i); js.append(j); vs.append(0.5)
                b.append(0.0)
                y.append(0.0)
            k += 1
    c_v = np.concatenate([np.zeros(r), np.ones(n - r)])
    inst = si.Instance(n=n, m=k, c_i=np.arange(n, dtype=np.int32), c_j=np.arange(n, dtype=np.int32),
                       c_v=c_v, a_k=np.array(ks, np.int32), a_i=np.array(is_, np.int32),
                       a_j=np.array(js, np.int32), a_v=np.array(vs), b=np.array(b))
    return O.OracleProblem(inst), np.array(y)


@pytest.mark.parametrize("n,r", [(4, 2), (6, 3), (7, 4)])
def test_rank_r_example(n, r):
    P, y = _rank_r_example(n, r)
    X = np.diag(np.concatenate([np.full(r, 1 / (2 * r)), np.zeros(n - r)]))
    R = _factor_of(X)
    assert np.allclose(O.gradient(P, R, y, 1.0), 0.0, atol=1e-14)
    assert np.allclose(O.dual_candidate(P, R, y, 1.0), 0.0, atol=1e-14)
    # the unique minimiser is reached from a random start with rank >= r
    R0 = si.factor_init(n, r + 1, 11)
    R1 = _inner(P, R0, y, 1.0, "cg", tol=1e-12, max_it=50000)
    assert np.allclose(R1 @ R1.T, X, atol=1e-7)


# ------------------------------------------------------------------------------
# the spurious local minimiser of Sec. 4.3 (dual infeasible y)
# ------------------------------------------------------------------------------
def test_spurious_example_map_gradient_eigen_growth():
    g = _load("al_example_spurious.json")
    for c in g["cases"]:
        d, k, eta, rho, eps = c["d"], c["k"], c["eta"], c["rho"], c["eps"]
        a = eta ** 2 * k
        assert eps < eta ** 2 * rho / 4
        P = O.OracleProblem(si.t15_instance(d, eps, a))
        y = np.zeros(d)
        y[-1] = 2.0
        F = np.zeros((d, k))
        F[:k, :k] = eta * np.eye(k)
        assert np.allclose(O.amap(P, F), P.b, atol=1e-14)
        expect = np.zeros((d, d))
        expect[-1, -1] = -eps
        assert np.allclose(O.slack_dense(P, y), expect, atol=1e-14)
        assert np.allclose(O.gradient(P, F, y, rho), 0.0, atol=1e-14)
        # smallest eigenpair of grad_X L = Z(w), w = y since A(FF^T) = b
        w = O.dual_candidate(P, F, y, rho)
        lam, v, _ = O.lambda_min(P, w)
        assert lam == pytest.approx(-eps, abs=1e-14)
        assert abs(abs(v[-1]) - 1.0) < 1e-12
        # rank-one growth step: ||A(e_d e_d^T)||^2 = eps^2 -> s* = 1/(rho eps)
        assert O.growth_step(P, lam, v, rho) == pytest.approx(1.0 / (rho * eps), rel=1e-12)
        # the lowered AL value matches the exact expansion along v v^T
        s = O.growth_step(P, lam, v, rho)
        Fg = np.hstack([F, math.sqrt(s) * v.reshape(-1, 1)])
        drop = O.aug_lagrangian(P, Fg, y, rho) - O.aug_lagrangian(P, F, y, rho)
        assert drop == pytest.approx(-0.5 * lam ** 2 / (rho * eps ** 2), rel=1e-10)


# ------------------------------------------------------------------------------
# gradient: central finite differences of the augmented Lagrangian
# ------------------------------------------------------------------------------
def _instances_small():
    return [
        si.er_maxcut(40, 0.2, seed=5, weights="pm1"),
        si.lovasz_theta(12, *si.cycle_edges(12)),
        si.random_general(25, 9, seed=3),
        si.random_general(18, 30, seed=4, lr_k=2, diag_frac=0.2),
    ]


@pytest.mark.parametrize("idx", range(4))
def test_gradient_finite_differences(idx):
    inst = _instances_small()[idx]
    P = O.OracleProblem(inst)
    rng = np.random.default_rng(idx)
    r = 3
    R = rng.standard_normal((P.n, r)) * 0.7
    y = rng.standard_normal(P.m)
    sigma = 1.7
    G = O.gradient(P, R, y, sigma)
    h = 1e-6 * max(1.0, np.linalg.norm(R))
    # directional derivatives along random directions and along unit coordinates
    for t in range(6):
        D = rng.standard_normal(R.shape) if t < 4 else np.eye(P.n, r, k=-t)
        fd = (O.aug_lagrangian(P, R + h * D, y, sigma) - O.aug_lagrangian(P, R - h * D, y, sigma)) / (2 * h)
        assert np.sum(G * D) == pytest.approx(fd, rel=1e-6, abs=1e-7 * (1 + np.abs(G).sum()))


# ------------------------------------------------------------------------------
# line search: phi(alpha) through eval reproduces q0..q4; alpha* vs brute force
# ------------------------------------------------------------------------------
@pytest.mark.parametrize("idx", range(4))
def test_quartic_coefficients_interpolate_eval(idx):
    inst = _instances_small()[idx]
    P = O.OracleProblem(inst)
    rng = np.random.default_rng(10 + idx)
    R = rng.standard_normal((P.n, 4))
    D = rng.standard_normal((P.n, 4))
    y = rng.standard_normal(P.m)
    sigma = 0.9
    q = O.quartic_coeffs(P, R, D, y, sigma)
    alphas = np.array([-1.0, -0.5, 0.0, 0.5, 1.0])
    phi = np.array([O.aug_lagrangian(P, R + a * D, y, sigma) for a in alphas])
    V = np.vander(alphas, 5, increasing=True)
    q_fit = np.linalg.solve(V, phi)
    assert np.allclose(q, q_fit, rtol=1e-9, atol=1e-9 * np.abs(phi).max())
    # directional derivative identity: <G, D> = q1
    G = O.gradient(P, R, y, sigma)
    assert q[1] == pytest.approx(float(np.sum(G * D)), rel=1e-10, abs=1e-10)


def _brute_argmin(q, hi):
    xs = np.linspace(0.0, hi, 200001)
    vals = O.quartic_value(q, xs)
    i = int(np.argmin(vals))
    lo_, hi_ = xs[max(i - 1, 0)], xs[min(i + 1, xs.size - 1)]
    gr = (math.sqrt(5) - 1) / 2
    a, b = lo_, hi_
    for _ in range(200):
        c = b - gr * (b - a)
        d = a + gr * (b - a)
        if O.quartic_value(q, c) < O.quartic_value(q, d):
            b = d
        else:
            a = c
    return 0.5 * (a + b)


def test_exact_step_brute_force():
    rng = np.random.default_rng(0)
    for t in range(300):
        q = rng.standard_normal(5)
        q[4] = abs(q[4]) + 0.05
        if t % 5 == 0:
            q[1] = abs(q[1])           # increasing at 0 -> possibly no positive minimiser
        a = O.exact_step(q)
        # Cauchy bound on the roots of phi' = 4q4 a^3 + 3q3 a^2 + 2q2 a + q1
        hi = 1.5 * (1.0 + max(abs(3 * q[3]), abs(2 * q[2]), abs(q[1])) / (4 * q[4]))
        ab = _brute_argmin(q, hi)
        assert O.quartic_value(q, a) <= O.quartic_value(q, ab) + 1e-9
        if a > 0:
            assert abs(a - ab) < 1e-5 or abs(O.quartic_value(q, a) - O.quartic_value(q, ab)) < 1e-10


def test_exact_step_special_cases():
    # pure quadratic (q3 = q4 = 0): alpha = -q1/(2 q2)
    assert O.exact_step([0, -2.0, 4.0, 0, 0]) == pytest.approx(0.25)
    # no descent: alpha = 0
    assert O.exact_step([0, 1.0, 1.0, 0.0, 1.0]) == 0.0
    # unbounded below
    assert O.exact_step([0, -1.0, 0.0, 0.0, 0.0]) == math.inf
    assert O.exact_step([0, 1.0, 0.0, 0.0, -1.0]) == math.inf
    # symmetric double well (x^2 - 1)^2 shifted: minima at 1 (and -1, excluded)
    assert O.exact_step([1.0, 0.0, -2.0, 0.0, 1.0]) == pytest.approx(1.0)


# ------------------------------------------------------------------------------
# smallest eigenvalue: closed spectra and Lanczos against dense eigh
# ------------------------------------------------------------------------------
@pytest.mark.parametrize("n1,n2,sigma", [(4, 6, 1.0), (8, 8, 0.5), (6, 10, 2.0)])
def test_lambda_min_torus_closed_form(n1, n2, sigma):
    """R = 0, y = 0: w = sigma*b, Z(w) = -L/4 - sigma I; L of an even torus has
    largest eigenvalue 8, so lambda_min = -2 - sigma."""
    P = O.OracleProblem(si.torus_maxcut(n1, n2, weights="unit"))
    R = np.zeros((P.n, 1))
    w = O.dual_candidate(P, R, np.zeros(P.m), sigma)
    lam, v, _ = O.lambda_min(P, w)
    assert lam == pytest.approx(-2.0 - sigma, abs=1e-12)
    lam2, _, res = O.lambda_min(P, w, dense_max=0, tol=1e-12)
    assert lam2 == pytest.approx(-2.0 - sigma, abs=1e-9)


@pytest.mark.parametrize("n", [7, 10])
def test_lambda_min_complete_and_cycle(n):
    Pk = O.OracleProblem(si.maxcut(n, *si.complete_edges(n), np.ones(n * (n - 1) // 2)))
    lam, _, _ = O.lambda_min(Pk, np.zeros(n))
    assert lam == pytest.approx(-n / 4, abs=1e-12)        # L(K_n) spectrum {0, n}
    Pc = O.OracleProblem(si.maxcut(n, *si.cycle_edges(n), np.ones(n)))
    lam, _, _ = O.lambda_min(Pc, np.zeros(n))
    top = 4.0 if n % 2 == 0 else 2 + 2 * math.cos(math.pi / n)
    assert lam == pytest.approx(-top / 4, abs=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lanczos_matches_dense(seed):
    inst = [si.er_maxcut(600, 0.01, seed=seed, weights="pm1"),
            si.random_general(400, 60, seed=seed, lr_k=1),
            si.theta_er(500, 6.0, seed=seed)][seed]
    P = O.OracleProblem(inst)
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(P.m) * 0.3
    lam_d, v_d, _ = O.lambda_min(P, w, dense_max=10 ** 9)
    lam_l, v_l, res = O.lambda_min(P, w, dense_max=0, tol=1e-11)
    assert lam_l == pytest.approx(lam_d, abs=1e-8 * (1 + abs(lam_d)))
    S = O.slack_dense(P, w)
    assert np.linalg.norm(S @ v_l - lam_l * v_l) <= 1e-6 * np.abs(S).sum(axis=1).max()


def test_frobenius_norm_of_C_with_low_rank():
    for inst in [si.random_general(30, 5, seed=9, lr_k=2), si.theta_er(40, 4.0, seed=2)]:
        P = O.OracleProblem(inst)
        Cd = O.slack_dense(P, np.zeros(P.m))       # Z(0) = C
        assert P.norm_C == pytest.approx(np.linalg.norm(Cd), rel=1e-12)


def test_preconditioner_inverts_its_row_blocks():
    """Z = P^{-1} G: applying the row block P_i = 2 s_i I + 4 sigma a_i^2 r_i r_i^T to Z_i
    gives back G_i (Sherman-Morrison written out), with s_i = max(S_ii, floor)."""
    inst = si.er_maxcut(50, 0.2, seed=4, weights="pm1")
    P = O.OracleProblem(inst)
    rng = np.random.default_rng(3)
    R = rng.standard_normal((P.n, 5)) * 0.4
    y = rng.uniform(-1, 1, P.m)
    sigma = 3.0
    G = rng.standard_normal(R.shape)
    Z = O.precondition(P, R, y, sigma, G)
    w = O.dual_candidate(P, R, y, sigma)
    s = np.asarray(O.slack_sparse(P, w).diagonal())
    cdiag = np.zeros(P.n)
    np.add.at(cdiag, P.c_i[P.c_i == P.c_j], P.c_v[P.c_i == P.c_j])
    s = np.maximum(s, 1e-2 * (1 + np.mean(np.abs(cdiag))))
    for i in range(P.n):
        Pi = 2 * s[i] * np.eye(5) + 4 * sigma * np.outer(R[i], R[i])   # a_i = 1 for MaxCut
        assert np.allclose(Pi @ Z[i], G[i], atol=1e-12)
