"""FP64 CPU oracle of ALM-BM / ALORA (TEST INFRASTRUCTURE ONLY; see package doc).

Notation follows the paper: the SDP (P) is ``min <C, X>  s.t.  A(X) = b, X >= 0``
with ``[A(X)]_k = <A_k, X>`` (Sec. 1.2); the factor is ``R`` (the paper's ``F``),
``X = R R^T``; the penalty is ``sigma`` (the paper's ``rho``).  Symmetric data is
given by upper-triangle entries: an off-diagonal entry ``v`` at (i, j) stands for
``M_ij = M_ji = v`` and so contributes ``2 v X_ij`` to ``<M, X>``.

Derived quantities used throughout:
  w = y - sigma (A(RR^T) - b)                        (the ALM dual update, Eq. ALM)
  S = C - A^*(w) = grad_X L_sigma(X, y) at X = RR^T  (dual slack map Z(w), Sec. 1.2)
  grad_R L = 2 S R                                    (BM gradient 2 grad f(FF^T) F, Sec. 4.2)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg
import scipy.sparse as sp


# ----------------------------------------------------------------------------------
# problem
# ----------------------------------------------------------------------------------
class OracleProblem:
    """(C, {A_k}, b) of (P), from the coordinate form of ``sdp_instances.Instance``."""

    def __init__(self, inst):
        self.n = int(inst.n)
        self.m = int(inst.m)
        n = self.n
        self.c_i = np.asarray(inst.c_i, np.int64)
        self.c_j = np.asarray(inst.c_j, np.int64)
        self.c_v = np.asarray(inst.c_v, np.float64)
        self.a_k = np.asarray(inst.a_k, np.int64)
        self.a_i = np.asarray(inst.a_i, np.int64)
        self.a_j = np.asarray(inst.a_j, np.int64)
        self.a_v = np.asarray(inst.a_v, np.float64)
        self.b = np.asarray(inst.b, np.float64)
        self.lr_u = np.asarray(inst.c_lr_u, np.float64).reshape(-1, n) if inst.c_lr_k else np.zeros((0, n))
        self.lr_s = np.asarray(inst.c_lr_s, np.float64).reshape(-1)
        assert np.all(self.c_i <= self.c_j) and np.all(self.a_i <= self.a_j)
        # kappa: weight of an upper entry in the trace inner product
        self.c_kappa = np.where(self.c_i == self.c_j, 1.0, 2.0)
        self.a_kappa = np.where(self.a_i == self.a_j, 1.0, 2.0)
        self.C_sparse = _sym_from_upper(n, self.c_i, self.c_j, self.c_v)
        self.norm_b = float(np.linalg.norm(self.b))
        self.norm_C = _frobenius_C(self)


def _sym_from_upper(n, i, j, v):
    """Symmetric scipy matrix with M_ij = M_ji = v for each upper entry (duplicates add)."""
    off = i != j
    rows = np.concatenate([i, j[off]])
    cols = np.concatenate([j, i[off]])
    vals = np.concatenate([v, v[off]])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def _frobenius_C(P: OracleProblem) -> float:
    """||C||_F of C = C_sparse + sum_l s_l u_l u_l^T (KKT denominator, Sec. 6)."""
    Cs = P.C_sparse
    t = float(Cs.multiply(Cs).sum())
    if P.lr_s.size:
        U, s = P.lr_u, P.lr_s
        # <C_s, u_l u_l^T> = u_l^T C_s u_l ; <u_l u_l^T, u_q u_q^T> = (u_l . u_q)^2
        t += 2.0 * sum(s[l] * float(U[l] @ (Cs @ U[l])) for l in range(s.size))
        G = U @ U.T
        t += float(s @ (G * G) @ s)
    return math.sqrt(max(t, 0.0))


# ----------------------------------------------------------------------------------
# constraint map, cost, adjoint  (Sec. 1.2: [A(X)]_k = <A_k, X>, A^* its adjoint)
# ----------------------------------------------------------------------------------
def _xe(U, V, i, j):
    """Entries X_ij of the symmetric X = (U V^T + V U^T)/2 at index arrays i, j."""
    if U is V:
        return np.einsum("ec,ec->e", U[i], U[j])
    return 0.5 * (np.einsum("ec,ec->e", U[i], V[j]) + np.einsum("ec,ec->e", V[i], U[j]))


def amap(P: OracleProblem, U, V=None) -> np.ndarray:
    """A(X) for X = U U^T, or X = (U V^T + V U^T)/2 when V is given."""
    V = U if V is None else V
    x = _xe(U, V, P.a_i, P.a_j)
    return np.bincount(P.a_k, weights=P.a_kappa * P.a_v * x, minlength=P.m).astype(np.float64)


def cost(P: OracleProblem, U, V=None) -> float:
    """<C, X> for X = U U^T (or the symmetrised U V^T), sparse part plus the low-rank part."""
    V = U if V is None else V
    x = _xe(U, V, P.c_i, P.c_j)
    c = float(np.sum(P.c_kappa * P.c_v * x))
    for l in range(P.lr_s.size):
        u = P.lr_u[l]
        c += P.lr_s[l] * float((U.T @ u) @ (V.T @ u))
    return c


def adjoint(P: OracleProblem, w) -> sp.csr_matrix:
    """A^*(w) = sum_k w_k A_k as a sparse symmetric matrix."""
    vals = np.asarray(w, np.float64)[P.a_k] * P.a_v
    return _sym_from_upper(P.n, P.a_i, P.a_j, vals)


def slack_sparse(P: OracleProblem, w) -> sp.csr_matrix:
    """Sparse part of Z(w) = C - A^*(w) (the low-rank part of C is kept apart)."""
    return (P.C_sparse - adjoint(P, w)).tocsr()


def slack_matvec(P: OracleProblem, S_sparse, V):
    """Z(w) V = S_sparse V + sum_l s_l u_l (u_l^T V)."""
    out = S_sparse @ V
    for l in range(P.lr_s.size):
        u = P.lr_u[l]
        if np.ndim(V) == 2:
            out = out + P.lr_s[l] * np.outer(u, u @ V)
        else:
            out = out + P.lr_s[l] * u * (u @ V)
    return out


def slack_dense(P: OracleProblem, w) -> np.ndarray:
    """Z(w) as a dense matrix (small n only)."""
    S = slack_sparse(P, w).toarray()
    for l in range(P.lr_s.size):
        S += P.lr_s[l] * np.outer(P.lr_u[l], P.lr_u[l])
    return S


# ----------------------------------------------------------------------------------
# augmented Lagrangian and its gradient  (Eq. AL, Eq. AL-BM, Sec. 4.2)
# ----------------------------------------------------------------------------------
def aug_lagrangian(P: OracleProblem, R, y, sigma) -> float:
    """L_sigma(RR^T, y) = <C, X> + <y, b - A(X)> + sigma/2 ||A(X) - b||^2."""
    res = amap(P, R) - P.b
    return cost(P, R) - float(np.dot(y, res)) + 0.5 * sigma * float(np.dot(res, res))


def dual_candidate(P: OracleProblem, R, y, sigma) -> np.ndarray:
    """w = y + sigma (b - A(RR^T)): the ALM multiplier update (Eq. ALM)."""
    return np.asarray(y, np.float64) - sigma * (amap(P, R) - P.b)


def gradient(P: OracleProblem, R, y, sigma) -> np.ndarray:
    """grad_R L_sigma(RR^T, y) = 2 Z(w) R with w the ALM update of y (Sec. 4.2:
    grad h(F) = 2 grad f(FF^T) F, and grad_X L_sigma = C - A^*(w))."""
    w = dual_candidate(P, R, y, sigma)
    return 2.0 * slack_matvec(P, slack_sparse(P, w), R)


def precondition(P: OracleProblem, R, y, sigma, G) -> np.ndarray:
    """Z = P^{-1} G for the row-block Jacobi preconditioner of the inner CG.

    The Hessian of L_sigma(RR^T, y) in R has, in the block of row i, the part
    2 S_ii I + 4 sigma a_i^2 r_i r_i^T (S_ii = Z(w)_ii of the sparse part of C; a_i the
    coefficient of a constraint a_i e_i e_i^T on X_ii alone, 0 if there is none).  P_i is
    that block with S_ii floored at 1e-2 (1 + mean |C_ii|); Z_i = P_i^{-1} g_i by
    Sherman-Morrison.  (A heuristic of this implementation; the paper leaves the inner
    first-order method open.)"""
    n = P.n
    w = dual_candidate(P, R, y, sigma)
    S = slack_sparse(P, w)
    s = np.asarray(S.diagonal(), np.float64).copy()
    cdiag = np.zeros(n)
    np.add.at(cdiag, P.c_i[P.c_i == P.c_j], P.c_v[P.c_i == P.c_j])
    floor = 1e-2 * (1.0 + float(np.mean(np.abs(cdiag))))
    s = np.maximum(s, floor)
    # coefficient of the single-entry constraints on diagonal entries
    counts = np.bincount(P.a_k, minlength=P.m)
    a = np.zeros(n)
    diag_sel = (P.a_i == P.a_j) & (counts[P.a_k] == 1)
    first = np.full(n, False)
    for e in np.nonzero(diag_sel)[0]:
        i = P.a_i[e]
        if not first[i]:
            a[i] = P.a_v[e]
            first[i] = True
    ka = 4.0 * sigma * a * a
    rg = np.einsum("ij,ij->i", R, G)
    rr = np.einsum("ij,ij->i", R, R)
    coef = ka * rg / (2.0 * s + ka * rr)
    return (G - coef[:, None] * R) / (2.0 * s)[:, None]


# ----------------------------------------------------------------------------------
# exact line search on phi(alpha) = L_sigma((R + alpha D)(R + alpha D)^T, y)
# ----------------------------------------------------------------------------------
def quartic_coeffs(P: OracleProblem, R, D, y, sigma) -> np.ndarray:
    """Coefficients q0..q4 of phi(alpha) = sum_k q_k alpha^k.

    X(alpha) = RR^T + alpha (RD^T + DR^T) + alpha^2 DD^T, so with
    a0 = A(RR^T) - b, a1 = A(RD^T + DR^T), a2 = A(DD^T), c0 = <C,RR^T>,
    c1 = <C, RD^T + DR^T>, c2 = <C, DD^T>, expanding Eq. AL gives
      q0 = c0 - y.a0 + sigma/2 |a0|^2
      q1 = c1 - y.a1 + sigma a0.a1
      q2 = c2 - y.a2 + sigma (|a1|^2/2 + a0.a2)
      q3 = sigma a1.a2
      q4 = sigma/2 |a2|^2
    """
    y = np.asarray(y, np.float64)
    a0 = amap(P, R) - P.b
    a1 = 2.0 * amap(P, R, D)          # A(RD^T + DR^T) = 2 A(sym(R D^T))
    a2 = amap(P, D)
    c0 = cost(P, R)
    c1 = 2.0 * cost(P, R, D)
    c2 = cost(P, D)
    return np.array([
        c0 - y @ a0 + 0.5 * sigma * (a0 @ a0),
        c1 - y @ a1 + sigma * (a0 @ a1),
        c2 - y @ a2 + sigma * (0.5 * (a1 @ a1) + a0 @ a2),
        sigma * (a1 @ a2),
        0.5 * sigma * (a2 @ a2),
    ])


def quartic_value(q, alpha):
    return q[0] + alpha * (q[1] + alpha * (q[2] + alpha * (q[3] + alpha * q[4])))


def exact_step(q) -> float:
    """alpha* = argmin_{alpha >= 0} phi(alpha) over the real critical points of phi
    (roots of phi' = 4q4 a^3 + 3q3 a^2 + 2q2 a + q1, found by numpy.roots), the
    smallest alpha among equal minima; alpha = 0 when no positive critical point
    lowers phi.  Returns +inf when phi is unbounded below on alpha >= 0."""
    q = np.asarray(q, np.float64)
    if q[4] < 0 or (q[4] == 0 and (q[3] < 0 or (q[3] == 0 and (q[2] < 0 or (q[2] == 0 and q[1] < 0))))):
        return math.inf
    coeffs = np.array([4 * q[4], 3 * q[3], 2 * q[2], q[1]])
    nz = np.nonzero(coeffs)[0]
    if nz.size == 0:
        return 0.0
    roots = np.roots(coeffs[nz[0]:]) if nz[0] < 3 else np.array([])
    scale = max(1.0, float(np.max(np.abs(roots)))) if roots.size else 1.0
    cand = [float(z.real) for z in roots if abs(z.imag) <= 1e-9 * scale and z.real > 0]
    best_a, best_v = 0.0, quartic_value(q, 0.0)
    for a in sorted(cand):
        v = quartic_value(q, a)
        if v < best_v:
            best_a, best_v = a, v
    return best_a


# ----------------------------------------------------------------------------------
# smallest eigenpair of Z(w)  (Alg. 1: eigenvectors of grad_X L; Sec. 6 KKT)
# ----------------------------------------------------------------------------------
def lanczos_min(matvec, n, k=32, tol=1e-10, max_restarts=400, seed=0, norm_est=None):
    """Smallest eigenpair of a symmetric operator by Lanczos with full
    reorthogonalisation (classical Gram-Schmidt, applied twice), restarted from
    the current Ritz vector; stops when ||A v - theta v|| <= tol * ||A||_est.
    Returns (theta, v, residual_norm, matvecs)."""
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(n)
    q /= np.linalg.norm(q)
    theta, v, res, nmv = 0.0, q, math.inf, 0
    anorm = norm_est or 0.0
    for _ in range(max_restarts):
        kk = min(k, n)
        Q = np.zeros((n, kk + 1))
        alpha = np.zeros(kk)
        beta = np.zeros(kk)
        Q[:, 0] = q
        m = kk
        for j in range(kk):
            z = matvec(Q[:, j])
            nmv += 1
            for _pass in range(2):
                h = Q[:, : j + 1].T @ z
                z = z - Q[:, : j + 1] @ h
                if _pass == 0:
                    alpha[j] = h[j]
                else:
                    alpha[j] += h[j]
            beta[j] = np.linalg.norm(z)
            anorm = max(anorm, abs(alpha[j]) + beta[j] + (beta[j - 1] if j else 0.0))
            if beta[j] <= 1e-14 * max(anorm, 1e-300):
                m = j + 1
                break
            Q[:, j + 1] = z / beta[j]
        evals, evecs = scipy.linalg.eigh_tridiagonal(alpha[:m], beta[: m - 1])
        theta = float(evals[0])
        s = evecs[:, 0]
        v = Q[:, :m] @ s
        v /= np.linalg.norm(v)
        r = matvec(v) - theta * v
        nmv += 1
        res = float(np.linalg.norm(r))
        if res <= tol * max(anorm, 1e-300):
            break
        q = v
    return theta, v, res, nmv


def lambda_min(P: OracleProblem, w, dense_max=1500, k=32, tol=1e-10, seed=0):
    """(lambda_min(Z(w)), unit eigenvector, residual).  Dense symmetric
    eigendecomposition for n <= dense_max, Lanczos above."""
    if P.n <= dense_max:
        evals, evecs = np.linalg.eigh(slack_dense(P, w))
        v = evecs[:, 0]
        return float(evals[0]), v, 0.0
    S = slack_sparse(P, w)
    est = float(abs(S).sum(axis=1).max()) + float(np.sum(np.abs(P.lr_s) * np.sum(P.lr_u ** 2, axis=1)))
    theta, v, res, _ = lanczos_min(lambda x: slack_matvec(P, S, x), P.n, k=k, tol=tol, seed=seed, norm_est=est)
    return theta, v, res


def growth_step(P: OracleProblem, lam, v, sigma):
    """Step size s* >= 0 of the rank-one negative-curvature move X + s v v^T
    (Alg. 1's small SDP restricted to one vector): L is quadratic in X, so
    L(X + s vv^T) = L(X) + s v^T Z(w) v + s^2 sigma/2 ||A(vv^T)||^2 and
    s* = -lambda / (sigma ||A(vv^T)||^2).  Returns inf when A(vv^T) = 0."""
    av = amap(P, v.reshape(-1, 1))
    den = sigma * float(av @ av)
    if den <= 0.0:
        return math.inf
    return max(0.0, -lam / den)


def lbfgs_direction(G, pairs):
    """H G for the L-BFGS inverse-Hessian estimate H built from the (s, y) pairs (oldest
    first) by the two-loop recursion of Nocedal (1980), initial scaling s.y / y.y of the
    newest pair; G itself when there is no pair.  Matrices are treated as vectors."""
    q = np.array(G, copy=True)
    al = []
    for sk, yk in reversed(pairs):
        rho = 1.0 / float(np.sum(yk * sk))
        a = rho * float(np.sum(sk * q))
        q -= a * yk
        al.append((a, rho, sk, yk))
    if pairs:
        sk, yk = pairs[-1]
        q *= float(np.sum(sk * yk)) / float(np.sum(yk * yk))
    for a, rho, sk, yk in reversed(al):
        b = rho * float(np.sum(yk * q))
        q += (a - b) * sk
    return q


def _proj_psd(S):
    """Nearest positive semidefinite matrix in the Frobenius norm (clip the eigenvalues)."""
    S = 0.5 * (S + S.T)
    ev, Q = np.linalg.eigh(S)
    return (Q * np.maximum(ev, 0.0)) @ Q.T


def block_growth_map(P: OracleProblem, V):
    """The linear map S -> A(V S V^T) for symmetric k x k S, as an m x k^2 matrix acting on
    vec(S) (row-major): column (a, b) is A((v_a v_b^T + v_b v_a^T)/2)."""
    k = V.shape[1]
    M = np.zeros((P.m, k * k))
    for a in range(k):
        for b in range(k):
            M[:, a * k + b] = amap(P, V[:, [a]], V[:, [b]])
    return M


def block_growth_step(P: OracleProblem, lams, V, sigma, iters=20000, tol=1e-13):
    """Alg. 1's small SDP along the negative-curvature directions: with V (n x k) the
    orthonormal eigenvectors of Z(w) = grad_X L for the eigenvalues lams,
    S* = argmin_{S >= 0} L(X + V S V^T) - L(X) = <diag(lams), S> + sigma/2 ||A(V S V^T)||^2
    (exact: L is quadratic in X and V^T Z(w) V = diag(lams)).  A convex quadratic over the
    k x k PSD cone, solved by projected gradient with step 1/Lip, Lip = sigma ||M^T M||.
    Returns None when A(V S V^T) can vanish along a direction of negative curvature (L
    unbounded below)."""
    lams = np.asarray(lams, np.float64)
    k = lams.size
    M = block_growth_map(P, V)
    H = M.T @ M
    Lip = sigma * float(np.linalg.eigvalsh(0.5 * (H + H.T)).max()) if k else 0.0
    if not Lip > 0.0:
        return None
    Lam = np.diag(lams)
    S = np.zeros((k, k))
    for _ in range(iters):
        grad = Lam + sigma * (H @ S.reshape(-1)).reshape(k, k)
        S_new = _proj_psd(S - 0.5 * (grad + grad.T) / Lip)
        if np.linalg.norm(S_new - S) <= tol * max(1.0, np.linalg.norm(S)):
            S = S_new
            break
        S = S_new
    return S


def psd_sqrt(S):
    """Symmetric square root of a PSD matrix (eigenvalues clipped at 0)."""
    ev, Q = np.linalg.eigh(0.5 * (S + S.T))
    return (Q * np.sqrt(np.maximum(ev, 0.0))) @ Q.T


# ----------------------------------------------------------------------------------
# termination measure  (Sec. 6, "Termination criteria")
# ----------------------------------------------------------------------------------
def kkt(P: OracleProblem, R, y, lam_dual):
    """(primal, dual, gap) terms of the relative KKT error with l2 norms:
    ||A(X)-b||/(1+||b||), |min(0, lambda_min(C - A^* y))|/(1+||C||_F),
    |<C,X> - b^T y|/(1+|<C,X>|+|b^T y|)."""
    res = amap(P, R) - P.b
    cx = cost(P, R)
    by = float(P.b @ y)
    p = float(np.linalg.norm(res)) / (1.0 + P.norm_b)
    d = abs(min(0.0, lam_dual)) / (1.0 + P.norm_C)
    g = abs(cx - by) / (1.0 + abs(cx) + abs(by))
    return p, d, g


# ----------------------------------------------------------------------------------
# ALORA (Alg. 1) with gradient descent + exact line search as the inner solver
# ----------------------------------------------------------------------------------
@dataclass
class SolveOptions:
    sigma: float = 1.0
    eps: float = 1e-6
    r_max: int = 32
    max_outer: int = 200
    max_inner: int = 5000
    inner_method: str = "cg"    # "cg": Polak-Ribiere+ directions; "gd": D = -G; "lbfgs": L-BFGS
    lbfgs_m: int = 8            # L-BFGS memory (pairs kept)
    inner_precond: str = "block_jacobi"  # "none" | "block_jacobi" (row blocks of the Hessian)
    inner_rel: float = 0.1      # tau_in = max(inner_floor*eps, min(inner_rel*KKT_prev, inner_decay*tau_in_prev))
    inner_decay: float = 0.7
    sigma_rule: str = "fixed"   # "fixed" | "adaptive": sigma <- min(2 sigma, sigma_max) when the
    sigma_max: float = 1e6      # primal term fell by less than a factor 4 since the last KKT test
    inner_floor: float = 0.1
    inner_start: float = 1e-1   # tau_in before the first KKT value exists
    dense_max: int = 1500
    lanczos_k: int = 32
    growth_k: int = 1           # directions per rank-growth step (Alg. 1 uses r; > 1 needs n <= dense_max)
    lanczos_tol: float = 1e-10
    seed: int = 0
    log: bool = False


@dataclass
class SolveResult:
    R: np.ndarray
    y: np.ndarray
    objective: float            # <C, X>
    kkt: tuple
    outer: int
    inner_total: int
    rank: int
    history: list = field(default_factory=list)
    sigma: float = 1.0


def solve(P: OracleProblem, R0, y0=None, opts: SolveOptions | None = None) -> SolveResult:
    """ALORA (Alg. 1): repeat { inner solve of (AL-BM) at fixed y; smallest
    eigenpair of grad_X L; rank-one growth along it if lambda_min < -tau_lambda;
    y <- y + sigma (b - A(RR^T)) } until KKT <= eps (Sec. 6).

    Readings of what the paper leaves open: the inner solver is a first-order
    method with the exact quartic line search -- gradient descent (Eq. GD) or
    nonlinear conjugate gradients with the Polak-Ribiere+ rule
    beta = max(0, <G, G - G_prev>/<G_prev, G_prev>), D = -G + beta D_prev
    (reset to -G when D is not a descent direction), optionally on the preconditioned
    gradient Z = P^{-1} G of `precondition` (then beta = max(0, (<Z,G> - <G,Z_prev>)/<Z_prev,G_prev>),
    D = -Z + beta D_prev) -- stopped when ||G||_F/(1+||C||_F) <= tau_in
    with tau_in = max(inner_floor*eps, min(inner_rel*KKT_prev, inner_decay*tau_in_prev))
    (so that tau_in falls every outer iteration even when the KKT value stalls), or when the step is 0,
    or after max_inner steps; tau_lambda = eps (1 + ||C||_F); one eigenvector per
    outer iteration; the KKT test is taken only in outer iterations without growth
    (its dual term is then lambda_min(Z(w)) at w = the updated y)."""
    opts = opts or SolveOptions()
    R = np.array(R0, np.float64, copy=True)
    y = np.zeros(P.m) if y0 is None else np.array(y0, np.float64, copy=True)
    sigma = opts.sigma
    tau_lam = opts.eps * (1.0 + P.norm_C)
    kkt_prev = None
    p_prev = math.inf
    inner_total = 0
    hist = []
    terms = (math.inf, math.inf, math.inf)
    outer = 0
    for outer in range(1, opts.max_outer + 1):
        if outer == 1:
            tau_in = opts.inner_start
        else:
            cap = opts.inner_decay * tau_in
            if kkt_prev is not None:
                cap = min(cap, opts.inner_rel * kkt_prev)
            tau_in = max(opts.inner_floor * opts.eps, cap)
        # --- inner solve (Alg. 1 line "F <- argmin L") -------------------------
        it = 0
        G_prev = Z_prev = D_prev = None
        pairs = []  # L-BFGS (s, y) pairs of this inner solve
        while it < opts.max_inner:
            G = gradient(P, R, y, sigma)
            gn = float(np.linalg.norm(G))
            if gn / (1.0 + P.norm_C) <= tau_in:
                break
            if opts.inner_method == "lbfgs":
                if G_prev is not None:
                    sk, yk = alpha * D_prev, G - G_prev
                    if float(np.sum(sk * yk)) > 1e-12 * float(np.linalg.norm(sk) * np.linalg.norm(yk)):
                        pairs.append((sk, yk))
                        pairs = pairs[-opts.lbfgs_m:]
                D = -lbfgs_direction(G, pairs)
                if float(np.sum(D * G)) >= 0.0:
                    D, pairs = -G, []
                q = quartic_coeffs(P, R, D, y, sigma)
                alpha = exact_step(q)
                if not math.isfinite(alpha):
                    raise FloatingPointError("augmented Lagrangian unbounded along the direction")
                if alpha == 0.0:
                    break
                R = R + alpha * D
                G_prev, D_prev = G, D
                it += 1
                continue
            Z = precondition(P, R, y, sigma, G) if opts.inner_precond == "block_jacobi" else G
            D = -Z
            if opts.inner_method == "cg" and G_prev is not None:
                beta = max(0.0, (float(np.sum(Z * G)) - float(np.sum(G * Z_prev)))
                           / float(np.sum(Z_prev * G_prev)))
                D = -Z + beta * D_prev
                if float(np.sum(D * G)) >= 0.0:
                    D = -Z
            q = quartic_coeffs(P, R, D, y, sigma)
            alpha = exact_step(q)
            if not math.isfinite(alpha):
                raise FloatingPointError("augmented Lagrangian unbounded along the gradient")
            if alpha == 0.0:
                break
            R = R + alpha * D
            G_prev, Z_prev, D_prev = G, Z, D
            it += 1
        inner_total += it
        # --- spectral information of grad_X L at X = RR^T ----------------------
        w = dual_candidate(P, R, y, sigma)
        lam, v, _ = lambda_min(P, w, dense_max=opts.dense_max, k=opts.lanczos_k,
                               tol=opts.lanczos_tol, seed=opts.seed + outer)
        grew = False
        if lam < -tau_lam and R.shape[1] < opts.r_max:
            kk = min(opts.growth_k, opts.r_max - R.shape[1])
            if kk > 1 and P.n <= opts.dense_max:
                # Alg. 1 with several directions: the eigenvectors whose eigenvalues are
                # below -tau_lambda, the k x k SDP for S, R <- [R, V S^{1/2}]
                ev, Q = np.linalg.eigh(slack_dense(P, w))
                sel = np.nonzero(ev[:kk] < -tau_lam)[0]
                S = block_growth_step(P, ev[sel], Q[:, sel], sigma)
                if S is None:
                    raise FloatingPointError("augmented Lagrangian unbounded along the eigenvectors")
                R = np.hstack([R, Q[:, sel] @ psd_sqrt(S)])
            else:
                s = growth_step(P, lam, v, sigma)
                if not math.isfinite(s):
                    raise FloatingPointError("augmented Lagrangian unbounded along the eigenvector")
                R = np.hstack([R, math.sqrt(s) * v.reshape(-1, 1)])
            grew = True
        # --- dual update (Eq. ALM) ---------------------------------------------
        y = dual_candidate(P, R, y, sigma)
        if grew:
            hist.append(dict(outer=outer, inner=it, rank=R.shape[1], lam=lam, grew=True))
            continue
        terms = kkt(P, R, y, lam)
        if opts.sigma_rule == "adaptive" and kkt_prev is not None and terms[0] > 0.25 * p_prev:
            sigma = min(2.0 * sigma, opts.sigma_max)
        p_prev = terms[0]
        kkt_prev = max(terms)
        hist.append(dict(outer=outer, inner=it, rank=R.shape[1], lam=lam, grew=False, kkt=terms))
        if opts.log:
            print(f"outer {outer:4d} inner {it:5d} r {R.shape[1]:2d} lam {lam:+.3e} kkt {terms}")
        if kkt_prev <= opts.eps:
            break
    return SolveResult(R=R, y=y, objective=cost(P, R), kkt=terms, outer=outer,
                       inner_total=inner_total, rank=R.shape[1], history=hist, sigma=sigma)
