"""Parity at the benchmark's sizes.

* One inner step of the solver's fused inner loop -- the step + SpMM kernel and the
  direction + line-search kernel, run through alm_cg_step with the launch shape the
  benchmark uses -- from a seeded state (R, D, Z_old, y, alpha, zg_prev), FP32 form,
  r = 32, at n = 1e6 (the benchmark's 1000 x 1000 torus) and n = 1e7 (the random
  3-regular graph), against the FP64 oracle on the same inputs: R' = R + alpha D,
  diag(S), Z = P^{-1} G (oracle.gradient, oracle.precondition), the CG inner products,
  the Polak-Ribiere+ beta, D_new = -Z + beta D, and the quartic of the exact step along
  D_new (oracle.quartic_coeffs, oracle.exact_step).  Every element of R', Z and D_new is
  compared, at the FP32 bar of 1e-5 relative to the largest entry.
* The largest instance (n about 4,096) of the 4096-instance batch generator, solved by
  the persistent batch kernel: the oracle's KKT of its (R, y), with a dense eigensolver
  for the dual term, at 1e-6.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import sdp_instances as si  # noqa: E402
from gpu_common import as_np, rel_err  # noqa: E402

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2505_15775_gb300 import alm  # noqa: E402

ALPHA, SIGMA, ZG_PREV = 0.3, 10.0, 2.0
BENCH_SHAPE = dict(variant=1, stages=2, threads=128)


def _state(n, seed):
    """Seeded FP32 state of an inner step: unit rows (the MaxCut constraint holds), a
    direction and a previous preconditioned gradient of moderate size, a dual in [-3, -2].
    With these S_ii = C_ii - y_i + sigma (|r_i'|^2 - 1) stays in about [0.7, 4.3], away from
    the preconditioner's floor, where 1 / (2 S_ii) would amplify the FP32 rounding of R'
    itself beyond the bar (a property of the state, not of the kernels)."""
    rng = np.random.default_rng(seed)
    R = si.factor_init(n, 32, (seed, 7))
    R = (R / np.linalg.norm(R, axis=1, keepdims=True)).astype(np.float32)
    D = (0.05 * rng.standard_normal((n, 32))).astype(np.float32)
    Zold = (0.1 * rng.standard_normal((n, 32))).astype(np.float32)
    y = rng.uniform(-3.0, -2.0, n)
    return R, D, Zold, y


def _pr_beta(zg, go, gd, zg_prev):
    """Polak-Ribiere+ with the descent safeguard, as the solver documents it."""
    if zg_prev <= 0:
        return 0.0
    beta = max(0.0, (zg - go) / zg_prev)
    return 0.0 if -zg + beta * gd >= 0 else beta


def _check_step(inst, seed):
    R, D, Zold, y = _state(inst.n, seed)
    h = alm.alm_create(inst, precision=alm.ALM_FP32, sigma0=SIGMA)
    try:
        alm.alm_set_inner_shape(h, **BENCH_SHAPE)
        dev = lambda a: torch.as_tensor(a, device="cuda")
        Ro, Z, Dn, diag, sc = alm.alm_cg_step(h, dev(R), dev(D), dev(Zold), 32, dev(y), SIGMA, ALPHA, ZG_PREV)
        Ro, Z, Dn, diag = as_np(Ro), as_np(Z), as_np(Dn), as_np(diag)
    finally:
        alm.alm_destroy(h)
    # the oracle, in FP64, on the same seeded inputs
    P = O.OracleProblem(inst)
    R64, D64, Z64 = R.astype(np.float64), D.astype(np.float64), Zold.astype(np.float64)
    R1 = R64 + ALPHA * D64
    G = O.gradient(P, R1, y, SIGMA)
    Zo = O.precondition(P, R1, y, SIGMA, G)
    Sd = O.slack_sparse(P, O.dual_candidate(P, R1, y, SIGMA)).diagonal()
    gg, go, gd, zg = (float(np.sum(G * G)), float(np.sum(G * Z64)), float(np.sum(G * D64)), float(np.sum(Zo * G)))
    beta = _pr_beta(zg, go, gd, ZG_PREV)
    Dno = -Zo + beta * D64
    q = O.quartic_coeffs(P, R1, Dno, y, SIGMA)
    q[0] = 0.0  # L itself is not part of the step
    a_or = O.exact_step(q)

    assert rel_err(Ro, R1, float(np.abs(R1).max())) <= 1e-6
    # S_ii carries the FP32 rounding of R' (through sigma |r_i'|^2): the FP32 bar
    assert float(np.max(np.abs(diag - Sd) / np.maximum(1.0, np.abs(Sd)))) <= 1e-5
    assert rel_err(Z, Zo, float(np.abs(Zo).max())) <= 1e-5
    nG, nZ, nD = np.linalg.norm(G), np.linalg.norm(Z64), np.linalg.norm(D64)
    assert abs(sc["gg"] - gg) <= 1e-5 * gg
    assert abs(sc["go"] - go) <= 1e-5 * nG * nZ
    assert abs(sc["gd"] - gd) <= 1e-5 * nG * nD
    assert abs(sc["zg"] - zg) <= 1e-5 * abs(zg)
    assert abs(sc["beta"] - beta) <= 1e-5 * max(1.0, abs(beta))
    assert rel_err(Dn, Dno, float(np.abs(Dno).max())) <= 1e-5
    qg = np.array(sc["q"], np.float64)
    qg[0] = 0.0
    for t in np.linspace(0.0, 2.0 * max(a_or, 1e-3), 9):
        mag = sum(abs(q[k]) * t ** k for k in range(5))
        assert abs(O.quartic_value(qg, t) - O.quartic_value(q, t)) <= 1e-5 * mag
    assert abs(sc["alpha"] - a_or) <= 1e-4 * a_or
    return Ro, Z, Dn


def test_inner_step_at_1e6_torus():
    _check_step(si.torus_maxcut(1000, 1000, seed=2), seed=31)


def _host_ram_gb():
    import os

    try:
        return os.sysconf("SC_PHYS_PAGES") * os.sysconf("SC_PAGE_SIZE") / 2 ** 30
    except (ValueError, OSError, AttributeError):
        return 0.0


def test_inner_step_at_1e7_regular3():
    # the FP64 oracle holds about ten n x 32 matrices and the pattern gathers: ~40 GB
    if _host_ram_gb() < 96:
        pytest.skip("the FP64 oracle at n = 1e7 needs about 40 GB of host memory")
    _check_step(si.regular3_maxcut(10 ** 7, seed=4), seed=32)


def test_batch_instance_of_4096_rows_passes_the_oracle_kkt():
    specs = si.batch_specs(4096, seed=6)
    b = int(np.argmax([s[0] for s in specs]))
    n, p, sub = specs[b]
    inst = si.er_maxcut(n, p, seed=sub)
    hb = alm.alm_batch_create([inst], eps=1e-6, sigma0=10.0, r_max=32)
    try:
        R, rank = alm.batch_factor(hb, [si.factor_init(inst.n, 32, (b, 7))])
        y = torch.zeros(hb.rows, dtype=torch.float64, device="cuda")
        stats, per = alm.alm_batch_solve(hb, R, rank, y)
        torch.cuda.synchronize()
        Rb = as_np(R)[:, : int(rank[0])]
        yb = as_np(y)
    finally:
        alm.alm_batch_destroy(hb)
    assert n >= 4000 and stats["converged"] == 1, per
    P = O.OracleProblem(inst)
    lam = float(np.linalg.eigvalsh(O.slack_dense(P, yb))[0])
    assert max(O.kkt(P, Rb, yb, lam)) <= 1e-6
    assert O.cost(P, Rb) == pytest.approx(per[0]["objective"], rel=1e-6)
