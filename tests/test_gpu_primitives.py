"""GPU parity of the four hot-path primitives (through the C-ABI) against the FP64
oracle on the same seeded inputs, element by element.

Bar: FP64 within 1e-12 relative, FP32 within 1e-5 relative (relative to the largest
magnitude of the compared quantity)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import sdp_instances as si  # noqa: E402
from gpu_common import RTOL, as_np, dual_for, factor_for, instances_small, rel_err  # noqa: E402

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2505_15775_gb300 import alm  # noqa: E402

INSTANCES = instances_small()
CASES = [(name, r, prec) for name in INSTANCES for r in (1, 3, 8, 13, 32) for prec in (0, 1)]


@pytest.fixture(scope="module")
def handles():
    hs = {}
    yield hs
    for h in hs.values():
        alm.alm_destroy(h)


def _handle(handles, name, prec):
    key = (name, prec)
    if key not in handles:
        handles[key] = alm.alm_create(INSTANCES[name], precision=prec)
    return handles[key]


def _inputs(name, r, seed=0):
    inst = INSTANCES[name]
    P = O.OracleProblem(inst)
    R = factor_for(inst, r, 100 + r + seed)
    y = dual_for(inst, 7 + seed)
    return inst, P, R, y


@pytest.mark.parametrize("name,r,prec", CASES)
def test_eval_parity(handles, name, r, prec):
    inst, P, R, y = _inputs(name, r)
    h = _handle(handles, name, prec)
    sigma = 1.3
    Rd = alm.factor_tensor(h, R)
    Rq = as_np(Rd)[:, :r]            # the values the GPU sees (rounded in FP32 mode)
    L, AX, CX = alm.alm_eval(h, Rd, r, y, sigma)
    ax_o = O.amap(P, Rq)
    assert rel_err(as_np(AX), ax_o) <= RTOL[prec]
    assert CX == pytest.approx(O.cost(P, Rq), rel=RTOL[prec], abs=RTOL[prec])
    Lo = O.aug_lagrangian(P, Rq, y, sigma)
    scale = max(1.0, abs(Lo), abs(O.cost(P, Rq)), float(np.abs(y) @ np.abs(ax_o - P.b)))
    assert abs(L - Lo) <= RTOL[prec] * scale


@pytest.mark.parametrize("name,r,prec", CASES)
def test_grad_parity(handles, name, r, prec):
    inst, P, R, y = _inputs(name, r)
    h = _handle(handles, name, prec)
    sigma = 0.7
    Rd = alm.factor_tensor(h, R)
    Rq = as_np(Rd)[:, :r]
    G, g2 = alm.alm_grad(h, Rd, r, y, sigma)
    Go = O.gradient(P, Rq, y, sigma)
    Gg = as_np(G)
    assert np.all(Gg[:, r:] == 0.0)
    # scale: the magnitude of the terms summed into each entry
    w = O.dual_candidate(P, Rq, y, sigma)
    scale = max(1.0, float(np.max(np.abs(Go))), 2 * float(np.max(np.abs(O.slack_sparse(P, w)).sum(axis=1))) *
                float(np.max(np.abs(Rq))))
    assert rel_err(Gg[:, :r], Go, scale) <= RTOL[prec]
    assert g2 == pytest.approx(float(np.sum(Go * Go)), rel=10 * RTOL[prec] + 1e-14, abs=RTOL[prec] * scale ** 2)


@pytest.mark.parametrize("name,r,prec", CASES)
def test_linesearch_parity(handles, name, r, prec):
    inst, P, R, y = _inputs(name, r)
    h = _handle(handles, name, prec)
    sigma = 1.1
    rng = np.random.default_rng(r)
    D = rng.standard_normal(R.shape) * float(np.std(R))
    Rd = alm.factor_tensor(h, R)
    Dd = alm.factor_tensor(h, D)
    Rq, Dq = as_np(Rd)[:, :r], as_np(Dd)[:, :r]
    q, alpha = alm.alm_linesearch(h, Rd, Dd, r, y, sigma)
    qo = O.quartic_coeffs(P, Rq, Dq, y, sigma)
    # each coefficient against the magnitude of the products it sums
    a0 = O.amap(P, Rq) - P.b
    a1 = 2 * O.amap(P, Rq, Dq)
    a2 = O.amap(P, Dq)
    mag = max(1.0, float(np.abs(qo).max()), float(np.abs(y) @ (np.abs(a1) + np.abs(a2))),
              sigma * float(np.abs(a0) @ (np.abs(a1) + np.abs(a2))), sigma * float(a1 @ a1 + a2 @ a2))
    assert rel_err(q, qo, mag) <= 4 * RTOL[prec]
    # the step minimises the device's own quartic; compare phi values under the oracle's quartic
    ao = O.exact_step(qo)
    if prec == 0:
        assert alpha == pytest.approx(ao, rel=1e-9, abs=1e-12)
    else:
        assert O.quartic_value(qo, alpha) <= O.quartic_value(qo, ao) + 1e-5 * mag * max(1.0, ao) ** 4


def test_linesearch_along_negative_gradient_descends(handles):
    inst, P, R, y = _inputs("maxcut-er-800", 8)
    h = _handle(handles, "maxcut-er-800", 0)
    Rd = alm.factor_tensor(h, R)
    G, _ = alm.alm_grad(h, Rd, 8, y, 1.0)
    q, alpha = alm.alm_linesearch(h, Rd, -G, 8, y, 1.0)
    assert alpha > 0
    L0, _, _ = alm.alm_eval(h, Rd, 8, y, 1.0, want_ax=False)
    L1, _, _ = alm.alm_eval(h, Rd - alpha * G, 8, y, 1.0, want_ax=False)
    assert L1 < L0
    assert L1 == pytest.approx(O.quartic_value(q, alpha), rel=1e-11)


@pytest.mark.parametrize("name", list(INSTANCES))
@pytest.mark.parametrize("prec", [0, 1])
def test_lambda_min_parity(handles, name, prec):
    inst, P, R, y = _inputs(name, 5)
    h = _handle(handles, name, prec)
    sigma = 0.9
    Rd = alm.factor_tensor(h, R)
    Rq = as_np(Rd)[:, :5]
    lam, v, res = alm.alm_lambda_min(h, Rd, 5, y, sigma)
    w = O.dual_candidate(P, Rq, y, sigma)
    S = O.slack_dense(P, w)
    ev = np.linalg.eigvalsh(S)
    snorm = float(np.abs(ev).max())
    vv = as_np(v)
    assert abs(np.linalg.norm(vv) - 1.0) < (1e-5 if prec else 1e-12)
    true_res = float(np.linalg.norm(S @ vv - lam * vv))
    tol = 1e-7 if prec == 0 else 2e-4
    assert true_res <= tol * snorm + 1e-12
    # Rayleigh quotient >= lambda_min (up to the rounding of the working precision);
    # within the residual bound of it
    assert lam >= ev[0] - (1e-9 if prec == 0 else 1e-6) * snorm
    assert lam - ev[0] <= max(10 * true_res, 1e-8 * snorm) or abs(lam - ev[0]) <= tol * snorm


def test_lambda_min_closed_form_torus(handles):
    """R = 0, y = 0, unit torus: lambda_min(-L/4 - sigma I) = -2 - sigma."""
    inst = si.torus_maxcut(12, 16, weights="unit")
    h = alm.alm_create(inst, precision=0)
    try:
        for sigma in (0.5, 2.0):
            lam, v, res = alm.alm_lambda_min(h, None, 0, np.zeros(inst.m), sigma)
            assert lam == pytest.approx(-2.0 - sigma, abs=1e-9)
    finally:
        alm.alm_destroy(h)


def test_spurious_example_eigen_and_gradient(handles):
    """Sec. 4.3 example: zero gradient, lambda_min(grad_X L) = -eps with eigenvector e_d."""
    d, eps, k, eta = 9, 0.1, 4, 0.5
    inst = si.t15_instance(d, eps, eta ** 2 * k)
    h = alm.alm_create(inst, precision=0)
    try:
        y = np.zeros(d)
        y[-1] = 2.0
        F = np.zeros((d, k))
        F[:k, :k] = eta * np.eye(k)
        Fd = alm.factor_tensor(h, F)
        G, g2 = alm.alm_grad(h, Fd, k, y, 4.0)
        assert g2 <= 1e-28
        lam, v, res = alm.alm_lambda_min(h, Fd, k, y, 4.0)
        assert lam == pytest.approx(-eps, abs=1e-12)
        assert abs(abs(as_np(v)[-1]) - 1) < 1e-10
    finally:
        alm.alm_destroy(h)


def test_invalid_arguments_are_rejected(handles):
    h = _handle(handles, "maxcut-er-800", 0)
    R = alm.factor_tensor(h, np.ones((800, 3)))          # ldr = 4 doubles
    lib = alm.load()
    # ldr * 8 bytes not a multiple of 16
    st = lib.alm_eval(h.ptr, alm.C.c_void_p(R.data_ptr()), 3, 3, None, 1.0, None, None, None)
    assert st == alm.ALM_ERR_INVALID_ARG
    assert b"16 bytes" in lib.alm_last_error(h.ptr)
    with pytest.raises(alm.AlmError) as e:
        alm.alm_eval(h, R, 40, None, 1.0)                 # rank above the cap
    assert e.value.status == alm.ALM_ERR_INVALID_ARG
    with pytest.raises(alm.AlmError):
        alm.alm_eval(h, R, 3, None, -1.0)                 # negative penalty
