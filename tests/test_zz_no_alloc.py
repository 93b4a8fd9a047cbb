"""The allocation-free gradient entry point (alm_grad_unitdiag_noalloc) against the
regular one (alm_grad on a handle of the same problem).

Callers that cannot call cudaMalloc (a fixed memory budget reserved up front, an
allocator that must not be re-entered) pass the problem as device CSR arrays they own;
the library then works in its file-scope scratch array only.  The file name makes
pytest collect it last.  It runs alone in a fresh process as well as after the others.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import sdp_instances as si  # noqa: E402
from gpu_common import RTOL, as_np, rel_err  # noqa: E402

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2505_15775_gb300 import alm  # noqa: E402


def _csr_of(inst, dtype):
    """Full symmetric CSR of the off-diagonal part of C and its diagonal (test-side data,
    in caller-owned device memory)."""
    n = inst.n
    off = inst.c_i != inst.c_j
    i = np.concatenate([inst.c_i[off], inst.c_j[off]]).astype(np.int64)
    j = np.concatenate([inst.c_j[off], inst.c_i[off]]).astype(np.int64)
    v = np.concatenate([inst.c_v[off], inst.c_v[off]])
    order = np.lexsort((j, i))
    i, j, v = i[order], j[order], v[order]
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, i + 1, 1)
    rowptr = np.cumsum(rowptr)
    cdiag = np.zeros(n)
    np.add.at(cdiag, inst.c_i[~off], inst.c_v[~off])
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    return (dev(rowptr, torch.int32), dev(j, torch.int32), dev(v, dtype), dev(cdiag, dtype),
            dev(inst.b, torch.float64))


@pytest.mark.parametrize("prec", [alm.ALM_FP64, alm.ALM_FP32])
@pytest.mark.parametrize("which", ["torus", "er"])
def test_noalloc_gradient_matches_alm_grad_twice(prec, which):
    inst = si.torus_maxcut(40, 53, seed=5) if which == "torus" else si.er_maxcut(900, 0.01, seed=8, weights="pm1")
    h = alm.alm_create(inst, precision=prec)
    try:
        dtype = torch.float64 if prec == alm.ALM_FP64 else torch.float32
        rowptr, col, val, cdiag, b = _csr_of(inst, dtype)
        rng = np.random.default_rng(11)
        for call, (r, sigma) in enumerate([(13, 0.7), (8, 2.5)]):   # two calls in a row
            R = alm.factor_tensor(h, si.factor_init(inst.n, r, (call, 3)))
            y = torch.as_tensor(rng.uniform(-1, 1, inst.m), dtype=torch.float64, device="cuda")
            G_ref, _ = alm.alm_grad(h, R, r, y, sigma)
            G = torch.full_like(R, float("nan"))
            alm.alm_grad_unitdiag_noalloc(prec, rowptr, col, val, cdiag, b, y, sigma, R, r, G)
            torch.cuda.synchronize()
            g, gref = as_np(G), as_np(G_ref)
            assert np.all(g[:, r:] == 0.0)
            scale = max(1.0, float(np.abs(gref).max()), 8.0 * float(np.abs(as_np(R)).max()))
            assert rel_err(g[:, :r], gref[:, :r], scale) <= RTOL[prec]
    finally:
        alm.alm_destroy(h)


@pytest.mark.parametrize("prec", [alm.ALM_FP64, alm.ALM_FP32])
def test_noalloc_wide_row_stride(prec):
    """r = 3 in rows of stride 32: the lanes of a row cover fewer vectors than the stride
    holds, so the columns beyond the lanes' reach must be zeroed by the extra store loop;
    the first r columns still equal alm_grad's."""
    inst = si.er_maxcut(700, 0.012, seed=9, weights="pm1")
    h = alm.alm_create(inst, precision=prec)
    try:
        dtype = torch.float64 if prec == alm.ALM_FP64 else torch.float32
        rowptr, col, val, cdiag, b = _csr_of(inst, dtype)
        r, ldr, sigma = 3, 32, 1.3
        y = torch.as_tensor(np.random.default_rng(12).uniform(-1, 1, inst.m), dtype=torch.float64, device="cuda")
        R = alm.factor_tensor(h, si.factor_init(inst.n, r, (5, 3)), ldr=ldr)
        G_ref, _ = alm.alm_grad(h, R, r, y, sigma)
        for _ in range(2):
            G = torch.full_like(R, float("nan"))
            alm.alm_grad_unitdiag_noalloc(prec, rowptr, col, val, cdiag, b, y, sigma, R, r, G)
            torch.cuda.synchronize()
            g, gref = as_np(G), as_np(G_ref)
            assert np.all(g[:, r:] == 0.0)
            scale = max(1.0, float(np.abs(gref).max()), 8.0 * float(np.abs(as_np(R)).max()))
            assert rel_err(g[:, :r], gref[:, :r], scale) <= RTOL[prec]
    finally:
        alm.alm_destroy(h)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    one = torch.zeros(8, dtype=torch.float64, device="cuda")
    idx = torch.zeros(8, dtype=torch.int32, device="cuda")
    lib = alm.load()
    ptr = lambda t: alm.C.c_void_p(t.data_ptr())
    st = lib.alm_grad_unitdiag_noalloc(alm.ALM_FP64, (1 << 20) + 1, ptr(idx), ptr(idx), ptr(one), ptr(one),
                                       ptr(one), ptr(one), 1.0, ptr(one), 1, 2, ptr(one), None)
    assert st == alm.ALM_ERR_INVALID_ARG
    assert b"1048576" in lib.alm_last_error(None)
