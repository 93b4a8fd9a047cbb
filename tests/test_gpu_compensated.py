"""Accuracy of the compensated FP32 sums in the fused step + SpMM kernels (the float-pair
|r_i|^2 and S_ii, and the error-free accumulation of G), at a state where plain FP32 sums are
not enough.

Unit rows r_i ~ s_i u + 1e-4 e_i (random signs s_i, one unit vector u, Gaussian noise e_i) on
the +-1 torus, and a dual that cancels the u component of S R row by row, so that G = 2 S R is
about 1e-3 of its terms, as near the end of an inner solve.  With alpha = 0 (R' = R) and the
preconditioner off (Z = G), the kernel's G must match the FP64 gradient of the oracle at the
same FP32 factor to an absolute 1e-10 of the terms' scale, plus the FP32 rounding of G itself
and of the one plain FP32 product in S_ii, sigma (|r_i|^2 - 1), which vanishes with the
primal residual; and <G, G> to 1e-6 relative.  The same terms summed in plain FP32, in the kernel's
order, miss the bar by orders of magnitude; the test checks that too, so that it keeps
telling the two apart.
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import sdp_instances as si  # noqa: E402
from gpu_common import as_np  # noqa: E402

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2505_15775_gb300 import alm  # noqa: E402

SIGMA = 10.0
SHAPES = [dict(variant=1, stages=2, threads=128), dict(variant=1, stages=3, threads=256), dict(variant=0)]


def _state(n, seed):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(32)
    u /= np.linalg.norm(u)
    s = rng.choice([-1.0, 1.0], n)
    R = s[:, None] * u[None, :] + 1e-4 * rng.standard_normal((n, 32))
    return (R / np.linalg.norm(R, axis=1, keepdims=True)).astype(np.float32)


def _dual_cancelling(P, R64, Coff, cdiag):
    """y with S_ii r_i + sum_j C_ij r_j orthogonal to r_i: the multiplier update w = y -
    sigma (|r_i|^2 - 1) has C_ii - w_i = -(r_i . (C_off R)_i) / |r_i|^2."""
    W = Coff @ R64
    nr2 = np.einsum("ij,ij->i", R64, R64)
    sii = -np.einsum("ij,ij->i", R64, W) / nr2
    w = cdiag - sii
    return w + SIGMA * (nr2 - 1.0)


def _plain_fp32(R, Coff, sdiag):
    """The same terms summed in FP32 without compensation, diagonal term first, then the
    neighbours in column order."""
    Cc = Coff.tocsr()
    acc = (np.float32(1.0) * sdiag.astype(np.float32)[:, None] * R).astype(np.float32)
    width = np.diff(Cc.indptr)
    assert np.all(width == width[0])
    cols = Cc.indices.reshape(-1, width[0])
    vals = Cc.data.reshape(-1, width[0]).astype(np.float32)
    for k in range(width[0]):
        acc = (acc + vals[:, k:k + 1] * R[cols[:, k]]).astype(np.float32)
    return (np.float32(2.0) * acc).astype(np.float32)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "-".join(str(v) for v in s.values()))
def test_gradient_at_a_near_stationary_state(shape):
    inst = si.torus_maxcut(100, 100, seed=5, weights="pm1")
    P = O.OracleProblem(inst)
    R = _state(inst.n, seed=41)
    R64 = R.astype(np.float64)
    C = P.C_sparse.tocsr()
    cdiag = C.diagonal()
    Coff = (C - sp.diags(cdiag)).tocsr()
    Coff.eliminate_zeros()
    y = _dual_cancelling(P, R64, Coff, cdiag)
    G = O.gradient(P, R64, y, SIGMA)
    sdiag = O.slack_sparse(P, O.dual_candidate(P, R64, y, SIGMA)).diagonal()
    scale = float(np.max((np.abs(sdiag) + np.asarray(abs(Coff).sum(axis=1)).ravel()) * np.abs(R64).max(axis=1)))
    # the state: G is ~1e-3 of the terms that sum to it
    assert 1e-5 * scale < np.abs(G).max() < 3e-3 * scale

    h = alm.alm_create(inst, precision=alm.ALM_FP32, sigma0=SIGMA, inner_precond=0)
    try:
        alm.alm_set_inner_shape(h, **shape)
        dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
        zero = np.zeros_like(R)
        Ro, Z, Dn, diag, sc = alm.alm_cg_step(h, dev(R), dev(zero), dev(zero), 32, dev(y), SIGMA, 0.0, 0.0)
        Ro, Z = as_np(Ro), as_np(Z)
    finally:
        alm.alm_destroy(h)
    assert np.array_equal(Ro, R)  # alpha = 0: R' = R exactly
    res = SIGMA * np.abs(np.einsum("ij,ij->i", R64, R64) - 1.0)
    bar = 1e-10 * scale + 2.0 ** -23 * np.abs(G) + 2.0 ** -21 * res[:, None] * np.abs(R64)
    err = np.abs(Z.astype(np.float64) - G)
    assert np.all(err <= bar), float(np.max(err / bar))
    gg = float(np.sum(G * G))
    assert abs(sc["gg"] - gg) <= 1e-6 * gg
    # plain FP32 sums of the same terms fail the same bar
    Gp = _plain_fp32(R, Coff, sdiag).astype(np.float64)
    assert np.max(np.abs(Gp - G) / bar) > 100.0
