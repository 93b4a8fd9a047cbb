"""The primitives at the full n = 1e7 sizes (random 3-regular graph, seed 4; 2500 x 4000
torus with +-1 weights, seed 5), FP32 form, r = 32, in the launch configuration the
solver uses.  The checks are:
  * sampled rows of A(RR^T) and of G = 2 S R against their definitions evaluated row by
    row in FP64 on the host (Sec. 1.2 and Sec. 4.2), at the FP32 bar of 1e-5;
  * the line-search quartic against the FP64 oracle's (oracle.quartic_coeffs, sparse, on
    the whole instance; it needs about 30 GB of host memory), and against five evaluations
    of L_sigma along R + alpha D (a property of Eq. AL at any size);
  * the Lanczos pair (lambda, v): unit norm and a small residual ||S v - lambda v||
    measured with the gradient kernel on the one-column factor v (G = 2 S v)."""
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

R_COLS = 32
SIGMA = 1.7


def _instance(which):
    if which == "regular3-1e7":
        return si.regular3_maxcut(10 ** 7, seed=4)
    return si.torus_maxcut(2500, 4000, seed=5, weights="pm1")


@pytest.fixture(scope="module", params=["regular3-1e7", "torus-2500x4000"])
def big(request):
    inst = _instance(request.param)
    n = inst.n
    rng = np.random.default_rng(11)
    R = (rng.standard_normal((n, R_COLS), dtype=np.float32) / np.float32(np.sqrt(R_COLS)))
    y = rng.uniform(-1.0, 1.0, n)
    h = alm.alm_create(inst, precision=alm.ALM_FP32)
    off = inst.c_i != inst.c_j
    C = sp.coo_matrix((np.concatenate([inst.c_v[off], inst.c_v[off]]),
                       (np.concatenate([inst.c_i[off], inst.c_j[off]]), np.concatenate([inst.c_j[off], inst.c_i[off]]))),
                      shape=(n, n)).tocsr()
    cdiag = np.zeros(n)
    np.add.at(cdiag, inst.c_i[~off], inst.c_v[~off])
    yield dict(inst=inst, h=h, R=R, y=y, C=C, cdiag=cdiag)
    alm.alm_destroy(h)


def _rows(n, k=2000, seed=3):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([rng.integers(0, n, k), [0, n - 1]]))


def test_constraint_map_and_gradient_rows(big):
    inst, h, R, y, C, cd = big["inst"], big["h"], big["R"], big["y"], big["C"], big["cdiag"]
    Rd = torch.as_tensor(R, device="cuda")
    yd = torch.as_tensor(y, device="cuda")
    _, AX, _ = alm.alm_eval(h, Rd, R_COLS, yd, SIGMA)
    G, _ = alm.alm_grad(h, Rd, R_COLS, yd, SIGMA)
    AX, G = as_np(AX), as_np(G)
    rows = _rows(inst.n)
    R64 = R.astype(np.float64)
    x = np.einsum("ij,ij->i", R64[rows], R64[rows])
    assert np.max(np.abs(AX[rows] - x) / np.maximum(1.0, x)) <= 1e-5
    # G_i = 2 (S_ii r_i + sum_j C_ij r_j),  S_ii = C_ii - w_i,  w = y - sigma (|r_i|^2 - 1)
    w = y[rows] - SIGMA * (x - 1.0)
    Crow = C[rows]
    Gref = 2.0 * ((cd[rows] - w)[:, None] * R64[rows] + Crow @ R64)
    scale = 2.0 * (np.abs(cd[rows] - w)[:, None] * np.abs(R64[rows]) + abs(Crow) @ np.abs(R64))
    assert np.max(np.abs(G[rows] - Gref) / np.maximum(scale, 1.0)) <= 1e-5


def test_linesearch_quartic_interpolates_eval(big):
    h, R, y = big["h"], big["R"], big["y"]
    rng = np.random.default_rng(5)
    D = (rng.standard_normal(R.shape, dtype=np.float32) * np.float32(0.05))
    Rd, Dd = torch.as_tensor(R, device="cuda"), torch.as_tensor(D, device="cuda")
    yd = torch.as_tensor(y, device="cuda")
    q, alpha = alm.alm_linesearch(h, Rd, Dd, R_COLS, yd, SIGMA)
    import os

    if os.sysconf("SC_PHYS_PAGES") * os.sysconf("SC_PAGE_SIZE") >= 96 * 2 ** 30:
        qo = O.quartic_coeffs(O.OracleProblem(big["inst"]), R.astype(np.float64), D.astype(np.float64), y, SIGMA)
        for k in range(5):
            assert abs(q[k] - qo[k]) <= 1e-5 * max(abs(qo[k]), 1e-3 * float(np.abs(qo).max())), (k, q, qo)
        assert alpha == pytest.approx(O.exact_step(qo), rel=1e-4)
    for a in (0.0, 0.5, 1.0, -0.5, 2.0):
        L, _, _ = alm.alm_eval(h, Rd + a * Dd, R_COLS, yd, SIGMA, want_ax=False)
        phi = q[0] + a * (q[1] + a * (q[2] + a * (q[3] + a * q[4])))
        mag = abs(q[0]) + abs(a * q[1]) + abs(a * a * q[2]) + abs(a ** 3 * q[3]) + abs(a ** 4 * q[4])
        assert abs(L - phi) <= 1e-5 * mag
    assert alpha >= 0.0


def test_lanczos_pair_residual(big):
    h, R, y = big["h"], big["R"], big["y"]
    Rd = torch.as_tensor(R, device="cuda")
    yd = torch.as_tensor(y, device="cuda")
    lam, v, res = alm.alm_lambda_min(h, Rd, R_COLS, yd, SIGMA)
    vv = as_np(v)
    assert abs(np.linalg.norm(vv) - 1.0) < 1e-4
    # S v from the gradient kernel on the factor [v 0 0 0]: G = 2 S v (the constraint part of
    # S depends only on y, sigma and R through w, so evaluate S at the same R: w from R)
    _, AX, _ = alm.alm_eval(h, Rd, R_COLS, yd, SIGMA)
    w = yd - SIGMA * (AX - 1.0)  # the dual candidate at R (b = 1)
    V = torch.zeros((vv.size, 4), dtype=torch.float32, device="cuda")
    V[:, 0] = v
    Gv, _ = alm.alm_grad(h, V, 1, w, 0.0)  # sigma = 0: S = C - Diag(w)
    Sv = as_np(Gv)[:, 0] / 2.0
    snorm = float(np.abs(big["cdiag"]).max() + np.abs(as_np(w)).max() + 4.0)
    assert np.linalg.norm(Sv - lam * vv) <= 2e-4 * snorm
    assert res <= 2e-4 * snorm
