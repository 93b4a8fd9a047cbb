"""Pins of the FP64 warm-start network oracle (oracle.gnn): the counter generator against
its published outputs, the aggregation against its adjoint, the hand-derived backward
pass against central finite differences, and closed-form losses."""
import numpy as np
import pytest

import oracle.gnn as G
import sdp_instances as si


def _graphs():
    z = np.zeros(0, np.int64)
    return [
        G.Graph(si.er_maxcut(12, 0.35, seed=3)),
        G.Graph(si.maxcut(7, *si.cycle_edges(7), np.ones(7))),
        G.Graph(si.er_maxcut(20, 0.2, seed=4, weights="pm1")),
        G.Graph(si.maxcut(3, z, z, np.zeros(0))),  # no edges: aggregation is empty
    ]


def _targets(graphs, seed=5):
    rng = np.random.default_rng(seed)
    Rs, ys = [], []
    for g in graphs:
        R = rng.standard_normal((g.n, G.RANK))
        R /= np.linalg.norm(R, axis=1, keepdims=True)
        Rs.append(R)
        ys.append(rng.uniform(-3, 0, g.n))
    return Rs, ys


def test_splitmix64_published_outputs():
    """SplitMix64 from state 0 emits 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4,
    0x06c45d188009454f (the reference generator's first outputs); the features map the
    top 53 bits to [-1, 1)."""
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = G.splitmix_uniform_pm1(0, np.arange(3))
    want = [2.0 * ((z >> 11) / 2.0 ** 53) - 1.0 for z in expect]
    assert np.array_equal(got, np.array(want))


def test_aggregation_adjoint():
    rng = np.random.default_rng(1)
    for g in _graphs():
        h = rng.standard_normal((g.n, 5))
        u = rng.standard_normal((g.n, 5))
        lhs = float(np.sum(g.aggregate(h) * u))
        rhs = float(np.sum(h * G._agg_T(g, u)))
        assert lhs == pytest.approx(rhs, rel=1e-13, abs=1e-13)


def test_features_and_scales():
    g = G.Graph(si.er_maxcut(30, 0.2, seed=9))
    x = g.features(7)
    assert np.all(x[:, 0] == 1.0)
    assert x[:, 1].mean() == pytest.approx(g.deg.mean() / g.dbar)
    assert np.all(np.abs(x[:, 4:]) <= 1.0)
    # unit-weight MaxCut: C_ij = 1/4 on edges, so cbar = 1/4 and every a_ij = 1
    assert g.cbar == pytest.approx(0.25)
    assert np.allclose(g.a, 1.0)


def test_gradient_matches_central_differences():
    graphs = _graphs()
    Rs, ys = _targets(graphs)
    theta = G.init_params(3) * 1.5
    theta[-1] = 0.3
    lam = 0.3
    L, grad = G.loss_and_grad(theta, graphs, 11, Rs, ys, lam)
    rng = np.random.default_rng(2)
    idx = np.concatenate([rng.choice(theta.size, 120, replace=False),
                          np.arange(theta.size - 200, theta.size)])  # the heads and last biases in full
    for k in idx:
        h = 1e-6 * max(1.0, abs(theta[k]))
        tp = theta.copy()
        tm = theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (G.loss_and_grad(tp, graphs, 11, Rs, ys, lam)[0] - G.loss_and_grad(tm, graphs, 11, Rs, ys, lam)[0]) / (2 * h)
        assert grad[k] == pytest.approx(fd, rel=1e-5, abs=1e-8 * max(1.0, abs(L))), k


def test_zero_network_loss_closed_form():
    """theta = 0 except b_y: rhat = 0, yhat = b_y, so the loss is
    sum_P X*_p^2 / |P| + lam sum_i (b_y - y*_i/cbar)^2 / n."""
    graphs = _graphs()[:3]
    Rs, ys = _targets(graphs, seed=8)
    theta = np.zeros(G.n_params())
    theta[-1] = -1.25
    lam = 0.7
    L, grad = G.loss_and_grad(theta, graphs, 0, Rs, ys, lam)
    npat = sum(g.n + int(np.sum(g.i < g.j)) for g in graphs)
    nrow = sum(g.n for g in graphs)
    xs = sum(float(np.sum(np.einsum("ij,ij->i", R, R) ** 2)) +
             float(np.sum(np.einsum("ij,ij->i", R[g.i[g.i < g.j]], R[g.j[g.i < g.j]]) ** 2))
             for g, R in zip(graphs, Rs))
    ye = sum(float(np.sum((-1.25 - y / g.cbar) ** 2)) for g, y in zip(graphs, ys))
    assert L == pytest.approx(xs / npat + lam * ye / nrow, rel=1e-13)
    assert grad[-1] == pytest.approx(sum(float(np.sum(2 * lam * (-1.25 - y / g.cbar))) for g, y in zip(graphs, ys))
                                     / nrow, rel=1e-12)


def test_warm_start_rows_are_unit():
    g = G.Graph(si.er_maxcut(25, 0.3, seed=1))
    R0, y0 = G.warm_start(G.init_params(4), g, 3)
    assert np.allclose(np.linalg.norm(R0, axis=1), 1.0)
    assert y0.shape == (25,)


def _unit(M):
    return M / np.linalg.norm(M, axis=1, keepdims=True)


def test_mix_rows_indexing():
    """Row i of the mixing rows holds elements 32 i .. 32 i + 31 of the stream: row 0 of
    stream 0 starts with the generator's published first outputs."""
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = G.mix_rows(3, 0)
    assert u.shape == (3, G.RANK)
    assert np.array_equal(u[0, :3], np.array([2.0 * ((z >> 11) / 2.0 ** 53) - 1.0 for z in expect]))
    assert np.array_equal(u[2, 5:9], G.splitmix_uniform_pm1(0, np.arange(69, 73)))


def test_warm_start_mix_zero_is_the_unit_network_rows():
    g = G.Graph(si.er_maxcut(25, 0.3, seed=1))
    th = G.init_params(4)
    rhat, yhat, _ = G.forward(th, g, 3)
    R0, y0 = G.warm_start(th, g, 3, mix=0.0)
    assert np.allclose(R0, _unit(rhat), rtol=0, atol=1e-15)
    assert np.array_equal(y0, g.cbar * yhat)


@pytest.mark.parametrize("mix", [0.3, 1.0, 5.0])
def test_warm_start_mix_geometry(mix):
    """R0_i is the unit vector along a_i + mix b_i (a_i the network's unit row, b_i the
    seeded unit row): it lies in span(a_i, b_i), has unit norm, and its components along
    a_i and b_i stand in the ratio (1 + mix c) : (c + mix), c = a_i . b_i.  At mix = 1 it
    bisects the angle between a_i and b_i."""
    g = G.Graph(si.er_maxcut(30, 0.25, seed=2))
    th = G.init_params(6)
    rhat, _, _ = G.forward(th, g, 5)
    a = _unit(rhat)
    b = _unit(G.splitmix_uniform_pm1(5 ^ 0x3A1D, np.arange(g.n * 32)).reshape(g.n, 32))
    R0, _ = G.warm_start(th, g, 5, mix=mix)
    assert np.allclose(np.linalg.norm(R0, axis=1), 1.0, atol=1e-14)
    c = np.einsum("ij,ij->i", a, b)
    # least-squares coordinates of R0 in the basis (a, b); the residual must vanish
    for i in range(g.n):
        B = np.stack([a[i], b[i]], axis=1)
        coef, *_ = np.linalg.lstsq(B, R0[i], rcond=None)
        assert np.linalg.norm(B @ coef - R0[i]) <= 1e-13
        assert coef[1] / coef[0] == pytest.approx(mix, rel=1e-11)
        ra, rb = R0[i] @ a[i], R0[i] @ b[i]
        assert ra / rb == pytest.approx((1 + mix * c[i]) / (c[i] + mix), rel=1e-11)
    if mix == 1.0:
        assert np.allclose(np.einsum("ij,ij->i", R0, a), np.einsum("ij,ij->i", R0, b), atol=1e-14)


def test_warm_start_zero_network():
    """theta = 0 gives rhat = 0: the warm start is e_1 without mixing and the seeded unit
    row with it; y0 = cbar * b_y."""
    g = G.Graph(si.er_maxcut(15, 0.3, seed=3))
    th = np.zeros(G.n_params())
    th[-1] = 0.5
    R0, y0 = G.warm_start(th, g, 9, mix=0.0)
    e1 = np.zeros((15, 32))
    e1[:, 0] = 1.0
    assert np.array_equal(R0, e1)
    assert np.allclose(y0, g.cbar * 0.5)
    R1, _ = G.warm_start(th, g, 9, mix=2.0, mix_seed=77)
    assert np.allclose(R1, _unit(G.mix_rows(15, 77)), atol=1e-15)


def test_warm_start_large_mix_tends_to_the_seeded_rows():
    g = G.Graph(si.er_maxcut(20, 0.3, seed=4))
    th = G.init_params(2)
    R0, _ = G.warm_start(th, g, 1, mix=1e9)
    assert np.max(np.abs(R0 - _unit(G.mix_rows(20, 1 ^ 0x3A1D)))) <= 3e-9
