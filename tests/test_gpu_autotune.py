"""The launch shapes of the two inner-step kernels and their autotuner (alm_set_inner_shape,
alm_autotune): every candidate shape solves the benchmark's form of the MaxCut SDP (FP32
bulk, r0 = r_max = 32, sigma0 = 10) to the oracle's objective, the oracle confirms the
KKT residual of each result, and the JSON-lines cache returns the tuned shape without
timing it again."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import sdp_instances as si  # noqa: E402
from gpu_common import as_np  # noqa: E402

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2505_15775_gb300 import alm  # noqa: E402

OPTS = dict(eps=1e-7, r_max=32, sigma0=10.0, lanczos_warm=1)


def _instance(which):
    # the torus's first lattice row has more upper neighbours than the narrow ELL holds (the
    # overflow list); a random 3-regular graph sends about an eighth of its rows there
    return si.torus_maxcut(40, 50, seed=3, weights="pm1") if which == "torus" else si.regular3_maxcut(1500, seed=12)


@pytest.fixture(scope="module", params=["torus", "regular3"])
def case(request):
    inst = _instance(request.param)
    R0 = si.factor_init(inst.n, 32, 0)
    P = O.OracleProblem(inst)
    ref = O.solve(P, R0, opts=O.SolveOptions(eps=1e-7, sigma=10.0))
    assert max(ref.kkt) <= 1e-7
    return inst, R0, P, ref


@pytest.mark.parametrize("k", range(len(alm.alm_inner_shapes()) if torch.cuda.is_available() else 0))
def test_every_shape_reaches_the_oracle_objective(case, k):
    inst, R0, P, ref = case
    shape = alm.alm_inner_shapes()[k]
    h = alm.alm_create(inst, precision=alm.ALM_FP32, **OPTS)
    try:
        alm.alm_set_inner_shape(h, **shape)
        got = alm.alm_get_inner_shape(h)
        assert got["variant"] == shape["variant"]
        if shape["variant"] == 1:
            assert got == shape
        R, r, y, st = alm.alm_solve(h, R0)
        R, y = as_np(R), as_np(y)
    finally:
        alm.alm_destroy(h)
    assert st["status"] == 0, (shape, st)
    assert st["objective"] == pytest.approx(ref.objective, rel=1e-6), shape
    lam = float(np.linalg.eigvalsh(O.slack_dense(P, y))[0])
    assert max(O.kkt(P, R, y, lam)) <= 1e-6, shape
    assert O.cost(P, R) == pytest.approx(st["objective"], rel=1e-6)


def test_autotune_and_its_cache(tmp_path):
    inst = _instance("torus")
    R0 = si.factor_init(inst.n, 32, 0)
    cache = str(tmp_path / "shapes.jsonl")
    h = alm.alm_create(inst, precision=alm.ALM_FP32, **OPTS)
    try:
        R = alm.factor_tensor(h, R0)
        Rc = R.clone()
        best, times, hit = alm.alm_autotune(h, R, 32, None, steps=16, cache=cache)
        assert not hit
        assert len(times) == len(alm.alm_inner_shapes())
        assert all(t > 0 for _, t in times)
        fastest = min(times, key=lambda x: x[1])[0]
        assert best["variant"] == fastest["variant"]
        if best["variant"] == 1:
            assert best == fastest
        assert alm.alm_get_inner_shape(h)["variant"] == best["variant"]
        assert torch.equal(R, Rc)  # the factor passed in is not modified
        _, _, _, st = alm.alm_solve(h, R0)
        assert st["status"] == 0
    finally:
        alm.alm_destroy(h)
    lines = [json.loads(x) for x in open(cache).read().splitlines()]
    assert len(lines) == 1 and lines[0]["variant"] == best["variant"]
    assert f"n={inst.n} " in lines[0]["key"] and " r=32 " in lines[0]["key"]
    # a new handle of the same problem takes the shape from the cache without timing
    h2 = alm.alm_create(inst, precision=alm.ALM_FP32, **OPTS)
    try:
        best2, times2, hit2 = alm.alm_autotune(h2, alm.factor_tensor(h2, R0), 32, None, steps=16, cache=cache)
        assert hit2 and times2 == [] and best2["variant"] == best["variant"]
        if best["variant"] == 1:
            assert best2 == best
    finally:
        alm.alm_destroy(h2)
    assert len(open(cache).read().splitlines()) == 1


def test_shape_rejects_invalid_values():
    inst = _instance("torus")
    h = alm.alm_create(inst, precision=alm.ALM_FP32, **OPTS)
    try:
        for bad in (dict(variant=2), dict(variant=1, stages=5), dict(variant=1, stages=2, threads=192)):
            with pytest.raises(alm.AlmError) as e:
                alm.alm_set_inner_shape(h, **bad)
            assert e.value.status == alm.ALM_ERR_INVALID_ARG
    finally:
        alm.alm_destroy(h)
