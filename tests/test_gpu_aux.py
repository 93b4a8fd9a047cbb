"""Auxiliary subsystems of the library on the GPU: the per-outer-iteration JSON-lines log of
alm_solve (alm_set_log) and the host-side fault injection of alm_create (ALM_FAULT_INJECT).
Injection corrupts only the library's private copy of the problem or fails an allocation
on the host: no GPU fault is made."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import sdp_instances as si  # noqa: E402

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2505_15775_gb300 import alm  # noqa: E402

KEYS = {"outer", "inner", "inner_total", "rank", "sigma", "lambda_min", "grew", "kkt", "objective", "alpha_last",
        "time_ms"}


def _solve(inst, log=None, **opt):
    h = alm.alm_create(inst, precision=alm.ALM_FP64, eps=1e-7, **opt)
    try:
        if log is not None:
            alm.alm_set_log(h, log)
        return alm.alm_solve(h, si.factor_init(inst.n, 2, 1))[3]
    finally:
        alm.alm_destroy(h)


def test_log_has_one_line_per_outer_iteration(tmp_path):
    inst = si.er_maxcut(200, 0.05, seed=3)
    path = str(tmp_path / "solve.jsonl")
    st = _solve(inst, log=path)
    lines = [json.loads(x) for x in open(path).read().splitlines()]
    assert st["status"] == alm.ALM_OK
    assert len(lines) == st["outer"]
    assert all(set(x) == KEYS for x in lines)
    assert [x["outer"] for x in lines] == list(range(1, st["outer"] + 1))
    assert sum(x["inner"] for x in lines) == st["inner_total"] == lines[-1]["inner_total"]
    last = lines[-1]
    assert not last["grew"] and last["rank"] == st["rank"]
    assert last["kkt"] == list(st["kkt"]) and max(last["kkt"]) <= 1e-7
    assert last["objective"] == pytest.approx(st["objective"], rel=1e-12)
    assert sum(x["grew"] for x in lines) == st["growth_steps"]
    for x in lines:
        assert x["sigma"] > 0 and x["time_ms"]["total"] >= x["time_ms"]["inner"] >= 0
        assert (x["lambda_min"] is None) == (x["time_ms"]["lanczos"] == 0)
    # appending: a second solve adds its own lines; switching the log off adds none
    st2 = _solve(inst, log=path)
    assert len(open(path).read().splitlines()) == st["outer"] + st2["outer"]
    _solve(inst, log=None)
    h = alm.alm_create(inst, precision=alm.ALM_FP64)
    try:
        alm.alm_set_log(h, path)
        alm.alm_set_log(h, None)
        alm.alm_solve(h, si.factor_init(inst.n, 2, 1))
    finally:
        alm.alm_destroy(h)
    assert len(open(path).read().splitlines()) == st["outer"] + st2["outer"]


def test_log_path_that_cannot_be_opened(tmp_path):
    inst = si.er_maxcut(50, 0.1, seed=4)
    h = alm.alm_create(inst, precision=alm.ALM_FP64)
    try:
        with pytest.raises(alm.AlmError) as e:
            alm.alm_set_log(h, str(tmp_path / "no_such_dir" / "x.jsonl"))
        assert e.value.status == alm.ALM_ERR_INVALID_ARG
    finally:
        alm.alm_destroy(h)


@pytest.mark.parametrize("mode,status,text", [("nan_b", "ALM_ERR_INVALID_ARG", "b[0] is not finite"),
                                              ("csr", "ALM_ERR_INVALID_ARG", "out of range"),
                                              ("oom", "ALM_ERR_OOM", "injected"),
                                              ("bogus", "ALM_ERR_INVALID_ARG", "ALM_FAULT_INJECT")])
def test_fault_injection(monkeypatch, mode, status, text):
    inst = si.er_maxcut(60, 0.1, seed=5)
    b0 = np.array(inst.b, copy=True)
    monkeypatch.setenv("ALM_FAULT_INJECT", mode)
    with pytest.raises(alm.AlmError) as e:
        alm.alm_create(inst, precision=alm.ALM_FP32)
    assert e.value.status == getattr(alm, status)
    assert text in str(e.value)
    assert np.array_equal(inst.b, b0)  # the caller's arrays are untouched
    # with the variable unset the same problem creates and solves
    monkeypatch.delenv("ALM_FAULT_INJECT")
    st = _solve(inst)
    assert st["status"] == alm.ALM_OK
