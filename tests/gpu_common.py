"""Helpers shared by the GPU parity tests (no test functions here)."""
import math

import numpy as np
import torch

import oracle as O
import sdp_instances as si

# tolerances of the parity bar: FP64 primitives 1e-12 relative, FP32 primitives 1e-5 relative
RTOL = {0: 1e-12, 1: 1e-5}


def rel_err(a, b, scale=None):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    s = scale if scale is not None else max(1.0, float(np.max(np.abs(b))) if b.size else 1.0)
    return float(np.max(np.abs(a - b))) / s if a.size else 0.0


def instances_small():
    """Seeded instances spanning every data path (selector diagonal and off-diagonal
    constraints, general constraints on diagonal and off-diagonal entries, low-rank C,
    ragged row lengths, isolated vertices) at sizes the oracle finishes in seconds."""
    return {
        "maxcut-er-800": si.er_maxcut(800, 0.06, seed=1),
        "maxcut-torus-30x41-pm1": si.torus_maxcut(30, 41, seed=2, weights="pm1"),
        "maxcut-er-sparse-isolated": si.er_maxcut(997, 0.0015, seed=5, weights="pm1"),
        "theta-er-400": si.theta_er(400, 6.0, seed=3),
        "general-300": si.random_general(300, 120, seed=4, lr_k=2, diag_frac=0.4),
        "spurious-d9": si.t15_instance(9, 0.1, 2.0),
    }


def factor_for(inst, r, seed):
    scale = None if inst.kind in ("maxcut", "example", "general") else 1.0 / math.sqrt(inst.n * r)
    return si.factor_init(inst.n, r, seed, scale=scale)


def dual_for(inst, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, inst.m)


def as_np(t):
    return t.detach().to("cpu", torch.float64).numpy()
