"""Training the warm-start network on the method's own solutions (argument marshalling
over the C ABI only: the solves run in the batched persistent kernel, the forward,
backward and Adam steps in the network's kernels).

The paper's local convergence result for the BM subproblem (Sec. 4.2) and the
examples of Sec. 3.2 and 4.3 make a starting factor near a solution and a multiplier
near y* worth predicting; the network is trained on solutions that ALORA itself
computes for instances of the same generator (never on the instances it is applied to).
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import alm


def solve_cold(hb: alm.BatchHandle, factors) -> tuple[torch.Tensor, torch.Tensor, torch.Tensor, dict, list]:
    """Solve every instance of `hb` from the given initial factors and y0 = 0;
    -> (R, rank, y, batch stats, per-instance stats)."""
    R, rank = alm.batch_factor(hb, factors)
    y = torch.zeros(hb.rows, dtype=torch.float64, device="cuda")
    stats, per = alm.alm_batch_solve(hb, R, rank, y)
    return R, rank, y, stats, per


def train_warm_start(instances, factors, steps: int = 1500, lr: float = 3e-3, lam: float = 0.01,
                     storage: int = alm.ALM_GNN_BF16, feat_seed: int = 0x6E6E, init_seed: int = 7,
                     **batch_options) -> tuple[alm.GnnHandle, dict]:
    """Solve the training instances with the batched solver, then fit the network to
    their solutions with `steps` full-batch Adam steps.  -> (network, report)"""
    t0 = time.perf_counter()
    hb = alm.alm_batch_create(instances, **batch_options)
    try:
        R, rank, y, stats, per = solve_cold(hb, factors)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        g = alm.alm_gnn_create(storage, feat_seed=feat_seed, init_seed=init_seed)
        losses = alm.alm_gnn_train(g, hb, R, y, lam, steps, lr)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
    finally:
        alm.alm_batch_destroy(hb)
    report = {"train_instances": len(instances), "train_converged": stats["converged"],
              "solve_s": t1 - t0, "fit_s": t2 - t1, "steps": steps, "lr": lr, "lam": lam,
              "loss_first": float(losses[0]) if len(losses) else None,
              "loss_last": float(losses[-1]) if len(losses) else None}
    return g, report
