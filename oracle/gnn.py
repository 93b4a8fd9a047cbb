"""FP64 CPU oracle of the learned warm start (TEST INFRASTRUCTURE ONLY; see package doc).

The paper has no network.  Its local linear convergence result for the BM subproblem
(Sec. 4.2) and the examples of Sec. 3.2 and 4.3 show that ALM-BM is fast from an initial
factor near a solution and a multiplier near y*; the warm start predicts such a pair
(R0, y0) for a unit-diagonal SDP  min <C, X>  s.t.  diag(X) = 1,  X >= 0  from C alone.

Network (every quantity per instance with n rows; C's off-diagonal pattern in full
symmetric form, entries c_ij, diagonal c_ii):
  deg_i = number of off-diagonal entries of row i,  s_i = sum_j c_ij
  dbar = max(mean_i deg_i, 1),  cbar = mean |c_ij| over the off-diagonal entries (1 if none),
  sbar = mean_i |s_i| (1 if 0)
  features x_i = [1, deg_i / dbar, s_i / sbar, log(n) / 8, u_1(i), u_2(i), u_3(i), u_4(i)]
      with u_k(i) = SplitMix64 uniform on [-1, 1), stream feat_seed + k, element i (local row)
  edge weights a_ij = c_ij / cbar
  layer l = 1, 2, 3:  agg_i = (sum_j a_ij h_j) / max(deg_i, 1)
                      h'_i = relu(Ws_l h_i + Wn_l agg_i + b_l)          (h^0 = x, width 8 -> 64)
  heads:  rhat_i = W_R h^3_i  (32 columns),   yhat_i = w_y . h^3_i + b_y
  warm start:  a_i = rhat_i / |rhat_i| (0 for a zero row),  u_i = the 32 SplitMix64 uniforms
               of stream mix_seed, elements 32 i .. 32 i + 31 (local row i),
               w_i = a_i + mix u_i / |u_i|,  R0_i = w_i / |w_i| (e_1 when w_i = 0),
               y0_i = cbar * yhat_i;  mix = 0 gives the network's unit rows alone, mix > 0
               keeps R0 of full rank (the library draws u from stream feat_seed ^ 0x3a1d)
Training loss over a set of instances with solutions (R*, y*), X* = R* R*^T:
  L = sum_b sum_{p in P_b} (rhat_i . rhat_j - X*_p)^2 / sum_b |P_b|
      + lam * sum_b sum_i (yhat_i - y*_i / cbar_b)^2 / sum_b n_b
with P_b the upper pattern including the diagonal: a loss on X, not on R, because R* is
unique only up to R* Q.

Parameters are one flat float vector in the order of ``param_layout``.
"""
from __future__ import annotations

import math

import numpy as np

FEAT = 8
HID = 64
LAYERS = 3
RANK = 32
MASK64 = (1 << 64) - 1


def param_layout():
    """[(name, shape)] in storage order."""
    out = []
    din = FEAT
    for l in range(LAYERS):
        out += [(f"Ws{l}", (HID, din)), (f"Wn{l}", (HID, din)), (f"b{l}", (HID,))]
        din = HID
    out += [("WR", (RANK, HID)), ("wy", (HID,)), ("by", (1,))]
    return out


def n_params() -> int:
    return sum(int(np.prod(s)) for _, s in param_layout())


def unpack(theta):
    out, o = {}, 0
    for name, shape in param_layout():
        k = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + k], np.float64).reshape(shape)
        o += k
    return out


def splitmix_uniform_pm1(seed: int, idx: np.ndarray) -> np.ndarray:
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) as a counter generator: element i of
    stream `seed` is mix(seed + (i + 1) * 0x9e3779b97f4a7c15); mapped to [-1, 1) through
    its top 53 bits.  Plain Python integers, exact modulo 2^64."""
    out = np.empty(len(idx))
    for t, i in enumerate(idx):
        z = (seed + (int(i) + 1) * 0x9E3779B97F4A7C15) & MASK64
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        z ^= z >> 31
        out[t] = 2.0 * ((z >> 11) * (1.0 / 9007199254740992.0)) - 1.0
    return out


class Graph:
    """C of one unit-diagonal instance as the network sees it (dense-free, FP64)."""

    def __init__(self, inst):
        n = inst.n
        off = inst.c_i != inst.c_j
        i = np.concatenate([inst.c_i[off], inst.c_j[off]]).astype(np.int64)
        j = np.concatenate([inst.c_j[off], inst.c_i[off]]).astype(np.int64)
        v = np.concatenate([inst.c_v[off], inst.c_v[off]]).astype(np.float64)
        # merge repeated entries
        key = i * n + j
        uk, inv = np.unique(key, return_inverse=True)
        vals = np.zeros(uk.size)
        np.add.at(vals, inv, v)
        self.n = n
        self.i = (uk // n).astype(np.int64)
        self.j = (uk % n).astype(np.int64)
        self.c = vals
        self.cdiag = np.zeros(n)
        np.add.at(self.cdiag, inst.c_i[~off], inst.c_v[~off])
        self.deg = np.bincount(self.i, minlength=n).astype(np.float64)
        self.s = np.bincount(self.i, weights=self.c, minlength=n)
        self.dbar = max(float(self.deg.mean()), 1.0)
        self.cbar = float(np.abs(self.c).mean()) if self.c.size else 1.0
        sb = float(np.abs(self.s).mean())
        self.sbar = sb if sb > 0 else 1.0
        self.a = self.c / self.cbar

    def features(self, feat_seed: int) -> np.ndarray:
        n = self.n
        x = np.zeros((n, FEAT))
        x[:, 0] = 1.0
        x[:, 1] = self.deg / self.dbar
        x[:, 2] = self.s / self.sbar
        x[:, 3] = math.log(n) / 8.0
        idx = np.arange(n)
        for k in range(4):
            x[:, 4 + k] = splitmix_uniform_pm1(feat_seed + k, idx)
        return x

    def aggregate(self, h):
        """(sum_j a_ij h_j) / max(deg_i, 1)"""
        out = np.zeros_like(h)
        np.add.at(out, self.i, self.a[:, None] * h[self.j])
        return out / np.maximum(self.deg, 1.0)[:, None]



def _agg_T(G: Graph, g):
    """Adjoint of ``Graph.aggregate``: out_j = sum_i a_ij g_i / max(deg_i, 1)."""
    out = np.zeros_like(g)
    scaled = g / np.maximum(G.deg, 1.0)[:, None]
    np.add.at(out, G.j, G.a[:, None] * scaled[G.i])
    return out


def forward(theta, G: Graph, feat_seed: int):
    """-> (rhat n x 32, yhat n, cache of the activations)"""
    P = unpack(theta)
    h = G.features(feat_seed)
    cache = []
    for l in range(LAYERS):
        agg = G.aggregate(h)
        z = h @ P[f"Ws{l}"].T + agg @ P[f"Wn{l}"].T + P[f"b{l}"]
        hn = np.maximum(z, 0.0)
        cache.append((h, agg, hn))
        h = hn
    rhat = h @ P["WR"].T
    yhat = h @ P["wy"] + P["by"][0]
    return rhat, yhat, cache


MIX_STREAM_XOR = 0x3A1D  # the library's mixing stream is feat_seed ^ this constant


def mix_rows(n: int, mix_seed: int) -> np.ndarray:
    """u (n x 32): element (i, c) is SplitMix64 uniform 32 i + c of stream mix_seed."""
    return splitmix_uniform_pm1(mix_seed, np.arange(n * RANK)).reshape(n, RANK)


def _unit_rows(M):
    nr = np.linalg.norm(M, axis=1)
    out = np.zeros_like(M)
    ok = nr > 0
    out[ok] = M[ok] / nr[ok, None]
    return out, ok


def warm_start(theta, G: Graph, feat_seed: int, mix: float = 0.0, mix_seed: int | None = None):
    """(R0 with unit rows, y0) from the network's heads: R0_i = normalise(rhat_i/|rhat_i|
    + mix u_i/|u_i|) with u_i the seeded uniform row of ``mix_rows`` (stream ``mix_seed``,
    by default feat_seed ^ 0x3a1d); a row whose sum is zero becomes e_1."""
    rhat, yhat, _ = forward(theta, G, feat_seed)
    w, _ = _unit_rows(rhat)
    if mix != 0.0:
        seed = (feat_seed ^ MIX_STREAM_XOR) if mix_seed is None else mix_seed
        u, _ = _unit_rows(mix_rows(G.n, seed))
        w = w + mix * u
    R0, ok = _unit_rows(w)
    R0[~ok, 0] = 1.0
    return R0, G.cbar * yhat


def pattern_targets(G: Graph, Rstar):
    """X*_p on P: the diagonal, then the strict upper entries (i < j)."""
    up = G.i < G.j
    xd = np.einsum("ij,ij->i", Rstar, Rstar)
    xo = np.einsum("ij,ij->i", Rstar[G.i[up]], Rstar[G.j[up]])
    return xd, xo, up


def loss_and_grad(theta, graphs, feat_seed: int, Rstars, ystars, lam: float):
    """Loss over a set of instances and its gradient, by reverse-mode differentiation
    written out layer by layer."""
    P = unpack(theta)
    grads = {k: np.zeros_like(v) for k, v in P.items()}
    npat = sum(G.n + int(np.sum(G.i < G.j)) for G in graphs)
    nrow = sum(G.n for G in graphs)
    L = 0.0
    for G, Rs, ys in zip(graphs, Rstars, ystars):
        rhat, yhat, cache = forward(theta, G, feat_seed)
        xd, xo, up = pattern_targets(G, Rs)
        ed = np.einsum("ij,ij->i", rhat, rhat) - xd
        iu, ju = G.i[up], G.j[up]
        eo = np.einsum("ij,ij->i", rhat[iu], rhat[ju]) - xo
        ey = yhat - ys / G.cbar
        L += (np.sum(ed ** 2) + np.sum(eo ** 2)) / npat + lam * np.sum(ey ** 2) / nrow
        # d/d rhat
        dr = (4.0 / npat) * ed[:, None] * rhat
        np.add.at(dr, iu, (2.0 / npat) * eo[:, None] * rhat[ju])
        np.add.at(dr, ju, (2.0 / npat) * eo[:, None] * rhat[iu])
        dy = (2.0 * lam / nrow) * ey
        h3 = cache[-1][2]
        grads["WR"] += dr.T @ h3
        grads["wy"] += h3.T @ dy
        grads["by"] += np.sum(dy)
        dh = dr @ P["WR"] + dy[:, None] * P["wy"][None, :]
        for l in reversed(range(LAYERS)):
            h, agg, hn = cache[l]
            dz = dh * (hn > 0.0)
            grads[f"Ws{l}"] += dz.T @ h
            grads[f"Wn{l}"] += dz.T @ agg
            grads[f"b{l}"] += dz.sum(axis=0)
            dh = dz @ P[f"Ws{l}"] + _agg_T(G, dz @ P[f"Wn{l}"])
    flat = np.concatenate([grads[name].reshape(-1) for name, _ in param_layout()])
    return L, flat


def init_params(seed: int) -> np.ndarray:
    """Seeded initial weights: U(-1, 1) * sqrt(3 / fan_in) (unit-variance preserving),
    zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in param_layout():
        if len(shape) == 2:
            parts.append(rng.uniform(-1.0, 1.0, shape).reshape(-1) * math.sqrt(3.0 / shape[1]))
        else:
            parts.append(np.zeros(int(np.prod(shape))))
    return np.concatenate(parts)
