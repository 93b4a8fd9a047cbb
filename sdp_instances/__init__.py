"""Seeded synthetic SDP instances: the one module both the CUDA path's tests and
the oracle read their inputs from.

It builds graphs and turns them into problem data (C, {A_k}, b) in the
coordinate form the C-ABI takes (upper-triangle COO, ``i <= j``, an off-diagonal
entry ``v`` at (i, j) meaning ``M_ij = M_ji = v``).  It holds none of the
method's arithmetic: no constraint map, gradient, line search or eigensolve.

Problem families
----------------
* MaxCut SDP (Sec. 6.1): ``max 1/4 <L, X>``, ``X_ii = 1``, ``X >= 0``.  It is
  stated in the minimisation form of (P) with ``C = -L/4``, ``A_i = e_i e_i^T``
  and ``b = 1``; the MaxCut value is ``-<C, X>``.
* Lovasz theta SDP: ``max <J, X>``, ``tr X = 1``, ``X_ij = 0`` on edges, as
  ``min <-J, X>`` with ``-J`` carried as the rank-one term ``-1 1^T`` and each
  edge constraint as ``(e_i e_j^T + e_j e_i^T)/2`` with right-hand side 0.

Graph families: Erdos-Renyi G(n, p), 2-D toroidal grids, random 3-regular
graphs (configuration model repaired by edge switches), cycles and complete
graphs.  Weights are either unit or Rademacher +-1 (p = 1/2 each).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Instance", "er_edges", "torus_edges", "cycle_edges", "complete_edges",
    "regular3_edges", "edge_weights", "maxcut", "lovasz_theta", "factor_init",
    "er_maxcut", "torus_maxcut", "regular3_maxcut", "theta_er", "batch_specs",
    "t8_instance", "t11_instance", "t15_instance", "random_general",
]


@dataclass
class Instance:
    """Problem data in the C-ABI's coordinate form (all host numpy arrays)."""
    n: int
    m: int
    c_i: np.ndarray          # int32, upper-triangle COO of C (i <= j)
    c_j: np.ndarray
    c_v: np.ndarray          # float64
    a_k: np.ndarray          # int32, constraint index of each A entry
    a_i: np.ndarray          # int32, i <= j
    a_j: np.ndarray
    a_v: np.ndarray          # float64
    b: np.ndarray            # float64, length m
    c_lr_u: np.ndarray = field(default_factory=lambda: np.zeros((0, 0)))  # (k, n) float64
    c_lr_s: np.ndarray = field(default_factory=lambda: np.zeros(0))       # (k,) float64
    name: str = ""
    kind: str = ""           # "maxcut" | "theta" | "example"
    graph: tuple | None = None  # (ei, ej, w) when built from a graph

    @property
    def c_lr_k(self) -> int:
        return int(self.c_lr_s.shape[0])


def _flat_seed(seed):
    """Nested seed tuples, e.g. ((6, i), 0) for stream 0 of batch instance i, flattened to
    the flat entropy list SeedSequence takes; flat seeds pass through unchanged."""
    if isinstance(seed, (tuple, list)):
        out = []
        for s in seed:
            f = _flat_seed(s)
            out.extend(f if isinstance(f, list) else [f])
        return out if any(isinstance(s, (tuple, list)) for s in seed) else list(seed)
    return seed


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(_flat_seed(seed))))


# ----------------------------------------------------------------------------------
# graphs (edges as int64 arrays i < j, no loops, no duplicates)
# ----------------------------------------------------------------------------------
def _tri_index_to_pair(t: np.ndarray, n: int) -> tuple[np.ndarray, np.ndarray]:
    """Map linear indices of the strict upper triangle (row-major) to (i, j)."""
    t = t.astype(np.float64)
    # number of pairs before row i: i*n - i*(i+1)/2
    i = np.floor((2 * n - 1 - np.sqrt((2 * n - 1) ** 2 - 8 * t)) / 2).astype(np.int64)
    i = np.clip(i, 0, n - 2)
    start = i * n - i * (i + 1) // 2
    # fix floating error in either direction
    while True:
        over = start > t
        if not over.any():
            break
        i[over] -= 1
        start = i * n - i * (i + 1) // 2
    nxt = (i + 1) * n - (i + 1) * (i + 2) // 2
    while True:
        under = t >= nxt
        if not under.any():
            break
        i[under] += 1
        start = i * n - i * (i + 1) // 2
        nxt = (i + 1) * n - (i + 1) * (i + 2) // 2
    j = (t.astype(np.int64) - start) + i + 1
    return i, j


def er_edges(n: int, p: float, seed) -> tuple[np.ndarray, np.ndarray]:
    """Erdos-Renyi G(n, p): the edge count is Binomial(n(n-1)/2, p) and the edge set
    a uniform sample of that many distinct pairs (the same law as per-pair coins)."""
    rng = _rng(seed)
    npairs = n * (n - 1) // 2
    if npairs == 0 or p <= 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    cnt = int(rng.binomial(npairs, min(p, 1.0)))
    t = np.sort(rng.choice(npairs, size=cnt, replace=False))
    return _tri_index_to_pair(t, n)


def torus_edges(n1: int, n2: int) -> tuple[np.ndarray, np.ndarray]:
    """2-D toroidal grid n1 x n2 (vertex a*n2+b joined to its right and lower
    neighbours, wrapping).  Needs n1, n2 >= 3 so that no edge repeats."""
    assert n1 >= 3 and n2 >= 3
    a, bb = np.meshgrid(np.arange(n1, dtype=np.int64), np.arange(n2, dtype=np.int64), indexing="ij")
    v = (a * n2 + bb).ravel()
    right = (a * n2 + (bb + 1) % n2).ravel()
    down = (((a + 1) % n1) * n2 + bb).ravel()
    i = np.concatenate([v, v])
    j = np.concatenate([right, down])
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    order = np.lexsort((hi, lo))
    return lo[order], hi[order]


def cycle_edges(n: int) -> tuple[np.ndarray, np.ndarray]:
    i = np.arange(n, dtype=np.int64)
    j = (i + 1) % n
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    order = np.lexsort((hi, lo))
    return lo[order], hi[order]


def complete_edges(n: int) -> tuple[np.ndarray, np.ndarray]:
    i, j = np.triu_indices(n, k=1)
    return i.astype(np.int64), j.astype(np.int64)


def regular3_edges(n: int, seed, max_rounds: int = 200) -> tuple[np.ndarray, np.ndarray]:
    """Random 3-regular simple graph: configuration-model pairing of 3n stubs, then
    every loop or repeated edge is removed by a random double-edge switch with
    another edge (degree-preserving).  n must be even."""
    assert n % 2 == 0 and n >= 4
    rng = _rng(seed)
    stubs = np.repeat(np.arange(n, dtype=np.int64), 3)
    rng.shuffle(stubs)
    u = stubs[0::2].copy()
    v = stubs[1::2].copy()
    ne = u.shape[0]
    for _ in range(max_rounds):
        lo, hi = np.minimum(u, v), np.maximum(u, v)
        key = lo * n + hi
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.zeros(ne, bool)
        dup[order[1:]] = ks[1:] == ks[:-1]
        bad = np.nonzero(dup | (u == v))[0]
        if bad.size == 0:
            break
        # switch each bad edge (a,b) with a random edge (c,d): (a,d), (c,b)
        partner = rng.integers(0, ne, size=bad.size)
        for e, f in zip(bad.tolist(), partner.tolist()):
            if e == f:
                continue
            u[e], v[e], u[f], v[f] = u[e], v[f], u[f], v[e]
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    assert np.all(lo != hi)
    order = np.lexsort((hi, lo))
    lo, hi = lo[order], hi[order]
    assert np.all((lo[1:] != lo[:-1]) | (hi[1:] != hi[:-1])), "repair did not converge"
    return lo, hi


def edge_weights(num_edges: int, kind: str, seed) -> np.ndarray:
    if kind == "unit":
        return np.ones(num_edges)
    if kind == "pm1":  # Rademacher +-1
        rng = _rng(seed)
        return np.where(rng.random(num_edges) < 0.5, -1.0, 1.0)
    raise ValueError(kind)


# ----------------------------------------------------------------------------------
# problem data
# ----------------------------------------------------------------------------------
def maxcut(n: int, ei, ej, w, name: str = "") -> Instance:
    """MaxCut SDP of Sec. 6.1 in (P)'s min form: C = -L/4, A_i = e_i e_i^T, b = 1.
    L_ii = sum_k w_ik and L_ij = -w_ij on edges, so C_ii = -deg_w(i)/4, C_ij = w_ij/4."""
    ei = np.asarray(ei, np.int64)
    ej = np.asarray(ej, np.int64)
    w = np.asarray(w, np.float64)
    degw = np.bincount(ei, weights=w, minlength=n) + np.bincount(ej, weights=w, minlength=n)
    diag = np.arange(n, dtype=np.int64)
    c_i = np.concatenate([diag, np.minimum(ei, ej)])
    c_j = np.concatenate([diag, np.maximum(ei, ej)])
    c_v = np.concatenate([-degw / 4.0, w / 4.0])
    return Instance(
        n=n, m=n,
        c_i=c_i.astype(np.int32), c_j=c_j.astype(np.int32), c_v=c_v,
        a_k=diag.astype(np.int32), a_i=diag.astype(np.int32), a_j=diag.astype(np.int32),
        a_v=np.ones(n), b=np.ones(n), name=name, kind="maxcut", graph=(ei, ej, w),
    )


def lovasz_theta(n: int, ei, ej, name: str = "") -> Instance:
    """Lovasz theta SDP: min <-J, X> s.t. tr X = 1 (constraint 0) and X_ij = 0 for
    every edge (constraint 1 + e, written (e_i e_j^T + e_j e_i^T)/2, b = 0).
    -J is carried as the low-rank term s u u^T with u = 1, s = -1."""
    ei = np.asarray(ei, np.int64)
    ej = np.asarray(ej, np.int64)
    ne = ei.shape[0]
    diag = np.arange(n, dtype=np.int64)
    a_k = np.concatenate([np.zeros(n, np.int64), 1 + np.arange(ne, dtype=np.int64)])
    a_i = np.concatenate([diag, np.minimum(ei, ej)])
    a_j = np.concatenate([diag, np.maximum(ei, ej)])
    a_v = np.concatenate([np.ones(n), np.full(ne, 0.5)])
    b = np.zeros(1 + ne)
    b[0] = 1.0
    return Instance(
        n=n, m=1 + ne,
        c_i=np.zeros(0, np.int32), c_j=np.zeros(0, np.int32), c_v=np.zeros(0),
        a_k=a_k.astype(np.int32), a_i=a_i.astype(np.int32), a_j=a_j.astype(np.int32),
        a_v=a_v, b=b, c_lr_u=np.ones((1, n)), c_lr_s=np.array([-1.0]),
        name=name, kind="theta", graph=(ei, ej, np.ones(ne)),
    )


def matrix_completion(n1: int, n2: int, rank: int, seed, m: int | None = None) -> Instance:
    """Nuclear-norm matrix completion as an SDP (Sec. 6.2): min tr(X)/2 over
    X = [[W1, Y], [Y^T, W2]] >= 0 with Y_ij = M_ij on the observed set.  M = U V^T with
    standard Gaussian U (n1 x rank), V (n2 x rank); the observed entries are a uniform
    sample of m distinct positions, m = ceil(gamma rank (n - rank)) with oversampling
    gamma = rank log(n), n = n1 + n2 (capped at n1 n2).  Constraint k is the off-diagonal
    entry (i, n1 + j) with value 1/2, i.e. X_{i, n1+j} = M_ij (b_k = M_ij); C = I/2."""
    rng = _rng(seed)
    n = n1 + n2
    U = rng.standard_normal((n1, rank))
    V = rng.standard_normal((n2, rank))
    if m is None:
        m = int(math.ceil(rank * math.log(n) * rank * (n - rank)))
    m = min(m, n1 * n2)
    pos = np.sort(rng.choice(n1 * n2, size=m, replace=False))
    oi, oj = pos // n2, pos % n2
    b = np.einsum("ij,ij->i", U[oi], V[oj])
    diag = np.arange(n, dtype=np.int64)
    return Instance(
        n=n, m=m,
        c_i=diag.astype(np.int32), c_j=diag.astype(np.int32), c_v=np.full(n, 0.5),
        a_k=np.arange(m, dtype=np.int32), a_i=oi.astype(np.int32), a_j=(n1 + oj).astype(np.int32),
        a_v=np.full(m, 0.5), b=b, name=f"mc-{n1}x{n2}-r{rank}", kind="mc",
        graph=(U, V, None),
    )


# ----------------------------------------------------------------------------------
# graphs shaped like the paper's MaxCut test families (Sec. 6.1, Tab. 1), by recipe only
# ----------------------------------------------------------------------------------
def rgg_edges(n: int, seed, radius_factor: float = 0.55) -> tuple[np.ndarray, np.ndarray]:
    """Random geometric graph: n uniform points in the unit square, an edge between points
    closer than radius_factor * sqrt(ln n / n) (the rule of the rgg_n_2_k family)."""
    from scipy.spatial import cKDTree

    rng = _rng(seed)
    pts = rng.random((n, 2))
    pairs = cKDTree(pts).query_pairs(radius_factor * math.sqrt(math.log(n) / n), output_type="ndarray")
    if pairs.size == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    i, j = pairs[:, 0].astype(np.int64), pairs[:, 1].astype(np.int64)
    return np.minimum(i, j), np.maximum(i, j)


def delaunay_edges(n: int, seed) -> tuple[np.ndarray, np.ndarray]:
    """Delaunay triangulation of n uniform points in the unit square (the delaunay_n_k family)."""
    from scipy.spatial import Delaunay

    rng = _rng(seed)
    tri = Delaunay(rng.random((n, 2))).simplices.astype(np.int64)
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [0, 2]]])
    e = np.unique(np.sort(e, axis=1), axis=0)
    return e[:, 0], e[:, 1]


def kron_edges(scale: int, seed, edge_factor: int = 16,
               abc: tuple[float, float, float] = (0.57, 0.19, 0.19)) -> tuple[np.ndarray, np.ndarray]:
    """Kronecker (R-MAT) graph on 2^scale vertices: edge_factor * 2^scale edges, each placed
    by choosing one of the four quadrants with probabilities (a, b, c, 1-a-b-c) at every
    level, then vertex labels permuted at random; loops and repeated edges dropped (a
    heavy-tailed degree distribution like the kron_g500 family)."""
    rng = _rng(seed)
    n = 1 << scale
    ne = edge_factor * n
    a, b, c = abc
    i = np.zeros(ne, np.int64)
    j = np.zeros(ne, np.int64)
    for _ in range(scale):
        u = rng.random(ne)
        ibit = (u >= a + b).astype(np.int64)                       # quadrants c, d: lower half
        jbit = (((u >= a) & (u < a + b)) | (u >= a + b + c)).astype(np.int64)  # quadrants b, d
        i = 2 * i + ibit
        j = 2 * j + jbit
    perm = rng.permutation(n)
    i, j = perm[i], perm[j]
    keep = i != j
    e = np.unique(np.stack([np.minimum(i[keep], j[keep]), np.maximum(i[keep], j[keep])], axis=1), axis=0)
    return e[:, 0], e[:, 1]


def rgg_maxcut(n: int, seed=7) -> Instance:
    ei, ej = rgg_edges(n, (seed, 0))
    return maxcut(n, ei, ej, np.ones(ei.shape[0]), name=f"maxcut-rgg-n{n}")


def delaunay_maxcut(n: int, seed=8) -> Instance:
    ei, ej = delaunay_edges(n, (seed, 0))
    return maxcut(n, ei, ej, np.ones(ei.shape[0]), name=f"maxcut-delaunay-n{n}")


def kron_maxcut(scale: int, seed=9) -> Instance:
    ei, ej = kron_edges(scale, (seed, 0))
    return maxcut(1 << scale, ei, ej, np.ones(ei.shape[0]), name=f"maxcut-kron-s{scale}")


def factor_init(n: int, r: int, seed, scale: float | None = None) -> np.ndarray:
    """Seeded Gaussian starting factor R0 (n x r, float64), entries N(0, scale^2);
    by default scale = 1/sqrt(r), so that E||r_i||^2 = 1 (the MaxCut diagonal)."""
    rng = _rng(seed)
    if scale is None:
        scale = 1.0 / math.sqrt(max(r, 1))
    return rng.standard_normal((n, r)) * scale


# ----------------------------------------------------------------------------------
# the named workloads (sizes and seeds of the benchmark configurations)
# ----------------------------------------------------------------------------------
def er_maxcut(n: int = 800, p: float = 0.06, seed=1, weights: str = "unit") -> Instance:
    ei, ej = er_edges(n, p, (seed, 0))
    w = edge_weights(ei.shape[0], weights, (seed, 1))
    return maxcut(n, ei, ej, w, name=f"maxcut-er-n{n}-p{p}")


def torus_maxcut(n1: int = 1000, n2: int = 1000, seed=2, weights: str = "pm1") -> Instance:
    ei, ej = torus_edges(n1, n2)
    w = edge_weights(ei.shape[0], weights, (seed, 1))
    return maxcut(n1 * n2, ei, ej, w, name=f"maxcut-torus-{n1}x{n2}-{weights}")


def regular3_maxcut(n: int, seed=4) -> Instance:
    ei, ej = regular3_edges(n, (seed, 0))
    return maxcut(n, ei, ej, np.ones(ei.shape[0]), name=f"maxcut-3reg-n{n}")


def theta_er(n: int = 20000, avg_deg: float = 20.0, seed=3) -> Instance:
    ei, ej = er_edges(n, avg_deg / (n - 1), (seed, 0))
    return lovasz_theta(n, ei, ej, name=f"theta-er-n{n}-d{avg_deg}")


def batch_specs(count: int = 4096, seed=6, n_lo: int = 64, n_hi: int = 4096,
                d_lo: float = 3.0, d_hi: float = 30.0) -> list[tuple[int, float, tuple]]:
    """(n, p, sub-seed) of each instance of a batch of ER MaxCut SDPs with
    n ~ U{n_lo..n_hi} and average degree ~ U[d_lo, d_hi]."""
    rng = _rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    ds = rng.uniform(d_lo, d_hi, size=count)
    return [(int(ns[i]), float(min(1.0, ds[i] / (ns[i] - 1))), (seed, i)) for i in range(count)]


# ----------------------------------------------------------------------------------
# worked examples of the paper, as problem data
# ----------------------------------------------------------------------------------
def t8_instance() -> Instance:
    """Sec. 3.2 (necessity of localness for low rank), n = 2, m = 3: C = 0,
    X_11 = 1, X_12 = 0, X_11 + X_22 = 1."""
    return Instance(
        n=2, m=3,
        c_i=np.zeros(0, np.int32), c_j=np.zeros(0, np.int32), c_v=np.zeros(0),
        a_k=np.array([0, 1, 2, 2], np.int32), a_i=np.array([0, 0, 0, 1], np.int32),
        a_j=np.array([0, 1, 0, 1], np.int32), a_v=np.array([1.0, 0.5, 1.0, 1.0]),
        b=np.array([1.0, 0.0, 1.0]), name="paper-example-n2-m3", kind="example",
    )


def t11_instance() -> Instance:
    """Sec. 3.2 (necessity of localness for quadratic growth): C = 0, A_1 = e_1 e_1^T,
    A_2 = e_2 e_2^T, b = (0, 1)."""
    return Instance(
        n=2, m=2,
        c_i=np.zeros(0, np.int32), c_j=np.zeros(0, np.int32), c_v=np.zeros(0),
        a_k=np.array([0, 1], np.int32), a_i=np.array([0, 1], np.int32),
        a_j=np.array([0, 1], np.int32), a_v=np.array([1.0, 1.0]),
        b=np.array([0.0, 1.0]), name="paper-example-qg", kind="example",
    )


def t15_instance(d: int, eps: float, a: float) -> Instance:
    """Sec. 4.3 (necessity of dual localness), with the dimension read as d = n:
    A_i = (e_i e_d^T + e_d e_i^T)/2 for i < d, A_d = eps*I, C = eps*diag(2 I_{d-1}, 1),
    b = eps*a*e_d."""
    n = d
    k_off = np.arange(d - 1, dtype=np.int64)
    a_k = np.concatenate([k_off, np.full(d, d - 1)])
    a_i = np.concatenate([k_off, np.arange(d)])
    a_j = np.concatenate([np.full(d - 1, d - 1), np.arange(d)])
    a_v = np.concatenate([np.full(d - 1, 0.5), np.full(d, eps)])
    c_v = np.full(d, 2 * eps)
    c_v[-1] = eps
    b = np.zeros(d)
    b[-1] = eps * a
    return Instance(
        n=n, m=d,
        c_i=np.arange(d, dtype=np.int32), c_j=np.arange(d, dtype=np.int32), c_v=c_v,
        a_k=a_k.astype(np.int32), a_i=a_i.astype(np.int32), a_j=a_j.astype(np.int32),
        a_v=a_v, b=b, name=f"paper-spurious-d{d}", kind="example",
    )


def random_general(n: int, m: int, seed, c_density: float = 0.05, per_con: int = 3,
                   lr_k: int = 1, diag_frac: float = 0.5) -> Instance:
    """A random SDP exercising every data path: sparse symmetric C with diagonal and
    off-diagonal entries, an optional low-rank part of C, constraints with several
    entries each (diagonal and off-diagonal, some entries shared between
    constraints), plus m_sel selector constraints (one entry each)."""
    rng = _rng(seed)
    # C: random off-diagonal entries and a random diagonal
    npairs = n * (n - 1) // 2
    cnt = int(rng.binomial(npairs, c_density)) if npairs else 0
    t = np.sort(rng.choice(npairs, size=cnt, replace=False)) if cnt else np.zeros(0, np.int64)
    ci, cj = _tri_index_to_pair(t, n) if cnt else (np.zeros(0, np.int64), np.zeros(0, np.int64))
    diag = np.arange(n, dtype=np.int64)
    c_i = np.concatenate([diag, ci])
    c_j = np.concatenate([diag, cj])
    c_v = np.concatenate([rng.uniform(-1, 1, n), rng.uniform(-1, 1, cnt)])
    # constraints
    ks, is_, js, vs = [], [], [], []
    for k in range(m):
        e = int(rng.integers(1, per_con + 1))
        for _ in range(e):
            if rng.random() < diag_frac:
                i = j = int(rng.integers(0, n))
            else:
                i, j = sorted(rng.choice(n, size=2, replace=False).tolist())
            ks.append(k); is_.append(i); js.append(j); vs.append(float(rng.uniform(-1, 1)))
    b = rng.uniform(-1, 1, m)
    u = rng.standard_normal((lr_k, n)) / math.sqrt(n)
    s = rng.uniform(-1, 1, lr_k)
    return Instance(
        n=n, m=m, c_i=c_i.astype(np.int32), c_j=c_j.astype(np.int32), c_v=c_v,
        a_k=np.array(ks, np.int32), a_i=np.array(is_, np.int32), a_j=np.array(js, np.int32),
        a_v=np.array(vs), b=b, c_lr_u=u if lr_k else np.zeros((0, 0)),
        c_lr_s=s if lr_k else np.zeros(0), name=f"random-general-n{n}-m{m}", kind="general",
    )
