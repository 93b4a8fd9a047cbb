"""Seeded generators of graphs shaped like the paper's MaxCut families (random geometric,
Delaunay, Kronecker): the structural facts each recipe fixes."""
import math

import numpy as np

import sdp_instances as si


def _degrees(n, ei, ej):
    return np.bincount(ei, minlength=n) + np.bincount(ej, minlength=n)


def _simple(ei, ej):
    assert np.all(ei < ej)
    key = ei.astype(np.int64) * (int(ej.max()) + 1) + ej
    assert np.unique(key).size == key.size


def test_rgg_degree_matches_the_radius_rule():
    n = 20000
    ei, ej = si.rgg_edges(n, 1)
    _simple(ei, ej)
    # expected degree ~ pi r^2 n (boundary effects lower it a little), r = 0.55 sqrt(ln n / n)
    expect = math.pi * 0.55 ** 2 * math.log(n)
    mean = 2 * ei.size / n
    assert 0.9 * expect <= mean <= 1.01 * expect


def test_delaunay_is_a_planar_triangulation():
    n = 5000
    ei, ej = si.delaunay_edges(n, 2)
    _simple(ei, ej)
    # a triangulation of a point set with h hull points has 3n - 3 - h edges
    assert 2.9 * n <= ei.size <= 3 * n - 6
    assert np.all(_degrees(n, ei, ej) >= 2)


def test_kron_is_heavy_tailed_and_simple():
    scale = 12
    n = 1 << scale
    ei, ej = si.kron_edges(scale, 3)
    _simple(ei, ej)
    d = _degrees(n, ei, ej)
    assert ei.size > 5 * n                 # edge factor 16 before dropping loops and repeats
    assert d.max() > 20 * d.mean()         # heavy tail
    assert np.sum(d == 0) > 0.05 * n       # many isolated vertices, as in R-MAT graphs


def test_maxcut_wrappers():
    for inst in (si.rgg_maxcut(500), si.delaunay_maxcut(500), si.kron_maxcut(8)):
        assert inst.kind == "maxcut" and inst.m == inst.n
        assert np.all(inst.b == 1.0)
