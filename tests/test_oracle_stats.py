"""Pins of the sampling statistics (nearest-neighbour distance, star
discrepancy) used to compare jittered, random and quasi-random draws
(Sec. 2.3, 3.2, Figs. 2-3).

* Nearest neighbours against scipy's k-d tree, and on a regular grid.
* Star discrepancy: closed forms (one point: max(1 - ab, a, b); the centred
  m x m grid: 1/m - 1/(4 m^2)), and an independent brute force of the
  definition (sup of |count/n - uv| over box corners nudged just inside and
  just outside every point coordinate).
"""
import numpy as np
import pytest

import oracle


def test_nearest_neighbour_vs_kdtree_and_grid():
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(0)
    pts = rng.uniform(size=(3, 500, 2)).astype(np.float32)
    nn = oracle.nearest_neighbour(pts)
    for s in range(3):
        d, _ = cKDTree(pts[s].astype(np.float64)).query(pts[s].astype(np.float64), k=2)
        assert np.allclose(nn[s], d[:, 1], rtol=1e-12, atol=0)
    g = (np.stack(np.meshgrid(np.arange(8), np.arange(8)), -1).reshape(-1, 2) * 0.125).astype(np.float32)
    assert np.allclose(oracle.nearest_neighbour(g), 0.125)
    assert oracle.nearest_neighbour(np.float32([[0.3, 0.4]]))[0, 0] == 0.0


def test_star_discrepancy_closed_forms():
    for a, b in ((0.3, 0.6), (0.9, 0.95), (0.5, 0.25)):
        a32, b32 = float(np.float32(a)), float(np.float32(b))
        assert oracle.star_discrepancy(np.float32([[a, b]]))[0] == pytest.approx(max(1 - a32 * b32, a32, b32), abs=1e-15)
    for m in (2, 3, 5, 8):
        c = (np.arange(m) + 0.5) / m
        g = np.stack(np.meshgrid(c, c), -1).reshape(-1, 2).astype(np.float32)
        assert oracle.star_discrepancy(g)[0] == pytest.approx(1 / m - 1 / (4 * m * m), abs=1e-7)


def test_star_discrepancy_vs_brute_force_definition():
    rng = np.random.default_rng(1)
    eps = 1e-9
    for n in (5, 17, 40):
        p = rng.uniform(size=(n, 2)).astype(np.float32).astype(np.float64)
        us = np.unique(np.concatenate([p[:, 0] - eps, p[:, 0] + eps, [1.0]]))
        vs = np.unique(np.concatenate([p[:, 1] - eps, p[:, 1] + eps, [1.0]]))
        us, vs = us[(us > 0) & (us <= 1)], vs[(vs > 0) & (vs <= 1)]
        inside = (p[None, None, :, 0] < us[:, None, None]) & (p[None, None, :, 1] < vs[None, :, None])
        brute = np.max(np.abs(inside.sum(-1) / n - us[:, None] * vs[None, :]))
        assert oracle.star_discrepancy(p.astype(np.float32))[0] == pytest.approx(brute, abs=3 * eps)
