"""Sampling statistics on the GPU against the oracle: nearest-neighbour
distances (FP32, 1e-6 relative) and the star discrepancy (exact integer counts
and exact FP64 products: bit-exact).  Draws of the three samplers the paper
compares (Sec. 2.3, 3.2: jittered grid, uniform random, quasi-random R2) on the
SQUARE domain with fmax = 0.5, shifted into [0,1]^2."""
import numpy as np
import pytest
import torch

import oracle
import paper_2404_02978_gb300 as qrs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_2404_02978_gb300 import build as B
    B.build()
    return qrs.Handle(0)


def unit_draw(h, sampler, n_side, n_real, seed, real_offset=0):
    """A realisation's frequencies in [0,1]^2 (SQUARE, fmax 0.5, +0.5): [n_real, n, 2] float32."""
    p = qrs.params(domain="square", fmax=0.5, sampler=sampler, seed=seed, n_rho=n_side, n_theta=n_side)
    d = qrs.qrs_draw(h, p, n_side * n_side, n_real, real_offset=real_offset, outputs=("f_xy",))
    return d["f_xy"] + 0.5


@pytest.mark.parametrize("sampler", ["r2", "jitter", "uniform"])
def test_nearest_neighbour_parity(h, sampler):
    pts = unit_draw(h, sampler, 31, 3, seed=41)  # 961 points per set
    got = qrs.qrs_nearest_neighbour(h, pts)
    qrs.qrs_sync(h)
    ref = oracle.nearest_neighbour(pts.cpu().numpy())
    assert np.allclose(got.cpu().numpy(), ref, rtol=1e-6, atol=0)


def test_star_discrepancy_bit_exact(h):
    sets = [unit_draw(h, s, 14, 2, seed=42).cpu().numpy() for s in ("r2", "jitter", "uniform")]
    c = (np.arange(14) + 0.5) / 14
    grid = np.stack(np.meshgrid(c, c), -1).reshape(1, -1, 2).astype(np.float32)
    pts = np.concatenate(sets + [grid])  # 7 sets of 196 points
    got = qrs.qrs_star_discrepancy(h, torch.from_numpy(pts).cuda())
    qrs.qrs_sync(h)
    ref = oracle.star_discrepancy(pts)
    assert np.array_equal(got.cpu().numpy(), ref)
    assert got[-1].item() == pytest.approx(1 / 14 - 1 / (4 * 14 * 14), abs=1e-7)
    one = qrs.qrs_star_discrepancy(h, torch.tensor([[0.9, 0.95]], device="cuda"))
    assert one.item() == pytest.approx(float(np.float32(0.95)), abs=0)


def test_stats_arguments(h):
    x = torch.zeros(2, 0, 2, device="cuda")
    with pytest.raises(qrs.QrsError):
        qrs.qrs_star_discrepancy(h, x)


def test_quasi_random_has_no_clusters_or_gaps(h):
    """Sec. 3.2, Figs. 2-3 as numbers (1024 terms, 16 realisations each): R2
    keeps every nearest neighbour beyond a quarter cell and has the lowest
    discrepancy, per realisation and over 4 consecutive realisations (its
    stream continues); jittered grids show clusters, uniform draws more."""
    share, disc, union = {}, {}, {}
    for smp in ("r2", "jitter", "uniform"):
        pts = unit_draw(h, smp, 32, 16, seed=43)
        nn = qrs.qrs_nearest_neighbour(h, pts) * 32
        share[smp] = (nn < 0.25).float().mean().item()
        disc[smp] = qrs.qrs_star_discrepancy(h, pts).mean().item()
        union[smp] = qrs.qrs_star_discrepancy(h, pts[:4].reshape(1, 4096, 2)).item()
    qrs.qrs_sync(h)
    print("share < 1/4 cell", share, "D*", disc, "union D*", union)
    assert share["r2"] == 0.0 and share["jitter"] > 0.01 and share["uniform"] > 0.1
    assert disc["r2"] < 0.8 * disc["jitter"] and disc["jitter"] < 0.6 * disc["uniform"]
    assert union["r2"] < 0.6 * union["jitter"] and union["jitter"] < 0.7 * union["uniform"]
