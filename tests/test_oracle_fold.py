"""Pins of the oracle's folded baseline-frame cells (the learned proposal's
sampler and targets) against things other than themselves.

The differential-piston structure function at a baseline B depends on a
frequency only through |f| and |cos(angle between f and B)|, so a density over
log-polar cells may be laid out in the frame of B and repeated over F = 2 or 4
mirrored sectors of 1/F turn without changing what it estimates.

* Unbiased: E sum_k w_k over folded importance draws equals the closed-form
  annulus integral (Parseval), for any cell density, any fold and any frame.
* Geometry: every drawn frequency lies in one of the F mirror images of its
  cell (angles from atan2 in FP64, independent of the integer decision), and
  cells are hit in proportion to the quantised cell probabilities.
* Uniform logits: the folded sampler still draws uniform angles (KS).
* Continuity: the angle is a continuous, increasing function of the R2
  coordinate over the whole turn (a planted sampler that does not mirror the
  odd sectors fails here and nowhere else: it is valid, but breaks the
  stratification at sector edges).
* Targets: the folded cells regroup the unfolded ones exactly (sector q, cell i
  of F sectors = cell q n + i, or q n + n - 1 - i in mirrored sectors, of the
  whole-turn grid with F n cells); a baseline along +x gives the draw's own
  cells; a baseline along +y gives them shifted by a quarter turn.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import oracle.proposal as pr
from cdf_inputs import two_level_cdf
from oracle import analytic as an

DOM = (1e-3, 16.0)


def _angles_in_frame(f, frame):
    """Turns of each frequency relative to the frame, in [0, 1) (FP64 atan2)."""
    th = np.arctan2(f[..., 1].astype(np.float64), f[..., 0].astype(np.float64)) / (2 * np.pi)
    return np.mod(th - frame, 1.0)


@pytest.mark.parametrize("fold,frame", [(2, 0.3), (4, 0.3), (4, -0.125), (1, 0.71)])
def test_folded_importance_is_unbiased_and_in_its_cells(fold, frame):
    nr, nt = 12, 6
    nc = nr * nt
    rng = np.random.default_rng(17 + fold)
    p_c = 0.5 * rng.dirichlet(np.ones(nc)) + 0.5 / nc
    cdf, p_q = two_level_cdf(p_c, nr, nt)
    p = oracle.params(sampler="importance", n_rho=nr, n_theta=nt, cdf=cdf, r0=0.15, L0=30.0,
                      fmin=DOM[0], fmax=DOM[1], seed=19, fold=fold, frame=frame)
    d = oracle.draw(p, n_f=1024, n_real=30)
    E = an.parseval_annulus(0.15, 30.0, *DOM)
    assert np.mean(np.sum(d["F"] ** 2, axis=1)) == pytest.approx(E, rel=3e-2)
    # the radial band
    L = math.log(DOM[1] / DOM[0])
    rho = np.hypot(d["f"][..., 0], d["f"][..., 1]).astype(float)
    ir = d["cell"] // nt
    assert np.all(rho >= DOM[0] * np.exp(L * ir / nr) * (1 - 1e-6))
    assert np.all(rho <= DOM[0] * np.exp(L * (ir + 1) / nr) * (1 + 1e-6))
    # the angular cell, through the mirror images of the sector
    w = _angles_in_frame(d["f"], frame) * fold
    q = np.floor(w)
    v = w - q
    v = np.where(q % 2 == 1, 1.0 - v, v) * nt
    it = d["cell"] % nt
    near = np.abs(v - np.round(v)) < 1e-4  # FP32 frequencies on a cell edge
    assert np.all((np.floor(v) == it) | near)
    assert np.mean(near) < 1e-3
    # every sector is visited equally often, cells follow p_c
    cnt_q = np.bincount(np.minimum(q.astype(int).ravel(), fold - 1), minlength=fold)
    assert np.all(np.abs(cnt_q / cnt_q.sum() - 1.0 / fold) < 0.01)
    cnt = np.bincount(d["cell"].ravel(), minlength=nc)
    assert stats.chisquare(cnt, p_q * cnt.sum()).pvalue > 1e-4


def test_folded_uniform_density_draws_uniform_angles():
    nr, nt = 8, 8
    cdf, _ = two_level_cdf(np.ones(nr * nt), nr, nt)
    p = oracle.params(sampler="importance", n_rho=nr, n_theta=nt, cdf=cdf, fmin=DOM[0], fmax=DOM[1], seed=23,
                      fold=4, frame=0.05)
    d = oracle.draw(p, n_f=4096, n_real=2)
    th = _angles_in_frame(d["f"], 0.0).ravel()
    assert stats.kstest(th, "uniform").pvalue > 1e-3
    # log-radial uniform as well
    L = math.log(DOM[1] / DOM[0])
    u = np.log(np.hypot(d["f"][..., 0], d["f"][..., 1]).astype(float).ravel() / DOM[0]) / L
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def _raw(n_theta, fold, g, kind):
    return pr.targets("von_karman", (1e-3, 10.0), 16, n_theta, 31, 2048, 4, g, raw=True, kind=kind, fold=fold)


@pytest.mark.parametrize("kind", ["mean", "rms"])
def test_folded_targets_regroup_the_whole_turn_cells(kind):
    g = np.array([[0.1, 25.0, 1.0, 10.0, 3.0], [0.15, 40.0, 8.0, -20.0, 56.5], [0.08, 20.0, 2.0, 3.0, -4.0]])
    n = 8
    whole = _raw(4 * n, 1, g, kind).reshape(len(g), 16, 4, n)  # baseline frame, no fold
    folded = _raw(n, 4, g, kind).reshape(len(g), 16, n)
    half = _raw(2 * n, 2, g, kind).reshape(len(g), 16, 2 * n)
    # sector q, cell i of the folded grid = whole-turn cell q n + i, mirrored in odd sectors
    copies = np.stack([whole[:, :, 0], whole[:, :, 1, ::-1], whole[:, :, 2], whole[:, :, 3, ::-1]], 2)
    halves = np.stack([whole.reshape(len(g), 16, 4 * n)[:, :, :2 * n],
                       whole.reshape(len(g), 16, 4 * n)[:, :, 2 * n:][:, :, ::-1]], 2)
    if kind == "rms":
        assert np.allclose(folded ** 2, (copies ** 2).sum(2), rtol=1e-10, atol=0)
        assert np.allclose(half ** 2, (halves ** 2).sum(2), rtol=1e-10, atol=0)
    else:
        assert np.allclose(folded, copies.sum(2), rtol=1e-10, atol=0)
        assert np.allclose(half, halves.sum(2), rtol=1e-10, atol=0)


def test_baseline_frame_is_the_rotated_draw_frame():
    n = 16
    gx = np.array([[0.1, 25.0, 2.0, 30.0, 0.0]])  # along +x: the frame is the draw's own
    assert np.array_equal(_raw(n, 1, gx, "mean"), _raw(n, 0, gx, "mean"))
    gy = np.array([[0.1, 25.0, 2.0, 0.0, 30.0]])  # along +y: a quarter turn
    frame = _raw(n, 1, gy, "mean").reshape(16, n)
    own = _raw(n, 0, gy, "mean").reshape(16, n)
    assert np.array_equal(frame, np.roll(own, -n // 4, axis=1))


@pytest.mark.parametrize("fold", [2, 4])
def test_folded_map_is_continuous_and_increasing(fold):
    """Mirrored sectors make the angle a continuous, increasing function of
    the R2 coordinate y over the whole turn (the stratification of Eq. 6 is
    kept across sector edges): the point n = 0 is placed at s0 = (x, y)."""
    nr, nt = 4, 5
    rng = np.random.default_rng(29)
    cdf, _ = two_level_cdf(0.3 * rng.dirichlet(np.ones(nr * nt)) + 0.7 / (nr * nt), nr, nt)
    M = 1500
    ys = [(j * (2**64 // M) + 12345) % 2**64 for j in range(M)]
    th = []
    for y in ys:
        p = oracle.params(sampler="importance", n_rho=nr, n_theta=nt, cdf=cdf, fmin=DOM[0], fmax=DOM[1],
                          s0=(2**63 + 7, y), fold=fold, frame=0.2)
        th.append(_angles_in_frame(oracle.draw(p, n_f=1, n_real=1)["f"][0], 0.2)[0])
    d = np.diff(np.unwrap(np.asarray(th) * 2 * np.pi)) / (2 * np.pi)
    assert np.all(d > -1e-6)  # increasing (FP32 frequencies)
    assert np.max(d) < 20.0 / M  # no jumps: steps bounded by the densest cell's stretch


@pytest.mark.parametrize("fold", [1, 4])
def test_folded_importance_structure_function_is_unbiased(fold):
    """E[D_draw(B)] over importance draws in the baseline frame (a random cell
    density, not fitted to the geometry) equals the Hankel integral D(B) of
    Sec. 4.4 with the Eq. 7 filter, within 3 sigma of the draw-to-draw spread."""
    r0, L0, D, B = 0.1, 25.0, 2.0, np.array([30.0, 10.0])
    dom = (1e-3, 10.0)
    nr, nt = 16, 8
    rng = np.random.default_rng(41)
    cdf, _ = two_level_cdf(0.5 * rng.dirichlet(np.ones(nr * nt)) + 0.5 / (nr * nt), nr, nt)
    p = oracle.params(sampler="importance", n_rho=nr, n_theta=nt, cdf=cdf, r0=r0, L0=L0, fmin=dom[0], fmax=dom[1],
                      seed=43, fold=fold, frame=float(np.arctan2(B[1], B[0]) / (2 * np.pi)))
    d = oracle.draw(p, n_f=256, n_real=400)
    f = d["f"].astype(np.float64)
    A = an.airy(np.hypot(f[..., 0], f[..., 1]), D)
    sf = np.sum(d["F"] ** 2 * A ** 2 * 2 * (1 - np.cos(2 * np.pi * (f[..., 0] * B[0] + f[..., 1] * B[1]))), axis=1)
    ref = an.piston_sf(float(np.hypot(*B)), r0, L0, D, 0.0, *dom)
    assert abs(sf.mean() - ref) <= 3 * sf.std() / np.sqrt(sf.size)
