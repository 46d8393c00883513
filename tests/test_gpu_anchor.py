"""The fused form's anchored phase path against the FP64 oracle, and its selection.

On the anchored path each group of 16 consecutive points forms the exact
phase (Eq. 3's f . x mod 1, fixed point or double-float) at its first and
last point only;
every point adds its FP32 offset from the nearer of the two.  The path applies
when fmax times the largest such offset is at most 8 turns; otherwise the
exact per-point paths run.  Tolerance: the field tolerance of every synthesis
form, |gpu - oracle| <= 1e-5 sigma per value, sigma^2 = sum_k F_k^2 of the
realisation.  Which path ran is seen by comparing with a handle created under
QRS_SYNTH_ANCHOR=0 (exact paths only): results differ in their rounding where
the anchored path ran and are identical where it did not.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2404_02978_gb300 as qrs
from paper_2404_02978_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
TOL_FIELD = 1e-5


@pytest.fixture(scope="module")
def handles():
    from paper_2404_02978_gb300 import build as B
    B.build()
    anchored = qrs.Handle(0)
    mp = pytest.MonkeyPatch()
    mp.setenv("QRS_SYNTH_ANCHOR", "0")
    try:
        exact = qrs.Handle(0)
    finally:
        mp.undo()
    return anchored, exact


def _sigma(p, n_f, n_real, off):
    d = oracle.draw(p, n_f=n_f, n_real=n_real, real_offset=off)
    return np.sqrt(np.sum(d["F"] ** 2, axis=1))


def _run(h, p, n_f, n_real, xy, off):
    out = qrs.qrs_synthesize_points(h, p, n_f, n_real, torch.from_numpy(np.ascontiguousarray(xy)).cuda(),
                                    real_offset=off)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _line(n, step, y=0.0):
    return np.stack([np.arange(n) * step - 0.5 * n * step, np.full(n, y)], -1).astype(np.float32)


def _track():
    # two telescopes' tracks sampled every 1 ms under a 10.2 m/s wind along
    # the 56.5 m baseline (Sec. 4.3 geometry), 1000 samples each
    t = np.arange(1000) * 1e-3
    ut1 = np.stack([-10.2 * t, np.zeros_like(t)], -1)
    ut2 = np.stack([56.5 - 10.2 * t, np.zeros_like(t)], -1)
    return np.concatenate([ut1, ut2]).astype(np.float32)


CASES = [
    # the phase screen's 256^2 pupil grid (dx = 8/256 m): groups cross rows,
    # ragged tail (7001 points: 3.4 tiles of 2048, a 9-point last group),
    # 700 terms (a 60-term last partial sum)
    dict(name="pupil256", pts=lambda: wl.pupil_grid(256, 8.0)[:7001],
         p=dict(domain="logpolar", fmax=16.0), n_f=700, n_real=2, anchored=True),
    # more terms than one shared-memory chunk (the chunk re-draw path)
    dict(name="pupil256-multichunk", pts=lambda: wl.pupil_grid(256, 8.0)[20000:21500],
         p=dict(domain="logpolar", fmax=16.0), n_f=4096 + 301, n_real=2, anchored=True),
    # literal Eq. 3 coefficients, square domain
    dict(name="pupil256-square-eq3", pts=lambda: wl.pupil_grid(256, 8.0)[9000:12000],
         p=dict(domain="square", fmax=4.0, coef="eq3"), n_f=37 * 37, n_real=2, anchored=True),
    # the pupil grid 170 m off the origin: f_max |x| far above the fixed-point
    # limit, so the anchors take the double-float reduction
    dict(name="pupil256-offset-df", pts=lambda: wl.pupil_grid(256, 8.0)[:5000] + np.float32([150.0, -80.0]),
         p=dict(domain="logpolar", fmax=16.0), n_f=600, n_real=2, anchored=True),
    # the Sec. 4.3 tracks with the Eq. 7 piston PSD: |x| up to 56.5 m, a group
    # that straddles the two tracks takes one anchor on each
    dict(name="track-piston", pts=_track,
         p=dict(domain="square", fmax=0.25, L0=22.0, r0=0.10, ap_D=8.0, ap_d=1.1), n_f=44 * 44, n_real=2,
         anchored=True),
    # one term, and one term past a whole 64-term partial sum
    dict(name="one-term", pts=lambda: wl.pupil_grid(256, 8.0)[3000:3500],
         p=dict(domain="logpolar", fmax=16.0), n_f=1, n_real=3, anchored=True),
    dict(name="65-terms", pts=lambda: wl.pupil_grid(256, 8.0)[3000:3500],
         p=dict(domain="logpolar", fmax=16.0), n_f=65, n_real=3, anchored=True),
    # fewer points than one group
    dict(name="five-points", pts=lambda: _line(5, 0.01, 0.3),
         p=dict(domain="logpolar", fmax=16.0), n_f=300, n_real=3, anchored=True),
    # a line of 128 points 0.065 m apart (whole groups): largest offset 7 x 0.065 m,
    # 16 x 0.455 = 7.3 turns
    dict(name="line-below-limit", pts=lambda: _line(128, 0.065), p=dict(domain="logpolar", fmax=16.0), n_f=300,
         n_real=2, anchored=True),
    # 0.08 m apart: 16 x 0.56 = 9.0 turns, above the limit: exact paths
    dict(name="line-above-limit", pts=lambda: _line(128, 0.08), p=dict(domain="logpolar", fmax=16.0), n_f=300,
         n_real=2, anchored=False),
    # the pupil grid in a random order: offsets span the pupil, exact paths
    dict(name="scattered", pts=lambda: wl.pupil_grid(256, 8.0)[np.random.default_rng(5).permutation(51468)[:4000]],
         p=dict(domain="logpolar", fmax=16.0), n_f=500, n_real=2, anchored=False),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c["name"])
def test_anchored_path_parity_and_selection(handles, case):
    anchored, exact = handles
    xy = case["pts"]()
    p = oracle.params(seed=41, **case["p"])
    off = 3
    ref = oracle.synthesize(p, case["n_f"], case["n_real"], xy, real_offset=off)
    sig = _sigma(p, case["n_f"], case["n_real"], off)
    got = _run(anchored, p, case["n_f"], case["n_real"], xy, off)
    base = _run(exact, p, case["n_f"], case["n_real"], xy, off)
    for out in (got, base):
        assert np.isfinite(out).all()
        err = np.abs(out.astype(np.float64) - ref) / sig[:, None]
        assert err.max() <= TOL_FIELD, "max err %.3g sigma" % err.max()
    assert np.array_equal(got, base) != case["anchored"]


def test_anchored_path_phase_screen_rows(handles):
    """Whole rows of the phase screen's pupil grid, one realisation of the
    benchmark draw (N_f = 4096): the anchored path's errors against the oracle
    are of the exact path's size (rms within 1e-6 sigma, as the full-size
    check asks), not only within the per-value tolerance."""
    anchored, exact = handles
    cfg = wl.PHASE_SCREEN
    p = wl.method_params(cfg)
    xy = wl.pupil_grid(cfg["grid"], cfg["pupil"])[24000:27000]
    off = 11
    ref = oracle.synthesize(p, cfg["n_f"], 1, xy, real_offset=off)
    sig = _sigma(p, cfg["n_f"], 1, off)
    got = _run(anchored, p, cfg["n_f"], 1, xy, off)
    base = _run(exact, p, cfg["n_f"], 1, xy, off)
    assert not np.array_equal(got, base)
    e_anchor = (got.astype(np.float64) - ref) / sig[:, None]
    e_exact = (base.astype(np.float64) - ref) / sig[:, None]
    rms_a, rms_e = np.sqrt(np.mean(e_anchor ** 2)), np.sqrt(np.mean(e_exact ** 2))
    print("anchored: max %.3g rms %.3g sigma; exact: max %.3g rms %.3g sigma"
          % (np.abs(e_anchor).max(), rms_a, np.abs(e_exact).max(), rms_e))
    assert np.abs(e_anchor).max() <= TOL_FIELD
    assert rms_a <= 1e-6
