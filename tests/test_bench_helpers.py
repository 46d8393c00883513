"""Host-side helpers of bench.py that its reported figures depend on.

The learned-proposal gain is measured against bench.hankel_piston_sf, the
expected differential-piston structure function of Sec. 4.4 (Eq. 7 filter,
von Karman PSD) over the sampled annulus. The measurement may not call the
oracle, so the helper is a separate quadrature; here it is pinned to the
oracle's analytic form, itself pinned to the Monte Carlo of the plain method.
"""
import numpy as np
import pytest

import bench
from oracle import analytic as an


@pytest.mark.parametrize("B", [1.0, 10.0, 56.5, 200.0])
@pytest.mark.parametrize("r0,L0,D", [(0.05, 10.0, 1.0), (0.15, 30.0, 8.0), (0.3, 100.0, 3.3)])
def test_hankel_piston_sf_matches_the_oracle_form(B, r0, L0, D):
    got = bench.hankel_piston_sf(B, r0, L0, D, 1e-3, 10.0)
    ref = an.piston_sf(B, r0, L0, D, 0.0, 1e-3, 10.0)
    assert got == pytest.approx(ref, rel=1e-6)


def test_hankel_piston_sf_limits():
    """Zero at zero baseline; twice the single-aperture piston variance when the
    apertures are far apart (the J0 term averages out)."""
    r0, L0, D = 0.15, 30.0, 2.0
    assert bench.hankel_piston_sf(1e-9, r0, L0, D, 1e-3, 10.0) == pytest.approx(0.0, abs=1e-12)
    far = bench.hankel_piston_sf(1e5, r0, L0, D, 1.0, 10.0)
    assert far == pytest.approx(2 * an.piston_variance(r0, L0, D, 0.0, 1.0, 10.0), rel=1e-3)
    assert np.isfinite(far)


@pytest.mark.parametrize("r", [0.05, 0.5, 2.0, 8.0, 40.0])
def test_vk_phase_sf_matches_the_oracle_closed_form(r):
    assert bench.vk_phase_sf(r, 0.15, 30.0) == pytest.approx(an.phase_sf_vk_infinite(r, 0.15, 30.0), rel=1e-10)


@pytest.mark.parametrize("r", [0.1, 1.0, 4.0])
def test_hankel_phase_sf_matches_the_oracle_quadrature(r):
    got = bench.hankel_phase_sf(r, 0.15, 30.0, 1e-3, 16.0)
    ref = an.phase_sf(r, 0.15, 30.0, 1e-3, 16.0)
    assert got == pytest.approx(ref, rel=1e-6)
