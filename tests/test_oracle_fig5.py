"""Pins of the piston-PSD synthesis and of the Sec. 4.3-4.4 experiment's
reference values (CPU only).

* With the PSD filtered by the Eq. 7 aperture factor, the Eq. 3 sum at a point
  is the piston of an aperture centred there: the oracle's filtered synthesis
  equals its per-aperture piston code (a different code path) at aperture
  positions.
* Parseval for the filtered PSD: E sum F^2 = the piston variance over the
  annulus (LOGPOLAR) and the 2-D integral over the square (SQUARE, Sec. 4.3).
* The square-domain temporal structure function (2-D quadrature) equals the
  isotropic Hankel form when the square is wide enough for both to be the
  whole-plane integral; and the oracle's Monte Carlo of the Sec. 4.3 setup
  (SQUARE, N = 44, D = 8 m, d = 1.1 m, B = 56.5 m, v = 10.2 m/s) agrees with it
  within the Monte-Carlo error.
* The Sec. 4.2 choice of N in libqrs (host code) equals an independent
  restatement with adaptive quadrature; g_inf equals the piston variance / 2 pi.
"""
import ctypes as C
import math

import numpy as np
import pytest

import oracle
from oracle import analytic as an

VLTI = dict(r0=0.10, L0=22.0, D=8.0, d=1.1, B=56.5, v=10.2, fmax=0.25, N=44)


def test_filtered_synthesis_is_the_aperture_piston():
    rng = np.random.default_rng(1)
    xy = rng.uniform(-60, 60, size=(9, 2)).astype(np.float32)
    for dom in (dict(domain="logpolar", fmin=1e-3, fmax=10.0), dict(domain="square", fmax=0.25)):
        p_plain = oracle.params(seed=5, r0=0.1, L0=22.0, **dom)
        p_filt = dict(p_plain, ap_D=8.0, ap_d=float(np.float32(1.1)))  # the piston code takes FP32 diameters
        n_f = 44 * 44 if dom["domain"] == "square" else 1024
        chi = oracle.synthesize(p_filt, n_f, 3, xy, real_offset=2)
        pis, _ = oracle.diff_piston(p_plain, n_f, 3, xy, np.full(9, 8.0), np.full(9, 1.1), real_offset=2)
        assert np.allclose(chi, pis, rtol=1e-11, atol=1e-11 * np.abs(pis).max())


def test_filtered_parseval_annulus_and_square():
    r0, L0, D, d = VLTI["r0"], VLTI["L0"], VLTI["D"], VLTI["d"]
    p = oracle.params(seed=6, r0=r0, L0=L0, fmin=1e-3, fmax=10.0, ap_D=D, ap_d=d)
    dr = oracle.draw(p, n_f=1024, n_real=200)
    assert np.mean(np.sum(dr["F"] ** 2, axis=1)) == pytest.approx(an.piston_variance(r0, L0, D, d, 1e-3, 10.0),
                                                                rel=5e-3)
    from scipy import integrate
    ps = oracle.params(seed=7, r0=r0, L0=L0, domain="square", fmax=VLTI["fmax"], ap_D=D, ap_d=d)
    ds = oracle.draw(ps, n_f=VLTI["N"] ** 2, n_real=100)
    q, _ = integrate.dblquad(lambda y, x: float(an.psd(math.hypot(x, y), r0, L0) * an.airy(math.hypot(x, y), D, d) ** 2),
                             0, VLTI["fmax"], 0, VLTI["fmax"], epsabs=1e-9, epsrel=1e-9)
    assert np.mean(np.sum(ds["F"] ** 2, axis=1)) == pytest.approx(4 * q, rel=1e-2)


def test_square_quadrature_equals_hankel_form_on_a_wide_square():
    taus = [0.1, 0.3]
    sq = an.square_temporal_piston_sf(taus, 5.0, 10.0, 0.1, 22.0, 8.0, 1.1, 2.0)
    iso = [an.temporal_piston_sf(t, 5.0, 10.0, 0.1, 22.0, 8.0, 1.1, 1e-7, 60.0) for t in taus]
    assert np.allclose(sq, iso, rtol=1e-5)
    # B = 0: the two apertures coincide, the differential piston vanishes
    assert np.allclose(an.square_temporal_piston_sf(taus, 0.0, 10.0, 0.1, 22.0, 8.0, 1.1, 0.25), 0.0, atol=1e-9)


def test_oracle_monte_carlo_of_the_vlti_setup():
    """300 realisations, 64 time samples 10 ms apart at both telescopes; the
    per-realisation SF at lags 1, 4, 16, 48 against the square quadrature."""
    v, B, M, dt = VLTI["v"], VLTI["B"], 64, 0.01
    t = np.arange(M) * dt
    xy = np.concatenate([np.stack([-v * t, 0 * t], -1), np.stack([B - v * t, 0 * t], -1)]).astype(np.float32)
    p = oracle.params(seed=8, r0=VLTI["r0"], L0=VLTI["L0"], domain="square", fmax=VLTI["fmax"], ap_D=VLTI["D"],
                      ap_d=VLTI["d"])
    R = 300
    chi = oracle.synthesize(p, VLTI["N"] ** 2, R, xy)
    delta = chi[:, :M] - chi[:, M:]
    lags = np.array([1, 4, 16, 48])
    per = np.stack([np.mean((delta[:, L:] - delta[:, :-L]) ** 2, axis=1) for L in lags], -1)  # [R][lags]
    mean, sem = per.mean(0), per.std(0, ddof=1) / np.sqrt(R)
    ref = an.square_temporal_piston_sf(lags * dt, B, v, VLTI["r0"], VLTI["L0"], VLTI["D"], VLTI["d"], VLTI["fmax"])
    z = (mean - ref) / sem
    assert np.all(np.abs(z) < 4), z


def _choose_n(psd, df, eps, n_max=10000):
    import paper_2404_02978_gb300 as qrs
    f = qrs.load().qrs_choose_n
    f.argtypes = [C.POINTER(qrs.QrsPsd), C.c_double, C.c_double, C.c_int32, C.POINTER(C.c_int32),
                  C.POINTER(C.c_double)]
    f.restype = C.c_int
    n, g = C.c_int32(), (C.c_double * 3)()
    st = f(C.byref(psd), df, eps, n_max, C.byref(n), g)
    return st, n.value, list(g)


def test_choose_n_matches_independent_restatement():
    import paper_2404_02978_gb300 as qrs
    r0, L0, D, d = VLTI["r0"], VLTI["L0"], VLTI["D"], VLTI["d"]
    df = 0.25 / L0
    for eps in (1e-2, 1e-3, 1e-5):
        st, n, g = _choose_n(qrs.QrsPsd(r0, L0, 0, 0, D, d), df, eps)
        n_ref, g_ref, g_inf = an.choose_n(r0, L0, D, d, df, eps)
        assert st == 0 and n == n_ref, (eps, n, n_ref)
        assert g[0] == pytest.approx(g_ref, rel=1e-8) and g[1] == pytest.approx(g_inf, rel=1e-8)
    # g_inf is the piston variance over the whole plane divided by 2 pi
    assert g[1] == pytest.approx(an.piston_variance(r0, L0, D, d, 1e-9, 1e3) / (2 * math.pi), rel=1e-8)
    # unfiltered von Karman: g saturates too (W ~ f^-11/3)
    st, n, g = _choose_n(qrs.QrsPsd(r0, L0, 0, 0, 0.0, 0.0), df, 1e-3)
    n_ref, _, _ = an.choose_n(r0, L0, 0.0, 0.0, df, 1e-3)
    assert st == 0 and n == n_ref
    # invalid requests
    assert _choose_n(qrs.QrsPsd(r0, L0, 1, 0, D, d), df, 1e-3)[0] == -1  # Kolmogorov: g diverges at 0
    assert _choose_n(qrs.QrsPsd(r0, L0, 0, 0, D, d), df, 1e-12, n_max=20)[0] == -1  # not met below n_max
