"""Pins of the oracle's FFT screen (Eq. 2, the comparison method of Sec. 2.2).

The screen is n^2 times the inverse DFT of the spectrum S(f) = (a + i b)
sqrt(W(f)) df on the FFT frequency grid, i.e. sum_f S(f) e^{2 pi i f.x}; its
real part is Eq. 3's sum F (a cos 2 pi f.x - b sin 2 pi f.x) over the grid
frequencies with F = sqrt(W) df.  Pinned against:
* the oracle's own Eq. 3 sum (oracle_synth_terms, separate C code) at the
  grid points, for the real and the imaginary part, odd and even n;
* the DFT's Parseval identity, mean over the grid of |chi|^2 = sum |S|^2,
  which fixes the normalisation exactly;
* S / (sqrt(W) df) standard normal in both parts, S(0) = 0;
* the ensemble structure function of the static sampling,
  E (chi(x + r) - chi(x))^2 = 2 sum_f W df^2 (1 - cos 2 pi f.r), by Monte Carlo
  within 3 sigma (the static-sampling bias of Sec. 2.3 is exactly this sum).
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import analytic as an


def _grid_freqs(n, dx):
    df = 1.0 / (n * dx)
    k = np.where(np.arange(n) < (n + 1) // 2, np.arange(n), np.arange(n) - n) * df
    FX, FY = np.meshgrid(k, k, indexing="xy")  # [i][j]: fy from the row, fx from the column
    return FX, FY, df


@pytest.mark.parametrize("n,dx", [(8, 0.5), (16, 0.125), (7, 0.25), (9, 0.3)])
def test_fft_screen_equals_direct_eq3_sum(n, dx):
    """Where the grid frequencies and points are exact in FP32 (dyadic pitches),
    against the oracle's Eq. 3 sum in C; elsewhere (odd n) against the
    definition sum_f S e^{2 pi i f.x} written out in FP64."""
    p = oracle.params(seed=5, r0=0.12, L0=20.0)
    S = oracle.fft_spectrum(p, n, dx, 2, real_offset=3)
    re, im = oracle.fft_screen(p, n, dx, 2, real_offset=3)
    FX, FY, df = _grid_freqs(n, dx)
    f = np.stack([FX.ravel(), FY.ravel()], -1)
    X, Y = np.meshgrid(np.arange(n) * dx, np.arange(n) * dx, indexing="xy")
    xy = np.stack([X.ravel(), Y.ravel()], -1)
    exact32 = np.array_equal(f.astype(np.float32).astype(np.float64), f) and \
        np.array_equal(xy.astype(np.float32).astype(np.float64), xy)
    for r in range(2):
        s = S[r].ravel()
        if exact32:
            direct_re = oracle.synth_terms(f, np.ones(s.size), np.stack([s.real, s.imag], -1), xy)
            direct_im = oracle.synth_terms(f, np.ones(s.size), np.stack([s.imag, -s.real], -1), xy)
        else:
            z = np.exp(2j * np.pi * (xy @ f.T)) @ s
            direct_re, direct_im = z.real, z.imag
        scale = np.sqrt(np.sum(np.abs(s) ** 2))
        assert np.max(np.abs(re[r].ravel() - direct_re)) <= 1e-12 * scale
        assert np.max(np.abs(im[r].ravel() - direct_im)) <= 1e-12 * scale


def test_fft_screen_parseval():
    p = oracle.params(seed=6)
    n = 32
    S = oracle.fft_spectrum(p, n, 0.05, 3)
    re, im = oracle.fft_screen(p, n, 0.05, 3)
    lhs = np.mean(re ** 2 + im ** 2, axis=(1, 2))
    rhs = np.sum(np.abs(S) ** 2, axis=(1, 2))
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=0)


def test_fft_spectrum_is_the_psd_times_normal_coefficients():
    p = oracle.params(seed=7, r0=0.1, L0=25.0)
    n, dx = 64, 0.1
    S = oracle.fft_spectrum(p, n, dx, 4)
    FX, FY, df = _grid_freqs(n, dx)
    F = np.sqrt(an.psd(np.hypot(FX, FY), 0.1, 25.0)) * df
    assert np.all(S[:, 0, 0] == 0)
    m = np.ones((n, n), bool)
    m[0, 0] = False
    c = S[:, m] / F[m]
    assert stats.kstest(c.real.ravel(), "norm").pvalue > 1e-3
    assert stats.kstest(c.imag.ravel(), "norm").pvalue > 1e-3
    assert abs(np.corrcoef(c.real.ravel(), c.imag.ravel())[0, 1]) < 0.02


def test_fft_spectrum_piston_filter():
    """With an aperture filter the spectrum carries the Eq. 7 factor A(|f|)."""
    n, dx = 16, 0.5
    p0 = oracle.params(seed=8, r0=0.1, L0=25.0)
    p1 = dict(p0, ap_D=2.0, ap_d=0.3)
    S0, S1 = oracle.fft_spectrum(p0, n, dx, 1), oracle.fft_spectrum(p1, n, dx, 1)
    FX, FY, _ = _grid_freqs(n, dx)
    A = an.airy(np.hypot(FX, FY).ravel(), 2.0, 0.3).reshape(n, n)
    assert np.allclose(S1[0], S0[0] * A, rtol=1e-12, atol=0)


def test_fft_static_sampling_structure_function_monte_carlo():
    """E (chi(x + r) - chi(x))^2 at lags along x equals 2 sum_f W df^2 (1 - cos 2 pi fx r)
    for both parts, within 3 sigma of the Monte Carlo."""
    p = oracle.params(seed=9, r0=0.15, L0=30.0)
    n, dx, R = 32, 0.25, 600
    re, im = oracle.fft_screen(p, n, dx, R)
    FX, FY, df = _grid_freqs(n, dx)
    W = an.psd(np.hypot(FX, FY), 0.15, 30.0)
    W[0, 0] = 0.0
    for lag in (1, 3, 8, 16):
        expect = 2.0 * np.sum(W * df * df * (1.0 - np.cos(2 * np.pi * FX * lag * dx)))
        for part in (re, im):
            d2 = (np.roll(part, -lag, axis=2) - part) ** 2  # periodic screen: every column pair
            per_real = d2.mean(axis=(1, 2))                # one value per realisation (independent)
            z = (per_real.mean() - expect) / (per_real.std(ddof=1) / np.sqrt(R))
            assert abs(z) < 3.0, (lag, z)
