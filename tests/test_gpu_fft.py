"""GPU parity of the FFT screen baseline (Eq. 2, Sec. 2.2) against the oracle,
and the static-sampling bias of its structure function (Sec. 2.3).

The spectrum comes from libqrs (qrs_fft_spectrum: Philox stream 4, Box-Muller,
the PSD on the FFT grid); the inverse DFT from cuFFT (torch.fft).  Tolerances:
spectrum samples within 1e-5 of their coefficient scale sqrt(W) df (FP32
Box-Muller and PSD against FP64; with an aperture filter, of the unfiltered
scale); screens within 1e-5 of the screen's standard
deviation sigma (sigma^2 = sum_f W df^2) per value."""
import numpy as np
import pytest
import torch

import oracle
import paper_2404_02978_gb300 as qrs
from oracle import analytic as an

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_2404_02978_gb300 import build as B
    B.build()
    return qrs.Handle(0)


def _grid_W(p, n, dx):
    df = 1.0 / (n * dx)
    k = np.where(np.arange(n) < (n + 1) // 2, np.arange(n), np.arange(n) - n) * df
    FX, FY = np.meshgrid(k, k, indexing="xy")
    fr = np.hypot(FX, FY)
    W = np.zeros_like(fr)
    m = fr > 0
    W[m] = an.psd(fr[m], p["r0"], p["L0"], p["psd"])
    if p.get("ap_D", 0.0):
        W[m] *= an.airy(fr[m], p["ap_D"], p.get("ap_d", 0.0)) ** 2
    return FX, FY, W, df


CASES = [
    dict(n=64, dx=0.1, p=dict()),
    dict(n=63, dx=0.125, p=dict(r0=0.1, L0=20.0)),                   # odd n
    dict(n=48, dx=0.5, p=dict(r0=0.1, L0=25.0, ap_D=2.0, ap_d=0.3)),  # piston field (Eq. 7 filter)
    dict(n=40, dx=0.2, p=dict(psd="kolmogorov", r0=0.2)),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "n%d" % c["n"])
def test_fft_spectrum_and_screens_against_the_oracle(h, case):
    n, dx = case["n"], case["dx"]
    p = oracle.params(seed=31, **case["p"])
    R, off = 3, 2
    spec = qrs.qrs_fft_spectrum(h, p, n, dx, R, real_offset=off)
    screens = qrs.fft_screens(h, p, n, dx, R, real_offset=off)
    qrs.qrs_sync(h)
    ref_spec = oracle.fft_spectrum(p, n, dx, R, off)
    ref_re, ref_im = oracle.fft_screen(p, n, dx, R, off)
    _, _, W, df = _grid_W(p, n, dx)
    F = np.sqrt(W) * df
    # spectrum samples in units of their unfiltered coefficient scale sqrt(W) df
    # (near a zero of the Eq. 7 filter the filtered scale vanishes)
    _, _, W0, _ = _grid_W(dict(p, ap_D=0.0, ap_d=0.0), n, dx)
    F0 = np.sqrt(W0) * df
    got = spec.cpu().numpy().astype(np.complex128)
    assert got[:, 0, 0].tolist() == [0j] * R
    m = F0 > 0
    assert np.max(np.abs(got - ref_spec)[:, m] / F0[m]) <= 1e-5
    sig = np.sqrt(np.sum(F ** 2))
    s = screens.cpu().numpy().astype(np.float64)
    assert np.isfinite(s).all()
    err = max(np.abs(s[0] - ref_re).max(), np.abs(s[1] - ref_im).max()) / sig
    print("FFT screen n=%d: max err %.3g sigma" % (n, err))
    assert err <= 1e-5


def test_fft_full_size_sampled(h):
    """The benchmark's screens: 256 x 256 at 8 m / 256 pitch, 1000 realisations in
    one spectrum call; realisations 0, 517 and 999 against the oracle."""
    n, dx, R = 256, 8.0 / 256, 1000
    p = oracle.params(seed=2, r0=0.15, L0=30.0)
    screens = qrs.fft_screens(h, p, n, dx, R)
    qrs.qrs_sync(h)
    _, _, W, df = _grid_W(p, n, dx)
    sig = np.sqrt(np.sum(W) * df * df)
    for r in (0, 517, R - 1):
        ref_re, ref_im = oracle.fft_screen(p, n, dx, 1, r)
        got = screens[:, r].cpu().numpy().astype(np.float64)
        err = max(np.abs(got[0] - ref_re[0]).max(), np.abs(got[1] - ref_im[0]).max()) / sig
        assert err <= 1e-5, (r, err)


def test_fft_static_sampling_bias(h):
    """The structure function along x of 2 x 300 FFT screens (von Karman, L0 = 30 m,
    8 m grid: df = 0.125 c/m) equals its static-sampling expectation
    2 sum_f W df^2 (1 - cos 2 pi fx r) within 3 sigma, and at r = 4 m falls short
    of the continuous spectrum's Hankel integral by more than 10 sigma: the bias of
    Sec. 2.3 that randomised (quasi-random) sampling removes."""
    n, dx, R = 256, 8.0 / 256, 300
    p = oracle.params(seed=12, r0=0.15, L0=30.0)
    screens = qrs.fft_screens(h, p, n, dx, R)  # [2, R, n, n]
    lags = np.array([4, 32, 128], np.int32)
    delta = screens.reshape(2 * R, n, n).permute(1, 0, 2).contiguous()  # [row][realisation][column]
    acc = qrs.qrs_structure_fn(h, delta, torch.from_numpy(lags).cuda())
    qrs.qrs_sync(h)
    a = acc.cpu().numpy()                      # [2R][lags][3]
    per = a[:, :, 0] / a[:, :, 2]               # per realisation: mean over rows and positions
    mean, sem = per.mean(0), per.std(0, ddof=1) / np.sqrt(per.shape[0])
    FX, FY, W, df = _grid_W(p, n, dx)
    for li, L in enumerate(lags):
        r = L * dx
        static = 2.0 * np.sum(W * df * df * (1.0 - np.cos(2 * np.pi * FX * r)))
        z = (mean[li] - static) / sem[li]
        print("FFT SF at %.2f m: %.4g (static %.4g, continuum %.4g), z %.2f"
              % (r, mean[li], static, an.phase_sf_vk_infinite(r, 0.15, 30.0), z))
        assert abs(z) < 3.0
    cont = an.phase_sf_vk_infinite(lags[-1] * dx, 0.15, 30.0)
    assert (cont - mean[-1]) / sem[-1] > 10.0
