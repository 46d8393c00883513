"""Pins of the FP64 oracle against things other than itself.

Each test ties one oracle function to a value fixed by the paper, by
mathematics or by an independent library routine, chosen so that a plausible
slip (a dropped factor, a wrong sign or index, a transposed operand) fails:

* Philox4x32-10: published known-answer vectors (tests/golden).
* Eq. 6 (R2): constants re-derived from a 50-digit plastic number; the
  fixed-point stream against the paper's recurrence run in 60-digit arithmetic.
* Eq. 5 / Sec. 3.2 square-to-disc / log-polar: numerical Jacobians of the maps
  against the J the weights use; the map ranges.
* Eq. 7: the PSD constant against its Gamma-function closed form; the filter
  against scipy's Bessel J1 and against a brute-force aperture average.
* Eq. 3: the sum against numpy's inverse FFT on an FFT grid; coefficient
  distributions (Gaussian vs the literal Eq. 3 form) by their moments.
* Parseval: E sum_k w_k against the closed-form integral of the PSD.
* Sec. 4.4: the conditional differential-piston structure function averaged
  over the continuing stream against the analytic Hankel integral; the Monte
  Carlo mean within 3 sigma.
* Structure-function accumulation against a numpy computation and a ramp.
"""
import math
import os

import mpmath as mp
import numpy as np
import pytest
from scipy import stats

import oracle
from cdf_inputs import two_level_cdf
from oracle import analytic as an

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- Philox
def test_philox_known_answers():
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        assert oracle.philox(v[:4], v[4:6]) == v[6:10]
        n += 1
    assert n == 3


def test_philox_words_uniform():
    d = oracle.draw(oracle.params(seed=7), n_f=4096, n_real=4, debug=True)
    w = d["words"].reshape(-1).astype(np.float64) / 2**32
    # chi-square over 64 bins
    h, _ = np.histogram(w, bins=64, range=(0, 1))
    assert stats.chisquare(h).pvalue > 1e-4
    # distinct counters give distinct words
    assert len(np.unique(d["words"][..., 0])) > 0.999 * d["words"][..., 0].size


# --------------------------------------------------------------------- R2
def _psi():
    mp.mp.dps = 60
    return mp.findroot(lambda x: x ** 3 - x - 1, mp.mpf("1.3"))


def test_r2_constants_from_plastic_number():
    psi = _psi()
    assert abs(psi ** 3 - psi - 1) < mp.mpf(10) ** -55
    a1 = int(mp.nint(mp.mpf(2) ** 64 / psi))
    a2 = int(mp.nint(mp.mpf(2) ** 64 / psi ** 2))
    # point 1 from a zero seed is exactly the increment
    assert oracle.r2_point((0, 0), 1) == (a1, a2)
    # psi printed in the paper (Sec. 3.2): 1.324717957244746...
    assert abs(float(psi) - 1.324717957244746) < 1e-15


def test_r2_stream_matches_recurrence():
    """Eq. 6 run literally (s <- {s + 1/psi}) in 60-digit arithmetic from s0=(0.5,0.5)."""
    psi = _psi()
    s0 = (1 << 63, 1 << 63)
    sx, sy = mp.mpf("0.5"), mp.mpf("0.5")
    for n in range(0, 2000):
        if n in (0, 1, 2, 3, 10, 999, 1999):
            Sx, Sy = oracle.r2_point(s0, n)
            # n additions of a rounded increment: |error| <= n/2 units of 2^-64
            assert abs(mp.mpf(Sx) / 2**64 - sx) <= (n + 1) * mp.mpf(2) ** -65
            assert abs(mp.mpf(Sy) / 2**64 - sy) <= (n + 1) * mp.mpf(2) ** -65
        sx = mp.frac(sx + 1 / psi)
        sy = mp.frac(sy + 1 / psi ** 2)


def test_r2_seed_fixed_and_random():
    assert oracle.r2_seed(0, s0=(1 << 63, 1 << 63)) == (1 << 63, 1 << 63)
    a, b = oracle.r2_seed(5), oracle.r2_seed(6)
    assert a != b
    # the random seed is Philox word pairs of counter (0,0,1,0)
    w = oracle.philox([0, 0, 1, 0], [5, 0])
    assert a == ((w[1] << 32) | w[0], (w[3] << 32) | w[2])


def test_r2_draw_continues_across_realisations():
    """Sec. 3.2: the stream is never re-initialised: realisation r, term k is point (r N_f + k)."""
    p = oracle.params(domain="square", fmax=1.0, seed=3)
    one = oracle.draw(p, n_f=64, n_real=3, debug=True)
    chunk = oracle.draw(p, n_f=64, n_real=2, real_offset=1, debug=True)
    assert np.array_equal(one["r2"][1:], chunk["r2"])
    assert np.array_equal(one["f"][1:], chunk["f"])
    s0 = oracle.r2_seed(3)
    assert tuple(int(v) for v in one["r2"][2, 5]) == oracle.r2_point(s0, 2 * 64 + 5)


# ----------------------------------------------------------------- domains
def test_square_map_eq5():
    # Eq. 5: f = delta_f N (s - 1/2), delta_f N = 2 max f
    assert oracle.domain_map("square", 0, 2.0, 0.0, 0.5) == (-2.0, 0.0)
    assert oracle.domain_map("square", 0, 2.0, 0.75, 0.25) == (1.0, -1.0)
    assert oracle.domain_jacobian("square", 0, 2.0, 0.3, 0.1) == 16.0


def _num_jac(kind, fmin, fmax, sx, sy, h=1e-6):
    fxp = np.array(oracle.domain_map(kind, fmin, fmax, sx + h, sy))
    fxm = np.array(oracle.domain_map(kind, fmin, fmax, sx - h, sy))
    fyp = np.array(oracle.domain_map(kind, fmin, fmax, sx, sy + h))
    fym = np.array(oracle.domain_map(kind, fmin, fmax, sx, sy - h))
    dx, dy = (fxp - fxm) / (2 * h), (fyp - fym) / (2 * h)
    return abs(dx[0] * dy[1] - dx[1] * dy[0])


@pytest.mark.parametrize("kind,fmin,fmax", [("disc", 0.0, 3.0), ("logpolar", 1e-3, 16.0)])
def test_map_jacobians(kind, fmin, fmax):
    rng = np.random.default_rng(1)
    for sx, sy in rng.uniform(0.02, 0.98, size=(40, 2)):
        if kind == "disc" and abs(abs(2 * sx - 1) - abs(2 * sy - 1)) < 1e-3:
            continue  # the concentric map has a kink on the diagonals
        fx, fy = oracle.domain_map(kind, fmin, fmax, sx, sy)
        J = oracle.domain_jacobian(kind, fmin, fmax, fx, fy)
        assert _num_jac(kind, fmin, fmax, sx, sy) == pytest.approx(J, rel=2e-6)


def test_disc_map_range_and_edges():
    f = oracle.domain_map("disc", 0, 2.0, 1.0, 0.5)
    assert f == pytest.approx((2.0, 0.0))
    f = oracle.domain_map("disc", 0, 2.0, 0.5, 1.0)
    assert f == pytest.approx((0.0, 2.0), abs=1e-15)
    rng = np.random.default_rng(2)
    r = [math.hypot(*oracle.domain_map("disc", 0, 2.0, a, b)) for a, b in rng.uniform(size=(500, 2))]
    assert max(r) <= 2.0 + 1e-12
    # area preserving: radius^2 uniform on [0, fmax^2]
    assert stats.kstest(np.array(r) ** 2 / 4.0, "uniform").pvalue > 1e-3


def test_logpolar_mean_jacobian_is_annulus_area():
    fmin, fmax = 1e-3, 16.0
    s = (np.arange(2000) + 0.5) / 2000
    J = [oracle.domain_jacobian("logpolar", fmin, fmax, *oracle.domain_map("logpolar", fmin, fmax, x, 0.3))
         for x in s]
    # integral over s of J = pi (fmax^2 - fmin^2); midpoint rule on 2000 nodes
    assert np.mean(J) == pytest.approx(np.pi * (fmax ** 2 - fmin ** 2), rel=2e-5)


# ---------------------------------------------------------------- PSD, Eq. 7
def test_psd_constant_and_slope():
    c = an.vk_coeff()
    assert oracle.psd("kolmogorov", 1.0, 1.0, 1.0) == pytest.approx(c, rel=1e-15)
    # paper's truncated constant 0.02289 (Eq. 7)
    assert abs(c - 0.02289) < 1e-5
    # Kolmogorov f^(-11/3) law, r0^(-5/3) law
    assert oracle.psd("kolmogorov", 0.1, 1, 4.0) / oracle.psd("kolmogorov", 0.1, 1, 1.0) == pytest.approx(2 ** (-11 / 3))
    assert oracle.psd("von_karman", 0.2, 25, 0.3) / oracle.psd("von_karman", 0.1, 25, 0.3) == pytest.approx(2 ** (-5 / 3))
    # von Karman: finite at f = 0, c r0^-5/3 L0^(11/3)
    assert oracle.psd("von_karman", 0.1, 25, 0.0) == pytest.approx(c * 0.1 ** (-5 / 3) * 25 ** (11 / 3))


@pytest.mark.parametrize("D,d", [(1.0, 0.0), (8.0, 1.1), (1.8, 0.0)])
def test_airy_filter_vs_scipy(D, d):
    f = np.concatenate([[0.0, 1e-9, 1e-6, 1e-5, 1e-4], np.geomspace(1e-3, 20, 300)])
    ref = an.airy(f, D, d)
    got = np.array([oracle.airy(x, D, d) for x in f])
    assert np.max(np.abs(got - ref)) < 1e-12


@pytest.mark.parametrize("D,d", [(1.0, 0.0), (8.0, 1.1)])
def test_airy_filter_is_aperture_average(D, d):
    """Eq. 7 filter = average of cos(2 pi f.x) over the (annular) pupil, brute force."""
    nr, nt = 400, 256
    # midpoint rule in r^2 (area-uniform) and theta
    u = (np.arange(nr) + 0.5) / nr
    r = np.sqrt((d / 2) ** 2 + u * ((D / 2) ** 2 - (d / 2) ** 2))
    th = (np.arange(nt) + 0.5) / nt * 2 * np.pi
    X = r[:, None] * np.cos(th)[None, :]
    for f in [0.05, 0.2, 0.5, 1.3]:
        avg = np.mean(np.cos(2 * np.pi * f * X))
        assert oracle.airy(f, D, d) == pytest.approx(avg, abs=2e-5)


# -------------------------------------------------------------- coefficients
def test_gauss_coefficients_are_standard_normal():
    d = oracle.draw(oracle.params(seed=11, coef="gauss"), n_f=8192, n_real=6)
    a, b = d["coef"][..., 0].ravel(), d["coef"][..., 1].ravel()
    for x in (a, b):
        assert stats.kstest(x, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.02
    assert np.mean(a ** 4) == pytest.approx(3.0, abs=0.12)


def test_eq3_coefficients_second_moments():
    """Literal Eq. 3: sqrt2 R_n cos(2 pi R_u): E a^2 = 1, but kurtosis 4.5 (not Gaussian)."""
    d = oracle.draw(oracle.params(seed=12, coef="eq3"), n_f=8192, n_real=6)
    a, b = d["coef"][..., 0].ravel(), d["coef"][..., 1].ravel()
    assert np.mean(a ** 2) == pytest.approx(1.0, abs=0.03)
    assert np.mean(b ** 2) == pytest.approx(1.0, abs=0.03)
    assert np.mean(a ** 4) == pytest.approx(4.5, abs=0.25)
    assert abs(np.mean(a * b)) < 0.03


def test_box_muller_from_words():
    d = oracle.draw(oracle.params(seed=13), n_f=256, n_real=1, debug=True)
    w = d["words"][0]
    U1 = ((w[:, 2] >> 8).astype(np.float64) + 1) * 2.0 ** -24
    rad2 = d["coef"][0, :, 0] ** 2 + d["coef"][0, :, 1] ** 2
    assert np.allclose(rad2, -2 * np.log(U1), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("coef", ["gauss", "eq3"])
def test_terms_in_amplitude_phase_form(coef):
    """The one-cosine form of Eq. 3 that the fused and piston kernels evaluate:
    with (a, b) of a term, a cos t - b sin t = amp cos(t + 2 pi u 2^-24), where
    for GAUSS amp = sqrt(-2 ln U1) and u is the 24-bit integer of U2, and for the
    literal Eq. 3 amp = sqrt2 R_n and u is that of R_u; the half turn in u's top
    bit then moves into the sign of amp (cos(x + pi) = -cos x).  Checked against
    the oracle's own coefficients at random angles t: a slip in which uniform is
    the angle, in its sign, or in the moved half turn fails."""
    seed = 14
    n_f, R = 512, 2
    d = oracle.draw(oracle.params(seed=seed, coef=coef), n_f=n_f, n_real=R, debug=True)
    w = d["words"].reshape(-1, 4).astype(np.uint64)
    ab = d["coef"].reshape(-1, 2)
    rad = np.sqrt(-2 * np.log(((w[:, 2] >> np.uint64(8)) + np.uint64(1)).astype(np.float64) * 2.0 ** -24))
    if coef == "gauss":
        amp = rad
        u = (w[:, 3] >> np.uint64(8)).astype(np.int64)
    else:
        U2 = (w[:, 3] >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
        amp = math.sqrt(2) * rad * np.cos(2 * np.pi * U2)
        u = np.array([oracle.philox([n, n >> 32, 2, 0], [seed, seed >> 32])[0] >> 8 for n in range(R * n_f)],
                     np.int64)
    amp = np.where(u >> 23, -amp, amp)
    u = u & 0x7FFFFF
    t = np.random.default_rng(5).uniform(0, 2 * np.pi, size=amp.shape)
    lhs = ab[:, 0] * np.cos(t) - ab[:, 1] * np.sin(t)
    rhs = amp * np.cos(t + 2 * np.pi * u * 2.0 ** -24)
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-12 * np.abs(amp).max())
    assert np.all(u < 2 ** 23) and np.mean(amp < 0) == pytest.approx(0.5, abs=0.05)


# --------------------------------------------------------------- weights, Parseval
def test_parseval_logpolar_config2():
    """E sum_k w_k = integral of W over the annulus (589.919 rad^2 for r0=0.15, L0=30, [1e-3,16])."""
    p = oracle.params(r0=0.15, L0=30.0, fmin=1e-3, fmax=16.0, seed=2)
    d = oracle.draw(p, n_f=4096, n_real=8)
    E = an.parseval_annulus(0.15, 30.0, 1e-3, 16.0)
    assert E == pytest.approx(589.9192, rel=1e-6)
    per = np.sum(d["F"] ** 2, axis=1)
    assert np.mean(per) == pytest.approx(E, rel=2e-3)
    assert np.all(np.abs(per / E - 1) < 2e-2)  # every realisation covers the whole spectrum


def test_parseval_square_eq5():
    """SQUARE: w = W delta_f^2 with N_f = N^2 (Eq. 3, 5); sum -> integral over the square."""
    from scipy import integrate
    fmax, r0, L0 = 0.25, 0.1, 22.0
    p = oracle.params(domain="square", fmax=fmax, r0=r0, L0=L0, seed=4)
    N = 44  # Sec. 4.3: delta_f = 0.25/22, f_max = 0.25 -> N = 44
    d = oracle.draw(p, n_f=N * N, n_real=40)
    dfc = 2 * fmax / N
    fx, fy = d["f"][..., 0].astype(float), d["f"][..., 1].astype(float)
    W = an.psd(np.hypot(fx, fy), r0, L0)
    assert np.allclose(d["F"] ** 2, W * dfc ** 2, rtol=1e-12)
    # 4 x quarter-square integral: peaked at the origin on the scale 1/L0
    q, _ = integrate.dblquad(lambda y, x: float(an.psd(math.hypot(x, y), r0, L0)), 0, fmax, 0, fmax,
                             epsabs=1e-10, epsrel=1e-10)
    assert np.mean(np.sum(d["F"] ** 2, axis=1)) == pytest.approx(4 * q, rel=1e-2)


def test_importance_uniform_cdf_is_unbiased():
    nr, nt = 16, 8
    nc = nr * nt
    rng = np.random.default_rng(5)
    p_c = 0.5 * rng.dirichlet(np.ones(nc)) + 0.5 / nc
    cdf, p_q = two_level_cdf(p_c, nr, nt)
    p = oracle.params(sampler="importance", n_rho=nr, n_theta=nt, cdf=cdf, r0=0.15, L0=30.0,
                      fmin=1e-3, fmax=16.0, seed=9)
    d = oracle.draw(p, n_f=1024, n_real=30)
    E = an.parseval_annulus(0.15, 30.0, 1e-3, 16.0)
    per = np.sum(d["F"] ** 2, axis=1)
    assert np.mean(per) == pytest.approx(E, rel=3e-2)
    # cells: frequencies lie inside their cell
    L = math.log(16.0 / 1e-3)
    rho = np.hypot(d["f"][..., 0], d["f"][..., 1]).astype(float)
    ir = d["cell"] // nt
    lo = 1e-3 * np.exp(L * ir / nr) * (1 - 1e-6)
    hi = 1e-3 * np.exp(L * (ir + 1) / nr) * (1 + 1e-6)
    assert np.all((rho >= lo) & (rho <= hi))
    # cell frequencies follow p_c
    cnt = np.bincount(d["cell"].ravel(), minlength=nc)
    assert stats.chisquare(cnt, p_q * cnt.sum()).pvalue > 1e-4


def test_jitter_one_point_per_cell():
    """Eq. 4: one jittered frequency per grid cell in every realisation."""
    p = oracle.params(sampler="jitter", domain="square", fmax=1.0, n_rho=16, n_theta=8, seed=21)
    d = oracle.draw(p, n_f=128, n_real=3)
    for r in range(3):
        assert sorted(d["cell"][r].tolist()) == list(range(128))


# ------------------------------------------------------------------ Eq. 3 sum
def test_synthesis_equals_inverse_fft_on_grid():
    """On an FFT grid the Eq. 3 sum is the real part of an inverse 2-D DFT."""
    n, L = 16, 4.0
    rng = np.random.default_rng(3)
    kx, ky = np.meshgrid(np.arange(-n // 2, n // 2), np.arange(-n // 2, n // 2), indexing="ij")
    f = np.stack([kx / L, ky / L], -1).reshape(-1, 2).astype(np.float32)
    F = rng.uniform(0.5, 2.0, size=n * n)
    coef = rng.normal(size=(n * n, 2))
    px, py = np.meshgrid(np.arange(n) * L / n, np.arange(n) * L / n, indexing="ij")
    xy = np.stack([px, py], -1).reshape(-1, 2).astype(np.float32)
    got = oracle.synth_terms(f, F, coef, xy).reshape(n, n)
    spec = np.zeros((n, n), complex)
    c = (F * (coef[:, 0] + 1j * coef[:, 1])).reshape(n, n)
    spec[kx % n, ky % n] = c
    ref = np.real(np.fft.ifft2(spec) * n * n)
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


def test_synthesis_at_origin_and_parseval_variance():
    p = oracle.params(r0=0.15, L0=30.0, fmin=1e-3, fmax=16.0, seed=8)
    d = oracle.draw(p, n_f=64, n_real=1)
    v0 = oracle.synth_terms(d["f"][0], d["F"][0], d["coef"][0], np.zeros((1, 2)))[0]
    assert v0 == pytest.approx(np.sum(d["F"][0] * d["coef"][0, :, 0]), rel=1e-13)
    out = oracle.synthesize(p, n_f=128, n_real=3000, xy=np.array([[0.7, -1.9]], np.float32))
    E = an.parseval_annulus(0.15, 30.0, 1e-3, 16.0)
    var = np.mean(out[:, 0] ** 2)
    assert abs(var / E - 1) < 3 * math.sqrt(2 / 3000) + 0.02


def test_shared_form_column0_and_col_psd():
    p = oracle.params(r0=0.15, L0=30.0, seed=31)
    xy = np.random.default_rng(0).uniform(-4, 4, size=(50, 2)).astype(np.float32)
    sh = oracle.synthesize_shared(p, n_f=64, n_real=3, xy=xy, real_offset=5)
    pe = oracle.synthesize(p, n_f=64, n_real=1, xy=xy, real_offset=5)
    assert np.array_equal(sh[0], pe[0])
    # weights scale as r0^(-5/6) at fixed L0
    sc = oracle.synthesize_shared(p, n_f=64, n_real=1, xy=xy, real_offset=5, col_psd=[(0.3, 30.0)])
    assert np.allclose(sc[0], pe[0] * 2.0 ** (-5 / 6), rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------- pistons
CFG1 = dict(r0=0.10, L0=25.0, fmin=1e-3, fmax=10.0)


def _cfg1_apertures():
    B = 10.0 ** (2 * np.arange(16) / 15)
    xy = np.concatenate([[[0.0, 0.0]], np.stack([B, np.zeros(16)], -1)]).astype(np.float32)
    pairs = np.array([(0, j) for j in range(1, 17)], np.int32)
    return B, xy, pairs


def test_conditional_piston_sf_matches_hankel_integral():
    """Average over the continuing R2 stream of the exact coefficient-average SF
    of each draw equals D(B) = 4 pi int f W A^2 (1 - J0(2 pi f B)) df."""
    B, xy, pairs = _cfg1_apertures()
    p = oracle.params(seed=0, **CFG1)
    d = oracle.draw(p, n_f=1024, n_real=300)
    f = d["f"].astype(np.float64)
    A = an.airy(np.hypot(f[..., 0], f[..., 1]).ravel(), 1.0).reshape(f.shape[:2])
    for b in (0, 5, 10, 15):
        Dd = an.conditional_piston_sf(f, d["F"], A, A, (B[b], 0.0))
        Dref = an.piston_sf(float(np.float32(B[b])), 0.10, 25.0, 1.0, 0.0, 1e-3, 10.0)
        assert np.mean(Dd) == pytest.approx(Dref, rel=3e-3)


@pytest.mark.slow
def test_piston_monte_carlo_within_3_sigma():
    """Config of the plain differential-piston case, 2000 realisations: mean
    Delta^2 within 3 sigma_MC of the analytic structure function."""
    B, xy, pairs = _cfg1_apertures()
    p = oracle.params(seed=0, **CFG1)
    pis, delta = oracle.diff_piston(p, n_f=1024, n_real=2000, ap_xy=xy, ap_D=np.ones(17), pairs=pairs)
    assert np.allclose(delta, pis[:, pairs[:, 0]] - pis[:, pairs[:, 1]], rtol=0, atol=1e-12)
    z = []
    for b in range(16):
        x2 = delta[:, b] ** 2
        Dref = an.piston_sf(float(np.float32(B[b])), 0.10, 25.0, 1.0, 0.0, 1e-3, 10.0)
        z.append((np.mean(x2) - Dref) / (np.std(x2) / np.sqrt(len(x2))))
    assert np.all(np.abs(z) < 3.5), z


def test_piston_with_tiny_aperture_is_point_value():
    p = oracle.params(seed=3, **CFG1)
    xy = np.array([[1.5, -2.0], [30.0, 4.0]], np.float32)
    pis, _ = oracle.diff_piston(p, n_f=256, n_real=2, ap_xy=xy, ap_D=np.full(2, 1e-7), pairs=[(0, 1)])
    pt = oracle.synthesize(p, n_f=256, n_real=2, xy=xy)
    assert np.allclose(pis, pt, rtol=1e-9, atol=1e-9)


# ------------------------------------------------------------- structure fn
def test_structure_fn_vs_numpy_and_ramp():
    rng = np.random.default_rng(4)
    x = rng.normal(size=(5, 3, 40)).astype(np.float32)
    lags = np.array([0, 1, 2, 7, 39], np.int32)
    acc = oracle.structure_fn(x, lags)
    xd = x.astype(np.float64)
    for li, L in enumerate(lags):
        dv = xd if L == 0 else xd[:, :, L:] - xd[:, :, :-L]
        assert np.allclose(acc[:, li, 0], np.sum(dv ** 2, axis=(0, 2)), rtol=1e-13)
        assert np.allclose(acc[:, li, 1], np.sum(dv ** 4, axis=(0, 2)), rtol=1e-13)
        assert np.all(acc[:, li, 2] == dv.shape[0] * dv.shape[2])
    ramp = np.tile(np.arange(10, dtype=np.float32), (2, 1, 1))
    a = oracle.structure_fn(ramp, np.array([3], np.int32))
    assert a[0, 0, 0] == 2 * 7 * 9.0 and a[0, 0, 2] == 14
