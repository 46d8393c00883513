"""Closed forms and quadratures that pin the oracle (test infrastructure only).

Everything here is an independent route to a number the method must reproduce
in expectation; none of it calls the C oracle or the CUDA library.  Special
functions come from scipy (Cephes), not from the C library the oracle links.

* von Karman constant (Eq. 7 first factor): c = Gamma(11/6)^2/(2 pi^(11/3)) *
  (24/5 Gamma(6/5))^(5/6).
* Parseval (Eq. 3): each term has variance F^2 = W J / N_f, so
  E sum_k w_k = integral of W over the sampled domain.  Over an annulus
  [f_min, f_max] the integral is closed form:
  (6 pi / 5) c r0^(-5/3) [(f_min^2 + L0^-2)^(-5/6) - (f_max^2 + L0^-2)^(-5/6)].
* Differential-piston structure function over a baseline B (Sec. 4.4,
  Wiener-Khinchin of Sec. 2.1 with the piston PSD of Eq. 7):
  D(B) = 2 int W A^2 (1 - cos 2 pi f.B) d^2f = 4 pi int f W A^2 (1 - J0(2 pi f B)) df.
* Phase structure function: the same with A = 1; its infinite-domain value is
  the textbook von Karman closed form with K_{5/6}, which pins the quadrature.
* Frozen-flow temporal structure function of the differential piston (Sec. 4.1
  Taylor hypothesis, Sec. 4.4): with Delta(t) = phi(p1 + v t) - phi(p2 + v t),
  <(Delta(t+tau) - Delta(t))^2> = 2 int W A^2 |e^{i2pi f.B} - 1|^2 |e^{i2pi f.v tau} - 1|^2 / 2 d^2f
  expanded into J0 terms (angular integrals of cosines).
"""
from __future__ import annotations

import numpy as np
from scipy import special as sp

PI = np.pi


def vk_coeff() -> float:
    return float(sp.gamma(11 / 6) ** 2 / (2 * PI ** (11 / 3)) * (24 / 5 * sp.gamma(6 / 5)) ** (5 / 6))


def psd(f, r0, L0, kind="von_karman"):
    a = 0.0 if kind == "kolmogorov" else 1.0 / L0 ** 2
    return vk_coeff() * r0 ** (-5 / 3) * (np.asarray(f, dtype=float) ** 2 + a) ** (-11 / 6)


def airy(f, D, d=0.0):
    """Eq. 7 aperture filter 2 (D J1(pi D f) - d J1(pi d f)) / (pi (D^2 - d^2) f), A(0)=1."""
    f = np.asarray(f, dtype=float)
    out = np.ones_like(f)
    nz = f > 0
    fn = f[nz]
    num = D * sp.j1(PI * D * fn) - (d * sp.j1(PI * d * fn) if d > 0 else 0.0)
    out[nz] = 2 * num / (PI * (D * D - d * d) * fn)
    return out


def parseval_annulus(r0, L0, fmin, fmax, kind="von_karman") -> float:
    a = 0.0 if kind == "kolmogorov" else 1.0 / L0 ** 2
    return float(6 * PI / 5 * vk_coeff() * r0 ** (-5 / 3)
                 * ((fmin ** 2 + a) ** (-5 / 6) - (fmax ** 2 + a) ** (-5 / 6)))


def _panels(fmin, fmax, osc_len, n_log=3000):
    """Breakpoints: log-spaced (the PSD's scale) merged with a linear grid fine
    enough to resolve oscillations of period 1/osc_len in f."""
    pts = [np.geomspace(max(fmin, 1e-12), fmax, n_log)]
    if osc_len > 0:
        n_lin = int(np.ceil(8 * (fmax - fmin) * osc_len)) + 2
        pts.append(np.linspace(fmin, fmax, min(n_lin, 400000)))
    b = np.unique(np.concatenate(pts))
    return b[(b >= fmin) & (b <= fmax)]


def _gl_integrate(g, breaks, order=8):
    x, w = np.polynomial.legendre.leggauss(order)
    a, b = breaks[:-1], breaks[1:]
    mid, half = (a + b) / 2, (b - a) / 2
    ff = mid[:, None] + half[:, None] * x[None, :]
    return float(np.sum(half[:, None] * w[None, :] * g(ff)))


def radial_integral(g, fmin, fmax, osc_len=0.0):
    """int_fmin^fmax g(f) df by composite 8-point Gauss-Legendre on merged panels."""
    return _gl_integrate(g, _panels(fmin, fmax, osc_len))


def piston_variance(r0, L0, D, d, fmin, fmax, kind="von_karman") -> float:
    """Variance of one aperture's piston: 2 pi int f W A^2 df."""
    return radial_integral(lambda f: 2 * PI * f * psd(f, r0, L0, kind) * airy(f, D, d) ** 2, fmin, fmax)


def piston_sf(B, r0, L0, D, d, fmin, fmax, kind="von_karman") -> float:
    """D(B) = 4 pi int f W A^2 (1 - J0(2 pi f B)) df, equal apertures D, d."""
    return radial_integral(
        lambda f: 4 * PI * f * psd(f, r0, L0, kind) * airy(f, D, d) ** 2 * (1 - sp.j0(2 * PI * f * B)),
        fmin, fmax, osc_len=B)


def piston_sf_general(B, r0, L0, D1, d1, D2, d2, fmin, fmax, kind="von_karman") -> float:
    """Apertures of different sizes: <(p1 - p2)^2> =
    2 pi int f W (A1^2 + A2^2 - 2 A1 A2 J0(2 pi f B)) df."""
    return radial_integral(
        lambda f: 2 * PI * f * psd(f, r0, L0, kind)
        * (airy(f, D1, d1) ** 2 + airy(f, D2, d2) ** 2 - 2 * airy(f, D1, d1) * airy(f, D2, d2)
           * sp.j0(2 * PI * f * B)), fmin, fmax, osc_len=B)


def phase_sf(r, r0, L0, fmin, fmax, kind="von_karman") -> float:
    """Phase structure function restricted to the annulus: 4 pi int f W (1 - J0(2 pi f r)) df."""
    return radial_integral(lambda f: 4 * PI * f * psd(f, r0, L0, kind) * (1 - sp.j0(2 * PI * f * r)),
                           fmin, fmax, osc_len=r)


def phase_sf_vk_infinite(r, r0, L0) -> float:
    """Textbook von Karman phase structure function on the whole plane:
    D(r) = c' (L0/r0)^(5/3) [Gamma(5/6)/2^(1/6) - (2 pi r/L0)^(5/6) K_{5/6}(2 pi r/L0)],
    c' = 2^(1/6) Gamma(11/6) / pi^(8/3) * (24/5 Gamma(6/5))^(5/6)."""
    cp = 2 ** (1 / 6) * sp.gamma(11 / 6) / PI ** (8 / 3) * (24 / 5 * sp.gamma(6 / 5)) ** (5 / 6)
    x = 2 * PI * r / L0
    return float(cp * (L0 / r0) ** (5 / 3) * (sp.gamma(5 / 6) / 2 ** (1 / 6) - x ** (5 / 6) * sp.kv(5 / 6, x)))


def conditional_piston_sf(f, F, A1, A2, B):
    """Exact coefficient-average of (p1 - p2)^2 for ONE draw (terms f [K][2],
    amplitude F [K], filters A1, A2 [K], baseline vector B [2]):
    sum_k F_k^2 (A1^2 + A2^2 - 2 A1 A2 cos 2 pi f.B)."""
    ph = 2 * PI * (f[..., 0] * B[0] + f[..., 1] * B[1])
    return np.sum(F ** 2 * (A1 ** 2 + A2 ** 2 - 2 * A1 * A2 * np.cos(ph)), axis=-1)


def temporal_piston_sf(tau, B, v, r0, L0, D, d, fmin, fmax, wind_angle=0.0, kind="von_karman"):
    """Frozen-flow temporal structure function of the differential piston of two
    equal apertures separated by the vector B (length |B| along x) with wind
    speed v at angle wind_angle to B:
      D(tau) = 8 pi int f W A^2 [1 - J0(2 pi f|B|) - J0(2 pi f v tau)
               + J0(2 pi f |B + v tau|)/2 + J0(2 pi f |B - v tau|)/2] df."""
    Bv = np.array([B, 0.0])
    w = np.array([np.cos(wind_angle), np.sin(wind_angle)]) * v * tau
    bp, bm, vt = np.linalg.norm(Bv + w), np.linalg.norm(Bv - w), v * tau
    osc = max(B, bp, bm, vt)
    return radial_integral(
        lambda f: 8 * PI * f * psd(f, r0, L0, kind) * airy(f, D, d) ** 2
        * (1 - sp.j0(2 * PI * f * B) - sp.j0(2 * PI * f * vt)
           + 0.5 * sp.j0(2 * PI * f * bp) + 0.5 * sp.j0(2 * PI * f * bm)), fmin, fmax, osc_len=osc)


def choose_n(r0, L0, D, d, delta_f, eps_rel, n_max=10000):
    """Sec. 4.2 choice of N: g(x) = int_0^x f W(f) A(f)^2 df (A = 1 when D = 0)
    saturates at g_inf; N = 2 m for the first m past the largest panel
    increment with g(m df) - g((m-1) df) < eps_rel g_inf.  Panels by adaptive
    quadrature (scipy.integrate.quad); g_inf from the full radial integral.
    Returns (N, g(m df), g_inf)."""
    from scipy import integrate

    def g(f):
        a = airy(f, D, d) if D > 0 else 1.0
        return f * psd(f, r0, L0) * a * a

    g_inf = radial_integral(g, 1e-12, 1e6) if D > 0 else radial_integral(g, 1e-12, 1e9)
    gm, peak = 0.0, 0.0
    for m in range(1, n_max // 2 + 1):
        inc = integrate.quad(g, (m - 1) * delta_f, m * delta_f, epsabs=0.0, epsrel=1e-12, limit=200)[0]
        gm += inc
        if inc < eps_rel * g_inf and inc < peak:
            return 2 * m, gm, g_inf
        peak = max(peak, inc)
    raise ValueError("criterion not met below n_max")


def square_temporal_piston_sf(taus, B, v, r0, L0, D, d, fmax, wind_angle=0.0, panel_nodes=8):
    """Frozen-flow temporal structure function of the differential piston of two
    equal apertures B = (|B|, 0) apart, wind speed v at wind_angle to B, for
    the SQUARE domain [-fmax, fmax)^2 (Eq. 5): with s = v tau (cos, sin)(angle),
      D(tau) = int W A^2 [4 - 4 cos 2 pi f.B - 4 cos 2 pi f.s
                          + 2 cos 2 pi f.(B + s) + 2 cos 2 pi f.(B - s)] d^2 f,
    the variance of Delta(t + tau) - Delta(t) for the covariance
    C(r) = int W A^2 cos 2 pi f.r of the piston field.  Tensor Gauss-Legendre
    on panels narrower than 1/8 of the shortest period of the cosines (one
    node grid for all lags).  Returns an array over taus."""
    taus = np.atleast_1d(np.asarray(taus, dtype=np.float64))
    Bv = np.array([B, 0.0])
    wdir = np.array([np.cos(wind_angle), np.sin(wind_angle)])
    Lmax = max([1.0 / fmax, abs(B)] + [np.linalg.norm(Bv + sg * wdir * v * t) for t in taus for sg in (-1, 1)])
    n_pan = int(np.ceil(2 * fmax * 8 * Lmax))
    x, w = np.polynomial.legendre.leggauss(panel_nodes)
    edges = np.linspace(-fmax, fmax, n_pan + 1)
    h = edges[1] - edges[0]
    nodes = (edges[:-1, None] + 0.5 * h * (x[None, :] + 1.0)).ravel()
    wts = np.tile(0.5 * h * w, n_pan)
    out = np.zeros(taus.size)
    for i0 in range(0, nodes.size, 256):  # blocks of rows
        fx = nodes[i0:i0 + 256, None]
        fy = nodes[None, :]
        fr = np.hypot(fx, fy)
        a = airy(fr.ravel(), D, d).reshape(fr.shape) if D > 0 else 1.0
        K = wts[i0:i0 + 256, None] * wts[None, :] * psd(fr, r0, L0) * a * a
        c0 = np.sum(K)
        cB = np.sum(K * np.cos(2 * PI * fx * B))
        for j, t in enumerate(taus):
            sx, sy = wdir * v * t
            cs = np.sum(K * np.cos(2 * PI * (fx * sx + fy * sy)))
            cp = np.sum(K * np.cos(2 * PI * (fx * (B + sx) + fy * sy)))
            cm = np.sum(K * np.cos(2 * PI * (fx * (B - sx) - fy * sy)))
            out[j] += 4 * c0 - 4 * cB - 4 * cs + 2 * cp + 2 * cm
    return out
