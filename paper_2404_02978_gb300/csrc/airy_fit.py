"""Coefficients of the large-argument form of the Eq. 7 aperture filter used by
the kernels (qrs_device.cuh, AiryLarge<DEG>): writes them as C++ initialisers.

For x >= x0 the Bessel function is written in modulus-phase form,
    J1(x) = sqrt(2 / (pi x)) M(x) cos(x - 3 pi / 4 + T(x) / x),
with M(x) = sqrt(pi x / 2) |J1 + i Y1| and x - 3 pi/4 + T(x)/x the argument of
J1 + i Y1; both M and T are smooth, even functions of u = 1/x, fitted here as
polynomials in w = 1/x^2 (least squares on a geometric grid of x in [x0, 2e4],
reference values from scipy.special.j1 / y1 in FP64).  The filter is then
    g(x) = 2 J1(x) / x = [2 sqrt(2/pi) M(w)] x^(-3/2) cos(2 pi [x / (2 pi) - 3/8 + u T(w) / (2 pi)]),
so the emitted coefficients are 2 sqrt(2/pi) M_i (amplitude) and T_i / (2 pi)
(phase in turns).  The script prints the largest error of g over the grid
for each fit.

    python paper_2404_02978_gb300/csrc/airy_fit.py
"""
import numpy as np
from scipy import special as sp

FITS = ((4.0, 4), (8.0, 2), (16.0, 1))  # (x0, degree in w)


def modulus_phase(x):
    J, Y = sp.j1(x), sp.y1(x)
    M = np.hypot(J, Y) * np.sqrt(np.pi * x / 2)
    d = np.arctan2(Y, J) - (x - 0.75 * np.pi)
    d = (d + np.pi) % (2 * np.pi) - np.pi
    return M, d * x  # T(x) = x (arg - (x - 3 pi / 4))


def fit(x0, deg):
    x = np.geomspace(x0, 2e4, 40000)
    w = 1.0 / (x * x)
    M, T = modulus_phase(x)
    cm = np.polynomial.polynomial.polyfit(w, M, deg)
    ct = np.polynomial.polynomial.polyfit(w, T, deg)
    amp = 2.0 * np.sqrt(2.0 / np.pi) * cm
    ph = ct / (2.0 * np.pi)
    # the error of g with the coefficients rounded to FP32, evaluated in FP64
    a32, p32 = amp.astype(np.float32).astype(np.float64), ph.astype(np.float32).astype(np.float64)
    g = 2.0 * sp.j1(x) / x
    ga = np.polynomial.polynomial.polyval(w, a32) * x ** -1.5 * \
        np.cos(2.0 * np.pi * (x / (2.0 * np.pi) - 0.375 + np.polynomial.polynomial.polyval(w, p32) / x))
    return amp, ph, float(np.max(np.abs(ga - g)))


if __name__ == "__main__":
    for x0, deg in FITS:
        amp, ph, err = fit(x0, deg)
        fmt = lambda c: ", ".join("%.9ef" % v for v in c)
        print("// x >= %g, degree %d in 1/x^2: max |g error| %.2e" % (x0, deg, err))
        print("//   amplitude {%s}" % fmt(amp))
        print("//   phase     {%s}" % fmt(ph))
