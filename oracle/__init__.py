"""FP64 CPU oracle for quasi-random frequency-sampling turbulence synthesis.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.
It shares no code with the CUDA library.  The C source ``qrs_oracle.c`` holds
the method (Philox4x32-10, the R2 sequence of Eq. 6, the domain maps of Eq. 5
and the square-to-disc remark of Sec. 3.2, the PSD and filter of Eq. 7, the
sum of Eq. 3, pistons and structure functions of Sec. 4); this module only
marshals numpy arrays into it.  ``analytic.py`` holds the closed forms and
quadratures that pin it.

Parameters are plain keyword dictionaries (see ``params()``) so that the
oracle never sees a structure of the CUDA binding.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qrs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PSD = {"von_karman": 0, "kolmogorov": 1}
DOMAIN = {"square": 0, "disc": 1, "logpolar": 2}
SAMPLER = {"r2": 0, "jitter": 1, "uniform": 2, "importance": 3}
COEF = {"gauss": 0, "eq3": 1}


def build(force: bool = False) -> str:
    """Compile liboracle.so from qrs_oracle.c with gcc (plain C, -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            u32p, u64p = C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)
            L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.oracle_r2_seed.argtypes = [C.c_uint64, C.c_int, C.c_uint64, C.c_uint64, u64p]
            L.oracle_r2_point.argtypes = [u64p, C.c_uint64, u64p]
            L.oracle_psd.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double]
            L.oracle_psd.restype = C.c_double
            L.oracle_airy.argtypes = [C.c_double, C.c_double, C.c_double]
            L.oracle_airy.restype = C.c_double
            L.oracle_domain_map.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                                            C.POINTER(C.c_double)]
            L.oracle_domain_jacobian.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
            L.oracle_domain_jacobian.restype = C.c_double
            P = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_double, C.c_double,
                 C.c_int, C.c_uint64, C.c_int, C.c_uint64, C.c_uint64, C.c_int, C.c_int, C.c_int,
                 C.c_void_p, C.c_int, C.c_double]
            L.oracle_draw.argtypes = P + [C.c_int64, C.c_int64, C.c_int64] + [C.c_void_p] * 7
            L.oracle_synth_terms.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                             C.c_void_p, C.c_int64, C.c_void_p]
            L.oracle_synthesize.argtypes = P + [C.c_int64, C.c_int64, C.c_int64, C.c_void_p,
                                                C.c_int64, C.c_void_p]
            L.oracle_synthesize_shared.argtypes = P + [C.c_int64, C.c_int64, C.c_int64, C.c_void_p,
                                                       C.c_void_p, C.c_int64, C.c_void_p]
            L.oracle_diff_piston.argtypes = P + [C.c_int64, C.c_int64, C.c_int64, C.c_void_p,
                                                 C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                                 C.c_int, C.c_void_p, C.c_void_p]
            L.oracle_structure_fn.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64,
                                              C.c_void_p, C.c_int, C.c_void_p]
            L.oracle_fft_spectrum.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int64,
                                              C.c_double, C.c_uint64, C.c_int64, C.c_int64, C.c_void_p]
            L.oracle_nearest_neighbour.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p]
            L.oracle_star_discrepancy.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p]
            for name in ("oracle_fft_spectrum", "oracle_nearest_neighbour", "oracle_star_discrepancy", "oracle_draw",
                         "oracle_synth_terms",
                         "oracle_synthesize",
                         "oracle_synthesize_shared", "oracle_diff_piston", "oracle_structure_fn"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def params(psd="von_karman", r0=0.15, L0=30.0, domain="logpolar", fmin=1e-3, fmax=16.0,
           sampler="r2", seed=0, s0=None, coef="gauss", n_rho=64, n_theta=32, cdf=None, ap_D=0.0, ap_d=0.0,
           fold=0, frame=0.0):
    """Plain dictionary of method parameters (shared vocabulary, no arithmetic).
    ap_D > 0 filters the PSD by the Eq. 7 aperture factor (the piston PSD);
    fold (2 or 4) and frame (turns) lay the IMPORTANCE cells over one mirrored
    sector of a rotated frame."""
    return dict(psd=psd, r0=r0, L0=L0, domain=domain, fmin=fmin, fmax=fmax, sampler=sampler,
                seed=seed, s0=s0, coef=coef, n_rho=n_rho, n_theta=n_theta, cdf=cdf, ap_D=ap_D, ap_d=ap_d,
                fold=fold, frame=frame)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _pargs(p):
    cdf = p.get("cdf")
    if cdf is not None:
        cdf = np.ascontiguousarray(cdf, dtype=np.uint32)
    s0 = p.get("s0")
    use_fixed = 0 if s0 is None else 1
    s0x, s0y = (0, 0) if s0 is None else (int(s0[0]), int(s0[1]))
    args = [PSD[p["psd"]], float(p["r0"]), float(p["L0"]), float(p.get("ap_D", 0.0) or 0.0),
            float(p.get("ap_d", 0.0) or 0.0), DOMAIN[p["domain"]], float(p["fmin"]),
            float(p["fmax"]), SAMPLER[p["sampler"]], int(p["seed"]) & (2**64 - 1), use_fixed, s0x, s0y,
            COEF[p["coef"]], int(p["n_rho"]), int(p["n_theta"]), _ptr(cdf), int(p.get("fold", 0) or 0),
            float(p.get("frame", 0.0) or 0.0)]
    return args, cdf  # keep cdf alive


# ------------------------------------------------------------------ primitives
def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def r2_seed(seed, s0=None):
    o = (C.c_uint64 * 2)()
    if s0 is None:
        lib().oracle_r2_seed(int(seed) & (2**64 - 1), 0, 0, 0, o)
    else:
        lib().oracle_r2_seed(0, 1, int(s0[0]), int(s0[1]), o)
    return int(o[0]), int(o[1])


def r2_point(s0, n):
    a = (C.c_uint64 * 2)(int(s0[0]), int(s0[1]))
    o = (C.c_uint64 * 2)()
    lib().oracle_r2_point(a, int(n), o)
    return int(o[0]), int(o[1])


def psd(kind, r0, L0, f2):
    return lib().oracle_psd(PSD[kind], float(r0), float(L0), float(f2))


def airy(f, D, d=0.0):
    return lib().oracle_airy(float(f), float(D), float(d))


def domain_map(kind, fmin, fmax, sx, sy):
    o = (C.c_double * 2)()
    lib().oracle_domain_map(DOMAIN[kind], float(fmin), float(fmax), float(sx), float(sy), o)
    return float(o[0]), float(o[1])


def domain_jacobian(kind, fmin, fmax, fx, fy):
    return lib().oracle_domain_jacobian(DOMAIN[kind], float(fmin), float(fmax), float(fx), float(fy))


# ---------------------------------------------------------------------- method
def draw(p, n_f, n_real=1, real_offset=0, debug=False):
    """Draw n_real x n_f terms.  Returns a dict of numpy arrays:
    f [n_real][n_f][2] float32, F, J [n_real][n_f] float64, coef [..][2] float64,
    cell int32 and, with debug, words [..][4] uint32 and r2 [..][2] uint64."""
    n = n_real * n_f
    f = np.zeros((n_real, n_f, 2), np.float32)
    F = np.zeros((n_real, n_f), np.float64)
    J = np.zeros((n_real, n_f), np.float64)
    coef = np.zeros((n_real, n_f, 2), np.float64)
    cell = np.zeros((n_real, n_f), np.int32)
    words = np.zeros((n_real, n_f, 4), np.uint32) if debug else None
    r2 = np.zeros((n_real, n_f, 2), np.uint64) if debug else None
    args, keep = _pargs(p)
    rc = lib().oracle_draw(*args, int(n_f), int(n_real), int(real_offset), _ptr(f), _ptr(F), _ptr(J),
                           _ptr(coef), _ptr(cell), _ptr(words), _ptr(r2))
    assert rc == 0 and n >= 0
    out = dict(f=f, F=F, J=J, coef=coef, cell=cell)
    if debug:
        out.update(words=words, r2=r2)
    return out


def synth_terms(f, F, coef, xy):
    """Eq. 3 at points xy for explicit terms (f [K][2] fp32, F [K], coef [K][2])."""
    f = np.ascontiguousarray(f, np.float32).reshape(-1, 2)
    F = np.ascontiguousarray(F, np.float64).reshape(-1)
    coef = np.ascontiguousarray(coef, np.float64).reshape(-1, 2)
    xy = np.ascontiguousarray(xy, np.float32).reshape(-1, 2)
    out = np.zeros(xy.shape[0], np.float64)
    lib().oracle_synth_terms(_ptr(f), _ptr(F), _ptr(coef), f.shape[0], _ptr(xy), xy.shape[0], _ptr(out))
    return out


def synthesize(p, n_f, n_real, xy, real_offset=0):
    xy = np.ascontiguousarray(xy, np.float32).reshape(-1, 2)
    out = np.zeros((n_real, xy.shape[0]), np.float64)
    args, keep = _pargs(p)
    rc = lib().oracle_synthesize(*args, int(n_f), int(n_real), int(real_offset), _ptr(xy), xy.shape[0],
                                 _ptr(out))
    assert rc == 0
    return out


def synthesize_shared(p, n_f, n_real, xy, real_offset=0, col_psd=None):
    xy = np.ascontiguousarray(xy, np.float32).reshape(-1, 2)
    out = np.zeros((n_real, xy.shape[0]), np.float64)
    cp = None if col_psd is None else np.ascontiguousarray(col_psd, np.float64).reshape(n_real, 2)
    args, keep = _pargs(p)
    rc = lib().oracle_synthesize_shared(*args, int(n_f), int(n_real), int(real_offset), _ptr(cp),
                                        _ptr(xy), xy.shape[0], _ptr(out))
    assert rc == 0
    return out


def diff_piston(p, n_f, n_real, ap_xy, ap_D, ap_d=None, pairs=None, real_offset=0):
    """Returns (piston [n_real][n_ap], delta [n_real][n_pairs]) in FP64."""
    ap_xy = np.ascontiguousarray(ap_xy, np.float32).reshape(-1, 2)
    n_ap = ap_xy.shape[0]
    ap_D = np.ascontiguousarray(ap_D, np.float32).reshape(n_ap)
    ap_d = np.zeros(n_ap, np.float32) if ap_d is None else np.ascontiguousarray(ap_d, np.float32).reshape(n_ap)
    if pairs is None:
        pairs = np.array([(i, j) for i in range(n_ap) for j in range(i + 1, n_ap)], np.int32).reshape(-1, 2)
    pairs = np.ascontiguousarray(pairs, np.int32).reshape(-1, 2)
    pis = np.zeros((n_real, n_ap), np.float64)
    out = np.zeros((n_real, pairs.shape[0]), np.float64)
    args, keep = _pargs(p)
    rc = lib().oracle_diff_piston(*args, int(n_f), int(n_real), int(real_offset), _ptr(ap_xy), _ptr(ap_D),
                                  _ptr(ap_d), n_ap, _ptr(pairs), pairs.shape[0], _ptr(pis), _ptr(out))
    assert rc == 0
    return pis, out


def structure_fn(delta, lags):
    """delta [n_real][n_series][T] float32 -> acc [n_series][n_lags][3] FP64."""
    delta = np.ascontiguousarray(delta, np.float32)
    assert delta.ndim == 3
    lags = np.ascontiguousarray(lags, np.int32).reshape(-1)
    acc = np.zeros((delta.shape[1], lags.shape[0], 3), np.float64)
    lib().oracle_structure_fn(_ptr(delta), delta.shape[0], delta.shape[1], delta.shape[2], _ptr(lags),
                              lags.shape[0], _ptr(acc))
    return acc


def nearest_neighbour(pts):
    """pts [n_sets][n][2] float32 -> nearest-other-point distance [n_sets][n] FP64."""
    pts = np.ascontiguousarray(pts, np.float32)
    if pts.ndim == 2:
        pts = pts[None]
    out = np.zeros(pts.shape[:2], np.float64)
    lib().oracle_nearest_neighbour(_ptr(pts), pts.shape[0], pts.shape[1], _ptr(out))
    return out


def star_discrepancy(pts):
    """pts [n_sets][n][2] float32 in [0,1]^2 -> D* [n_sets] FP64 (exact, O(n^3))."""
    pts = np.ascontiguousarray(pts, np.float32)
    if pts.ndim == 2:
        pts = pts[None]
    out = np.zeros(pts.shape[0], np.float64)
    lib().oracle_star_discrepancy(_ptr(pts), pts.shape[0], pts.shape[1], _ptr(out))
    return out


def fft_spectrum(p, n, dx, n_real, real_offset=0):
    """The Eq. 2 spectrum on the FFT grid (see oracle_fft_spectrum): complex128 [n_real][n][n]."""
    spec = np.zeros((n_real, n, n, 2), np.float64)
    rc = lib().oracle_fft_spectrum(PSD[p["psd"]], float(p["r0"]), float(p.get("L0", 0.0) or 0.0),
                                   float(p.get("ap_D", 0.0) or 0.0), float(p.get("ap_d", 0.0) or 0.0), int(n),
                                   float(dx), int(p.get("seed", 0)) & (2**64 - 1), int(n_real), int(real_offset),
                                   _ptr(spec))
    assert rc == 0
    return spec[..., 0] + 1j * spec[..., 1]


def fft_screen(p, n, dx, n_real, real_offset=0):
    """Eq. 2: n^2 times the inverse DFT of the spectrum, sum_f S(f) e^{2 pi i f.x} at
    x = (j dx, i dx) (numpy, FP64); returns (real part, imaginary part), each [n_real][n][n]
    (row i = y, column j = x)."""
    chi = np.fft.ifft2(fft_spectrum(p, n, dx, n_real, real_offset), norm="forward")
    return chi.real, chi.imag
