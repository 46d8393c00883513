"""Python binding of libqrs: quasi-random frequency-sampling turbulence synthesis
on one GB300 (sm_103a).

Thin marshalling over the C ABI declared in ``include/qrs.h`` (ctypes; torch
tensors are used only as device buffers and for the current CUDA stream).
Every step of the computation runs in libqrs's CUDA kernels; there is no CPU
or PyTorch fallback: if ``libqrs.so`` has not been built, every call raises.

The functions carry the C names (``qrs_draw``, ``qrs_synthesize_points``,
``qrs_diff_piston``, ``qrs_structure_fn``, ...).  Method parameters are a plain
dictionary, see ``params()``: PSD (Eq. 7), frequency domain (Eq. 5, the
square-to-disc map of Sec. 3.2, or log-polar), sampler (R2 of Eq. 6, jittered
grid of Eq. 4, uniform, importance cells) and coefficient form (Eq. 3).
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import threading

import torch

__all__ = ["params", "Handle", "qrs_create", "qrs_draw", "qrs_synthesize_points", "qrs_synthesize_grid", "qrs_diff_piston",
           "qrs_pair_diff", "qrs_choose_n", "qrs_fft_spectrum", "fft_screens", "qrs_nearest_neighbour", "qrs_star_discrepancy", "qrs_structure_fn", "qrs_sync", "QrsError", "lib_path", "load"]

_HERE = os.path.dirname(os.path.abspath(__file__))
# QRS_CHECKED=1 loads the bounds-checked build of the same library
_LIB_PATH = os.path.join(_HERE, "libqrs_checked.so" if os.environ.get("QRS_CHECKED") == "1" else "libqrs.so")

PSD = {"von_karman": 0, "kolmogorov": 1}
DOMAIN = {"square": 0, "disc": 1, "logpolar": 2}
SAMPLER = {"r2": 0, "jitter": 1, "uniform": 2, "importance": 3}
COEF = {"gauss": 0, "eq3": 1}
MODE = {"fused": 0, "gemm_3xtf32": 1, "gemm_bf16x3": 2, "gemm_tf32": 3}
PISTON_PERSISTENT, PISTON_GRAPH = 1, 2
STATUS = {0: "QRS_OK", -1: "QRS_ERR_ARG", -2: "QRS_ERR_CUDA", -3: "QRS_ERR_TIMEOUT", -4: "QRS_ERR_UNSUPPORTED",
          -5: "QRS_ERR_NOMEM", -6: "QRS_ERR_DEVICE_CHECK"}


class QrsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


# ------------------------------------------------------------------ C structs
class QrsPsd(C.Structure):
    _fields_ = [("r0_m", C.c_double), ("L0_m", C.c_double), ("kind", C.c_int32), ("reserved", C.c_int32),
                ("ap_D_m", C.c_double), ("ap_d_m", C.c_double)]


class QrsDomain(C.Structure):
    _fields_ = [("fmin", C.c_double), ("fmax", C.c_double), ("kind", C.c_int32), ("reserved", C.c_int32)]


class QrsSampler(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("s0", C.c_uint64 * 2), ("cell_cdf", C.c_void_p), ("kind", C.c_int32),
                ("coef_kind", C.c_int32), ("use_fixed_s0", C.c_int32), ("n_rho", C.c_int32),
                ("n_theta", C.c_int32), ("fold", C.c_int32), ("frame", C.c_double)]


class QrsDrawOut(C.Structure):
    _fields_ = [("f_xy", C.c_void_p), ("amp", C.c_void_p), ("coef", C.c_void_p), ("cell", C.c_void_p),
                ("words", C.c_void_p), ("r2", C.c_void_p)]


class QrsPistonJob(C.Structure):
    _fields_ = [("psd", QrsPsd), ("dom", QrsDomain), ("smp", QrsSampler), ("n_f", C.c_int64),
                ("n_real", C.c_int64), ("real_offset", C.c_int64), ("ap_xy", C.c_void_p), ("ap_D", C.c_void_p),
                ("ap_d", C.c_void_p), ("pairs", C.c_void_p), ("piston", C.c_void_p), ("delta", C.c_void_p),
                ("n_ap", C.c_int32), ("n_pairs", C.c_int32)]


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Load libqrs.so (raises if it has not been built: no fallback exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise ImportError("libqrs.so is not built (run `python -m paper_2404_02978_gb300.build` "
                              "or __graft_entry__.build()); this package has no CPU fallback")
        L = C.CDLL(_LIB_PATH)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.qrs_create.argtypes = [C.POINTER(vp), i32]
        L.qrs_destroy.argtypes = [vp]
        L.qrs_destroy.restype = None
        L.qrs_last_error.argtypes = [vp]
        L.qrs_last_error.restype = C.c_char_p
        L.qrs_sync.argtypes = [vp, vp]
        L.qrs_launch_count.argtypes = [vp]
        L.qrs_launch_count.restype = i64
        L.qrs_checked_build.argtypes = []
        L.qrs_checked_build.restype = i32
        L.qrs_check_selftest.argtypes = [vp, i64, vp]
        L.qrs_draw.argtypes = [vp, C.POINTER(QrsPsd), C.POINTER(QrsDomain), C.POINTER(QrsSampler), i64, i64, i64,
                               C.POINTER(QrsDrawOut), vp]
        L.qrs_synthesize_points.argtypes = [vp, C.POINTER(QrsPsd), C.POINTER(QrsDomain), C.POINTER(QrsSampler),
                                            i64, i64, i64, vp, i64, i32, vp, vp, vp]
        L.qrs_diff_piston.argtypes = [vp, C.POINTER(QrsPistonJob), i32, i32, vp]
        L.qrs_structure_fn.argtypes = [vp, vp, i64, i64, i64, vp, i32, vp, vp]
        for n in ("qrs_create", "qrs_sync", "qrs_draw", "qrs_synthesize_points", "qrs_diff_piston",
                  "qrs_structure_fn"):
            getattr(L, n).restype = C.c_int
        _lib = L
        return L


# ----------------------------------------------------------------- parameters
def params(psd="von_karman", r0=0.15, L0=30.0, domain="logpolar", fmin=1e-3, fmax=16.0, sampler="r2", seed=0,
           s0=None, coef="gauss", n_rho=64, n_theta=32, cdf=None, ap_D=0.0, ap_d=0.0, fold=0, frame=0.0):
    """Method parameters as a plain dictionary (cdf: device uint32 tensor or None;
    ap_D > 0: the PSD filtered by the Eq. 7 aperture factor; fold 2 or 4 and
    frame (turns): IMPORTANCE cells over mirrored sectors of a rotated frame;
    see include/qrs.h)."""
    return dict(psd=psd, r0=r0, L0=L0, domain=domain, fmin=fmin, fmax=fmax, sampler=sampler, seed=seed, s0=s0,
                coef=coef, n_rho=n_rho, n_theta=n_theta, cdf=cdf, ap_D=ap_D, ap_d=ap_d, fold=fold, frame=frame)


def _structs(p):
    psd = QrsPsd(float(p["r0"]), float(p.get("L0", 0.0) or 0.0), PSD[p["psd"]], 0, float(p.get("ap_D", 0.0) or 0.0),
                 float(p.get("ap_d", 0.0) or 0.0))
    dom = QrsDomain(float(p.get("fmin", 0.0) or 0.0), float(p["fmax"]), DOMAIN[p["domain"]], 0)
    s0 = p.get("s0")
    cdf = p.get("cdf")
    if cdf is not None:
        _check_dev(cdf, torch.int32, "cdf", allow=(torch.int32, getattr(torch, "uint32", torch.int32)))
    smp = QrsSampler(int(p.get("seed", 0)) & (2**64 - 1), (C.c_uint64 * 2)(*(s0 if s0 is not None else (0, 0))),
                     cdf.data_ptr() if cdf is not None else None, SAMPLER[p.get("sampler", "r2")],
                     COEF[p.get("coef", "gauss")], 0 if s0 is None else 1, int(p.get("n_rho", 64)),
                     int(p.get("n_theta", 32)), int(p.get("fold", 0) or 0), float(p.get("frame", 0.0) or 0.0))
    return psd, dom, smp


def _check_dev(t, dtype, name, allow=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    ok = (t.dtype in allow) if allow else (t.dtype == dtype)
    if not ok:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


def _stream(stream):
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


# --------------------------------------------------------------------- handle
class Handle:
    """Owns a qrs_handle on one CUDA device."""

    def __init__(self, device=0):
        self.L = load()
        self.device = int(device)
        h = C.c_void_p()
        st = self.L.qrs_create(C.byref(h), self.device)
        if st != 0:
            raise QrsError(st, "qrs_create(device=%d) failed" % self.device)
        self.h = h

    def _check(self, st):
        if st != 0:
            raise QrsError(st, self.L.qrs_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.qrs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def launch_count(self) -> int:
        return int(self.L.qrs_launch_count(self.h))


def qrs_create(device=0) -> Handle:
    return Handle(device)


def qrs_sync(h: Handle, stream=None):
    h._check(h.L.qrs_sync(h.h, _stream(stream)))


def checked_build() -> bool:
    """True when the loaded library is the bounds-checked build (QRS_CHECKED=1)."""
    return bool(load().qrs_checked_build())


def qrs_check_selftest(h: Handle, i: int, stream=None):
    """Checked build only: one store through the checked accessor at index i
    of an 8-float scratch (include/qrs.h); i outside [0, 8) is reported by the
    next qrs_sync as QRS_ERR_DEVICE_CHECK."""
    h._check(h.L.qrs_check_selftest(h.h, int(i), _stream(stream)))


def qrs_draw(h: Handle, p, n_f, n_real, real_offset=0, outputs=("f_xy", "amp", "coef", "cell"), stream=None):
    """Eq. 3/5/6 draw.  Returns a dict of new device tensors for the requested
    outputs among f_xy, amp, coef, cell, words, r2."""
    dev = torch.device("cuda", h.device)
    shapes = {"f_xy": ((n_real, n_f, 2), torch.float32), "amp": ((n_real, n_f), torch.float32),
              "coef": ((n_real, n_f, 2), torch.float32), "cell": ((n_real, n_f), torch.int32),
              "words": ((n_real, n_f, 4), torch.int32), "r2": ((n_real, n_f, 2), torch.int64)}
    res = {k: torch.empty(*shapes[k][0], dtype=shapes[k][1], device=dev) for k in outputs}
    o = QrsDrawOut(*[(res[k].data_ptr() if k in res else None) for k in ("f_xy", "amp", "coef", "cell", "words", "r2")])
    psd, dom, smp = _structs(p)
    h._check(h.L.qrs_draw(h.h, C.byref(psd), C.byref(dom), C.byref(smp), int(n_f), int(n_real), int(real_offset),
                          C.byref(o), _stream(stream)))
    return res


def qrs_synthesize_points(h: Handle, p, n_f, n_real, xy, out=None, mode="fused", real_offset=0, col_psd=None,
                          stream=None):
    """Eq. 3 at the points xy [P,2] (float32, device); returns out [n_real, P] float32."""
    _check_dev(xy, torch.float32, "xy")
    P = xy.shape[0]
    if out is None:
        out = torch.empty(n_real, P, dtype=torch.float32, device=xy.device)
    _check_dev(out, torch.float32, "out")
    if out.numel() != n_real * P:
        raise ValueError("out must hold n_real * n_points values")
    cp = None
    if col_psd is not None:
        _check_dev(col_psd, torch.float64, "col_psd")
        cp = col_psd.data_ptr()
    psd, dom, smp = _structs(p)
    h._check(h.L.qrs_synthesize_points(h.h, C.byref(psd), C.byref(dom), C.byref(smp), int(n_f), int(n_real),
                                       int(real_offset), xy.data_ptr(), int(P), MODE[mode], cp, out.data_ptr(),
                                       _stream(stream)))
    return out


def qrs_synthesize_grid(h: Handle, p, n_f, n_real, x, y, index=None, n_points=None, out=None, mode="gemm_3xtf32",
                        real_offset=0, stream=None):
    """Eq. 3 on the tensor-product grid {x} x {y} (float32 device vectors) by the
    separable tensor-core form.  index None: returns out [n_real, ny, nx];
    else index int32 [ny, nx] (output point per node, -1 = none) and out
    [n_real, n_points]; n_points is then required (the binding runs no
    kernel of its own to find it)."""
    _check_dev(x, torch.float32, "x")
    _check_dev(y, torch.float32, "y")
    nx, ny = x.numel(), y.numel()
    ip = None
    if index is not None:
        _check_dev(index, torch.int32, "index")
        if index.numel() != nx * ny:
            raise ValueError("index must hold ny * nx entries")
        if n_points is None:
            raise ValueError("n_points is required with an index (the number of output points)")
        ip = index.data_ptr()
        shape = (n_real, n_points)
    else:
        n_points = nx * ny
        shape = (n_real, ny, nx)
    if out is None:
        out = torch.empty(*shape, dtype=torch.float32, device=x.device)
    _check_dev(out, torch.float32, "out")
    if out.numel() != n_real * n_points:
        raise ValueError("out must hold n_real * n_points values")
    f = h.L.qrs_synthesize_grid
    if f.argtypes is None:
        f.argtypes = [C.c_void_p, C.POINTER(QrsPsd), C.POINTER(QrsDomain), C.POINTER(QrsSampler), C.c_int64,
                      C.c_int64, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                      C.c_int32, C.c_void_p, C.c_void_p]
        f.restype = C.c_int
    psd, dom, smp = _structs(p)
    h._check(f(h.h, C.byref(psd), C.byref(dom), C.byref(smp), int(n_f), int(n_real), int(real_offset), x.data_ptr(),
               int(nx), y.data_ptr(), int(ny), ip, int(n_points), MODE[mode], out.data_ptr(), _stream(stream)))
    return out


def qrs_pair_diff(h: Handle, values, pairs, out=None, stream=None):
    """Pair differences out[r][q] = values[r][pairs[q][0]] - values[r][pairs[q][1]]
    (values [n_real, n_points] float32, pairs [n_pairs, 2] int32, device)."""
    _check_dev(values, torch.float32, "values")
    _check_dev(pairs, torch.int32, "pairs")
    n_real, n_points = values.shape
    n_pairs = pairs.shape[0]
    if out is None:
        out = torch.empty(n_real, n_pairs, dtype=torch.float32, device=values.device)
    _check_dev(out, torch.float32, "out")
    if out.numel() != n_real * n_pairs:
        raise ValueError("out must hold n_real * n_pairs values")
    f = h.L.qrs_pair_diff
    if f.argtypes is None:
        f.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
        f.restype = C.c_int
    h._check(f(h.h, values.data_ptr(), int(n_real), int(n_points), pairs.data_ptr(), int(n_pairs), out.data_ptr(),
               _stream(stream)))
    return out


def _stats(h, name, pts, out, dtype, shape):
    _check_dev(pts, torch.float32, "pts")
    if pts.dim() == 2:
        pts = pts.unsqueeze(0)
    n_sets, n = pts.shape[0], pts.shape[1]
    if out is None:
        out = torch.empty(*shape(n_sets, n), dtype=dtype, device=pts.device)
    _check_dev(out, dtype, "out")
    f = getattr(h.L, name)
    if f.argtypes is None:
        f.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p]
        f.restype = C.c_int
    h._check(f(h.h, pts.data_ptr(), int(n_sets), int(n), out.data_ptr(), _stream(None)))
    return out


def qrs_nearest_neighbour(h: Handle, pts, out=None):
    """pts [n_sets, n, 2] (or [n, 2]) float32 -> nearest-other-point distance [n_sets, n] float32."""
    return _stats(h, "qrs_nearest_neighbour", pts, out, torch.float32, lambda s, n: (s, n))


def qrs_star_discrepancy(h: Handle, pts, out=None):
    """pts [n_sets, n, 2] (or [n, 2]) float32 in [0,1]^2 -> exact star discrepancy [n_sets] float64."""
    return _stats(h, "qrs_star_discrepancy", pts, out, torch.float64, lambda s, n: (s,))


def qrs_choose_n(p, delta_f, eps_rel, n_max=10000):
    """Sec. 4.2 choice of N (host computation in libqrs): returns
    (N, g(N delta_f / 2), g_inf, stopping increment) for the PSD of p (von
    Karman, optionally aperture-filtered by p["ap_D"], p["ap_d"])."""
    f = load().qrs_choose_n
    if f.argtypes is None:
        f.argtypes = [C.POINTER(QrsPsd), C.c_double, C.c_double, C.c_int32, C.POINTER(C.c_int32),
                      C.POINTER(C.c_double)]
        f.restype = C.c_int
    psd, _, _ = _structs(p)
    n, g = C.c_int32(), (C.c_double * 3)()
    st = f(C.byref(psd), float(delta_f), float(eps_rel), int(n_max), C.byref(n), g)
    if st != 0:
        raise QrsError(st, "qrs_choose_n: invalid PSD or arguments, or the criterion is not met below n_max")
    return n.value, g[0], g[1], g[2]


def piston_job(p, n_f, n_real, ap_xy, ap_D, ap_d=None, pairs=None, piston=None, delta=None, real_offset=0):
    """Build one QrsPistonJob (device tensors; keeps them referenced in ._keep)."""
    _check_dev(ap_xy, torch.float32, "ap_xy")
    n_ap = ap_xy.shape[0]
    _check_dev(ap_D, torch.float32, "ap_D")
    if ap_d is not None:
        _check_dev(ap_d, torch.float32, "ap_d")
    n_pairs = 0
    if pairs is not None:
        _check_dev(pairs, torch.int32, "pairs")
        n_pairs = pairs.shape[0]
    psd, dom, smp = _structs(p)
    j = QrsPistonJob(psd, dom, smp, int(n_f), int(n_real), int(real_offset), ap_xy.data_ptr(), ap_D.data_ptr(),
                     ap_d.data_ptr() if ap_d is not None else None, pairs.data_ptr() if pairs is not None else None,
                     piston.data_ptr() if piston is not None else None, delta.data_ptr() if delta is not None else None,
                     int(n_ap), int(n_pairs))
    j._keep = (ap_xy, ap_D, ap_d, pairs, piston, delta, p.get("cdf"))
    return j


def qrs_diff_piston(h: Handle, jobs, flags=0, stream=None):
    """Run a list of piston jobs (see piston_job)."""
    arr = (QrsPistonJob * len(jobs))(*jobs)
    h._check(h.L.qrs_diff_piston(h.h, arr, len(jobs), int(flags), _stream(stream)))


def qrs_structure_fn(h: Handle, delta, lags, acc=None, stream=None):
    """Sec. 4.4 sums: delta [R, S, T] float32, lags [L] int32 -> acc [S, L, 3] float64 (accumulated)."""
    _check_dev(delta, torch.float32, "delta")
    _check_dev(lags, torch.int32, "lags")
    R, S, T = delta.shape
    if acc is None:
        acc = torch.zeros(S, lags.shape[0], 3, dtype=torch.float64, device=delta.device)
    _check_dev(acc, torch.float64, "acc")
    h._check(h.L.qrs_structure_fn(h.h, delta.data_ptr(), int(R), int(S), int(T), lags.data_ptr(),
                                  int(lags.shape[0]), acc.data_ptr(), _stream(stream)))
    return acc


def qrs_fft_spectrum(h: Handle, p, n, dx, n_real, real_offset=0, out=None, stream=None):
    """Spectrum of the Eq. 2 FFT screens (include/qrs.h): complex64 [n_real, n, n] on the device."""
    if out is None:
        out = torch.empty(n_real, n, n, dtype=torch.complex64, device=torch.device("cuda", h.device))
    _check_dev(out, torch.complex64, "out")
    if out.numel() != n_real * n * n:
        raise ValueError("out must hold n_real * n * n values")
    f = h.L.qrs_fft_spectrum
    if f.argtypes is None:
        f.argtypes = [C.c_void_p, C.POINTER(QrsPsd), C.c_int64, C.c_double, C.c_uint64, C.c_int64, C.c_int64,
                      C.c_void_p, C.c_void_p]
        f.restype = C.c_int
    psd, _, _ = _structs(p)
    h._check(f(h.h, C.byref(psd), int(n), float(dx), int(p.get("seed", 0)) & (2**64 - 1), int(n_real),
               int(real_offset), out.data_ptr(), _stream(stream)))
    return out


def fft_screens(h: Handle, p, n, dx, n_real, real_offset=0, stream=None):
    """The paper's comparison method (Eq. 2): n_real spectra from qrs_fft_spectrum, then
    n^2 times their inverse DFT by cuFFT (torch.fft), whose real and imaginary parts are
    two screens each: returns float32 [2, n_real, n, n] (part, realisation, row y,
    column x), points (j dx, i dx).  Not the paper's method: a baseline whose static
    frequency grid biases the structure function."""
    spec = qrs_fft_spectrum(h, p, n, dx, n_real, real_offset, stream=stream)
    with torch.cuda.stream(stream) if isinstance(stream, torch.cuda.Stream) else contextlib.nullcontext():
        chi = torch.fft.ifft2(spec, norm="forward")
        return torch.stack([chi.real, chi.imag])


def qrs_synthesize_points_noalloc(p, n_f, n_real, xy, out=None, real_offset=0, stream=None):
    """No-allocation fused synthesis on the current device (no handle; see include/qrs.h).
    For callers that cannot allocate device memory: pass a preallocated `out`."""
    L = load()
    f = L.qrs_synthesize_points_noalloc
    if f.argtypes is None:
        f.argtypes = [C.POINTER(QrsPsd), C.POINTER(QrsDomain), C.POINTER(QrsSampler), C.c_int64, C.c_int64,
                      C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
        f.restype = C.c_int
    _check_dev(xy, torch.float32, "xy")
    P = xy.shape[0]
    if out is None:
        out = torch.empty(n_real, P, dtype=torch.float32, device=xy.device)
    _check_dev(out, torch.float32, "out")
    if out.numel() != n_real * P:
        raise ValueError("out must hold n_real * n_points values")
    psd, dom, smp = _structs(p)
    st = f(C.byref(psd), C.byref(dom), C.byref(smp), int(n_f), int(n_real), int(real_offset), xy.data_ptr(), int(P),
           out.data_ptr(), _stream(stream))
    if st != 0:
        raise QrsError(st, "qrs_synthesize_points_noalloc failed")
    return out


# ------------------------------------------------------- learned proposal
def _prop_fn(name, argtypes, restype=C.c_int):
    f = getattr(load(), name)
    if f.argtypes is None:
        f.argtypes = argtypes
        f.restype = restype
    return f


def qrs_mlp_param_count(n_cells) -> int:
    return int(_prop_fn("qrs_mlp_param_count", [C.c_int32], C.c_int64)(int(n_cells)))


def qrs_mlp_init(h: Handle, n_cells, seed, params=None, stream=None, out_scale=1.0):
    """He-normal parameters; the output layer's weights times out_scale."""
    n = qrs_mlp_param_count(n_cells)
    if params is None:
        params = torch.empty(n, dtype=torch.float32, device=torch.device("cuda", h.device))
    _check_dev(params, torch.float32, "params")
    f = _prop_fn("qrs_mlp_init", [C.c_void_p, C.c_int32, C.c_uint64, C.c_float, C.c_void_p, C.c_void_p])
    h._check(f(h.h, int(n_cells), int(seed) & (2**64 - 1), float(out_scale), params.data_ptr(), _stream(stream)))
    return params


def qrs_proposal_prior(h: Handle, p, n_rho, n_theta, geom, fold=0, out=None, stream=None):
    """Per-cell prior of the logits [n][n_rho n_theta] (geom: device float64 [n][5]); see include/qrs_proposal.h."""
    _check_dev(geom, torch.float64, "geom")
    n = geom.shape[0]
    if out is None:
        out = torch.empty(n, n_rho * n_theta, dtype=torch.float32, device=geom.device)
    _check_dev(out, torch.float32, "out")
    psd, dom, _ = _structs(p)
    f = _prop_fn("qrs_proposal_prior", [C.c_void_p, C.POINTER(QrsPsd), C.POINTER(QrsDomain), C.c_int32, C.c_int32,
                                        C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p])
    h._check(f(h.h, C.byref(psd), C.byref(dom), int(n_rho), int(n_theta), int(fold), geom.data_ptr(), int(n),
               out.data_ptr(), _stream(stream)))
    return out


def _opt_prior(prior, n, n_cells):
    if prior is None:
        return None
    _check_dev(prior, torch.float32, "prior")
    if prior.numel() != n * n_cells:
        raise ValueError("prior must hold n * n_cells values")
    return prior.data_ptr()


TARGET = {"mean": 0, "rms": 1}


def qrs_proposal_targets(h: Handle, p, n_rho, n_theta, seed, n_f, n_draws, geom, kind="rms", fold=0, out=None,
                         stream=None):
    """Per-cell training targets [n][n_rho n_theta] from plain draws (geom: device float64 [n][5]);
    fold 1, 2, 4: cells of each geometry's baseline frame over `fold` mirrored sectors."""
    _check_dev(geom, torch.float64, "geom")
    n = geom.shape[0]
    if out is None:
        out = torch.empty(n, n_rho * n_theta, dtype=torch.float32, device=geom.device)
    psd, dom, _ = _structs(p)
    f = _prop_fn("qrs_proposal_targets", [C.c_void_p, C.POINTER(QrsPsd), C.POINTER(QrsDomain), C.c_int32, C.c_int32,
                                          C.c_uint64, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                          C.c_int64, C.c_void_p, C.c_void_p])
    h._check(f(h.h, C.byref(psd), C.byref(dom), int(n_rho), int(n_theta), int(seed) & (2**64 - 1), int(n_f),
               int(n_draws), TARGET[kind], int(fold), geom.data_ptr(), int(n), out.data_ptr(), _stream(stream)))
    return out


def qrs_mlp_forward(h: Handle, n_cells, params, geom, out=None, stream=None, prior=None):
    """Logits [n][n_cells] = MLP(geom) (+ prior [n][n_cells] when given)."""
    _check_dev(params, torch.float32, "params")
    _check_dev(geom, torch.float64, "geom")
    n = geom.shape[0]
    if out is None:
        out = torch.empty(n, n_cells, dtype=torch.float32, device=geom.device)
    f = _prop_fn("qrs_mlp_forward", [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                     C.c_void_p])
    h._check(f(h.h, int(n_cells), params.data_ptr(), geom.data_ptr(), _opt_prior(prior, n, n_cells), int(n),
               out.data_ptr(), _stream(stream)))
    return out


def qrs_mlp_loss_grad(h: Handle, n_cells, params, geom, targets, grad=None, loss=None, stream=None, prior=None):
    _check_dev(params, torch.float32, "params")
    _check_dev(geom, torch.float64, "geom")
    _check_dev(targets, torch.float32, "targets")
    if grad is None:
        grad = torch.empty_like(params)
    if loss is None:
        loss = torch.empty(1, dtype=torch.float32, device=params.device)
    f = _prop_fn("qrs_mlp_loss_grad", [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p])
    n = int(geom.shape[0])
    h._check(f(h.h, int(n_cells), params.data_ptr(), geom.data_ptr(), _opt_prior(prior, n, n_cells), targets.data_ptr(),
               n, grad.data_ptr(), loss.data_ptr(), _stream(stream)))
    return grad, loss


def qrs_mlp_adam(h: Handle, n_cells, params, m, v, grad, lr, step, stream=None):
    f = _prop_fn("qrs_mlp_adam", [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_float,
                                  C.c_int64, C.c_void_p])
    h._check(f(h.h, int(n_cells), params.data_ptr(), m.data_ptr(), v.data_ptr(), grad.data_ptr(), float(lr), int(step),
               _stream(stream)))


def qrs_proposal_cdf(h: Handle, n_rho, n_theta, logits_row, eps=0.1, beta=1.0, out=None, stream=None):
    """Two-level sampling CDF (device int32 view of uint32 [n_rho + n_rho n_theta])
    from one row of logits [n_rho n_theta]: p = (1 - eps) softmax(beta z) + eps / C."""
    _check_dev(logits_row, torch.float32, "logits_row")
    if out is None:
        out = torch.empty(n_rho * (1 + n_theta), dtype=torch.int32, device=logits_row.device)
    f = _prop_fn("qrs_proposal_cdf", [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_float, C.c_float, C.c_void_p,
                                      C.c_void_p])
    h._check(f(h.h, int(n_rho), int(n_theta), logits_row.data_ptr(), float(eps), float(beta), out.data_ptr(),
               _stream(stream)))
    return out


class QrsMlpState(C.Structure):
    _fields_ = [("n_cells", C.c_int32), ("reserved", C.c_int32), ("step", C.c_int64), ("params", C.c_void_p),
                ("m", C.c_void_p), ("v", C.c_void_p)]


LR_SCHEDULE = {"constant": 0, "cosine": 1}


class ProposalState:
    """Resumable training state of the learned proposal: parameters, Adam
    moments (device tensors) and the step count; save() / load() go through
    libqrs's checkpoint file (qrs_mlp_save / qrs_mlp_load)."""

    def __init__(self, n_cells, params, m, v, step):
        self.n_cells, self.params, self.m, self.v, self.step = int(n_cells), params, m, v, int(step)

    def _c(self):
        for t, name in ((self.params, "params"), (self.m, "m"), (self.v, "v")):
            _check_dev(t, torch.float32, name)
        return QrsMlpState(self.n_cells, 0, self.step, self.params.data_ptr(), self.m.data_ptr(), self.v.data_ptr())

    def save(self, path, h: "Handle", stream=None):
        f = _prop_fn("qrs_mlp_save", [C.c_void_p, C.POINTER(QrsMlpState), C.c_char_p, C.c_void_p])
        st = self._c()
        h._check(f(h.h, C.byref(st), os.fsencode(str(path)), _stream(stream)))

    @staticmethod
    def load(path, h: "Handle", n_cells, stream=None):
        dev = torch.device("cuda", h.device)
        n = qrs_mlp_param_count(n_cells)
        s = ProposalState(n_cells, torch.empty(n, device=dev), torch.empty(n, device=dev), torch.empty(n, device=dev), 0)
        f = _prop_fn("qrs_mlp_load", [C.c_void_p, C.POINTER(QrsMlpState), C.c_char_p, C.c_void_p])
        st = s._c()
        h._check(f(h.h, C.byref(st), os.fsencode(str(path)), _stream(stream)))
        s.step = int(st.step)
        return s


def qrs_proposal_train(h: Handle, state: ProposalState, geom, targets, steps, lr, schedule="constant",
                       total_steps=None, loss_trace=None, stream=None, prior=None):
    """Full-batch Adam in libqrs (one call, include/qrs_proposal.h): advances
    `state` by `steps` steps; loss_trace (device float32 [steps]) receives
    each step's loss when given."""
    _check_dev(geom, torch.float64, "geom")
    _check_dev(targets, torch.float32, "targets")
    lt = None
    if loss_trace is not None:
        _check_dev(loss_trace, torch.float32, "loss_trace")
        if loss_trace.numel() < steps:
            raise ValueError("loss_trace must hold `steps` values")
        lt = loss_trace.data_ptr()
    total = int(total_steps) if total_steps is not None else state.step + int(steps)
    f = _prop_fn("qrs_proposal_train", [C.c_void_p, C.POINTER(QrsMlpState), C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_int64, C.c_int64, C.c_double, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p])
    st = state._c()
    n = int(geom.shape[0])
    h._check(f(h.h, C.byref(st), geom.data_ptr(), _opt_prior(prior, n, state.n_cells), targets.data_ptr(), n,
               int(steps), float(lr), LR_SCHEDULE[schedule], total, lt, _stream(stream)))
    state.step = int(st.step)
    return state


def train_proposal(h: Handle, n_cells, geom, targets, steps=2000, lr=2e-3, seed=0, params=None, stream=None,
                   log_every=0, state=None, return_state=False, schedule="constant", total_steps=None, prior=None,
                   out_scale=1.0):
    """Adam on the mean cross entropy, full batch, as one libqrs call
    (qrs_proposal_train).  schedule "cosine": step t of a run of total_steps
    (default: this call's last step) uses lr (1 + cos(pi (t - 1) /
    total_steps)) / 2.  Returns (params, list of (step, loss) every log_every
    steps), and the ProposalState after the last step when return_state is
    set; a `state` continues a checkpointed run (same result as an
    uninterrupted one when total_steps names the whole run)."""
    if schedule not in LR_SCHEDULE:
        raise ValueError("schedule must be 'constant' or 'cosine'")
    if state is not None:
        if state.n_cells != n_cells:
            raise ValueError("checkpoint has %d cells, not %d" % (state.n_cells, n_cells))
    else:
        if params is None:
            params = qrs_mlp_init(h, n_cells, seed, stream=stream, out_scale=out_scale)
        state = ProposalState(n_cells, params, torch.zeros_like(params), torch.zeros_like(params), 0)
    step0 = state.step
    trace = torch.empty(max(int(steps), 1), dtype=torch.float32, device=state.params.device) if log_every else None
    qrs_proposal_train(h, state, geom, targets, steps, lr, schedule=schedule,
                       total_steps=total_steps if total_steps is not None else step0 + steps, loss_trace=trace,
                       stream=stream, prior=prior)
    hist = []
    if log_every and steps > 0:
        tr = trace.cpu().numpy()
        hist = [(step0 + i + 1, float(tr[i])) for i in range(int(steps))
                if (step0 + i + 1) % log_every == 0 or step0 + i + 1 == 1]
    if return_state:
        return state.params, hist, state
    return state.params, hist
