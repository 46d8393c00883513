"""Seeded synthetic workloads shaped like the paper's cases.

Input construction only (point sets, aperture layouts, parameter sets): none
of the method's arithmetic lives here, so the CUDA path and the CPU reference
can both be fed from it.

* Pupil grid: an n x n grid of cell centres over an L x L square,
  x_i = (i + 1/2 - n/2) L/n, keeping the centres inside the circle of
  diameter L (51,468 points for 256^2 over 8 m; 205,892 for 512^2 over 16 m).
* Plain differential piston: apertures at the origin and at 16 baselines
  log-spaced from 1 to 100 m along x, D = 1 m (pairs (0, j)).
* VLTI-like unit-telescope pair of the paper's Sec. 4.3 example.
* Batched interferometers: n_ap ~ U{4..64} apertures, D ~ U(1.8, 8) m, centres
  uniform by area in a disc of diameter 200 m, N_f ~ U{256..8192}, R = 256.
"""
from __future__ import annotations

import numpy as np


def pupil_grid(n: int = 256, L: float = 8.0) -> np.ndarray:
    c = (np.arange(n, dtype=np.float64) + 0.5 - n / 2) * (L / n)
    X, Y = np.meshgrid(c, c, indexing="xy")
    inside = X ** 2 + Y ** 2 <= (L / 2) ** 2
    return np.stack([X[inside], Y[inside]], -1).astype(np.float32)


def log_baselines(n: int = 16, bmin: float = 1.0, bmax: float = 100.0) -> np.ndarray:
    return bmin * (bmax / bmin) ** (np.arange(n) / (n - 1))


def piston_plain_apertures(n_base: int = 16, D: float = 1.0):
    B = log_baselines(n_base)
    xy = np.concatenate([[[0.0, 0.0]], np.stack([B, np.zeros(n_base)], -1)]).astype(np.float32)
    pairs = np.array([(0, j) for j in range(1, n_base + 1)], np.int32)
    return B, xy, np.full(n_base + 1, D, np.float32), np.zeros(n_base + 1, np.float32), pairs


def all_pairs(n_ap: int) -> np.ndarray:
    return np.array([(i, j) for i in range(n_ap) for j in range(i + 1, n_ap)], np.int32).reshape(-1, 2)


def batched_instances(n_inst: int = 1000, seed: int = 4, n_real: int = 256, nf_range=(256, 8192),
                      ap_range=(4, 64), D_range=(1.8, 8.0), disc_diameter: float = 200.0):
    """List of dicts: ap_xy, ap_D, ap_d, pairs, n_f, n_real, seed (per instance)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_inst):
        n_ap = int(rng.integers(ap_range[0], ap_range[1] + 1))
        rad = (disc_diameter / 2) * np.sqrt(rng.uniform(size=n_ap))
        th = rng.uniform(0, 2 * np.pi, size=n_ap)
        xy = np.stack([rad * np.cos(th), rad * np.sin(th)], -1).astype(np.float32)
        out.append(dict(ap_xy=xy, ap_D=rng.uniform(*D_range, size=n_ap).astype(np.float32),
                        ap_d=np.zeros(n_ap, np.float32), pairs=all_pairs(n_ap),
                        n_f=int(rng.integers(nf_range[0], nf_range[1] + 1)), n_real=n_real,
                        seed=1000 * seed + i))
    return out


# Parameter sets of the five benchmark cases (units: m, cycles/m).
PISTON_PLAIN = dict(psd="von_karman", r0=0.10, L0=25.0, domain="logpolar", fmin=1e-3, fmax=10.0,
                    sampler="r2", seed=0, coef="gauss", n_f=1024, n_real=10_000)
PHASE_SCREEN = dict(psd="von_karman", r0=0.15, L0=30.0, domain="logpolar", fmin=1e-3, fmax=16.0,
                    sampler="r2", seed=2, coef="gauss", n_f=4096, n_real=1000, grid=256, pupil=8.0)
GEMM_SCREEN = dict(psd="von_karman", r0=0.15, L0=30.0, domain="logpolar", fmin=1e-3, fmax=16.0,
                   sampler="r2", seed=3, coef="gauss", n_f=16384, n_real=256, grid=512, pupil=16.0,
                   r0_range=(0.08, 0.20), L0_range=(20.0, 50.0), batches=4)
BATCHED = dict(psd="von_karman", r0=0.10, L0=25.0, domain="logpolar", fmin=1e-3, fmax=10.0,
               sampler="r2", coef="gauss", n_inst=1000, seed=4)
VLTI_UT = dict(psd="von_karman", L0=22.0, domain="square", fmax=0.25, sampler="r2", N=44, D=8.0, d=1.1,
               baseline=56.5, wind=10.2, n_real=2000)


def method_params(cfg: dict) -> dict:
    """The method-parameter subset of a case, in the binding's vocabulary."""
    keys = ("psd", "r0", "L0", "domain", "fmin", "fmax", "sampler", "seed", "coef")
    d = {k: cfg[k] for k in keys if k in cfg}
    d.setdefault("n_rho", 64)
    d.setdefault("n_theta", 32)
    d.setdefault("s0", None)
    d.setdefault("cdf", None)
    return d
