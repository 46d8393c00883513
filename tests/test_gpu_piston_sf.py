"""The plain differential-piston case at full size on the GPU (Sec. 4.4, Eq. 7).

Seventeen apertures of D = 1 m -- the origin and 16 baselines log-spaced from
1 to 100 m along x -- von Karman r0 = 0.10 m, L0 = 25 m, log-radial frequency
domain [1e-3, 10] cycles/m, N_f = 1024 terms per realisation, 10^4
realisations from seed 0, in one qrs_diff_piston launch (the launch the
benchmark times), followed by the FP64 sums of qrs_structure_fn.

Two checks:
* every pair difference against the FP64 oracle's, within 1e-5 of the pair's
  standard deviation (sigma^2 = sum_k F_k^2 (A_i^2 + A_j^2));
* the mean of Delta^2 per baseline within 3 Monte-Carlo standard errors of the
  expected structure function, 4 pi int f W(f) A(f)^2 (1 - J0(2 pi f B)) df
  over the sampled annulus (the Hankel form of Sec. 4.4's definition with the
  Eq. 7 filter), evaluated at the FP32 baseline the kernel sees.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2404_02978_gb300 as qrs
from oracle import analytic as an
from paper_2404_02978_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
TOL_FIELD = 1e-5


@pytest.fixture(scope="module")
def h():
    from paper_2404_02978_gb300 import build as B
    B.build()
    return qrs.Handle(0)


@pytest.fixture(scope="module")
def plain_case(h):
    cfg = wl.PISTON_PLAIN
    B, ap_xy, ap_D, ap_d, pairs = wl.piston_plain_apertures()
    p = wl.method_params(cfg)
    R, nf = cfg["n_real"], cfg["n_f"]
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    delta = torch.empty(R, pairs.shape[0], device="cuda")
    job = qrs.piston_job(p, nf, R, dev(ap_xy), dev(ap_D), dev(ap_d), dev(pairs), None, delta)
    qrs.qrs_diff_piston(h, [job])
    acc = qrs.qrs_structure_fn(h, delta.view(R, pairs.shape[0], 1), torch.zeros(1, dtype=torch.int32, device="cuda"))
    qrs.qrs_sync(h)
    return dict(cfg=cfg, B=B, ap_xy=ap_xy, ap_D=ap_D, ap_d=ap_d, pairs=pairs, p=p,
                delta=delta.cpu().numpy(), acc=acc.cpu().numpy()[:, 0, :])


def test_plain_piston_full_size_every_value_against_the_oracle(plain_case):
    c = plain_case
    cfg = c["cfg"]
    R, nf = cfg["n_real"], cfg["n_f"]
    _, ref = oracle.diff_piston(c["p"], nf, R, c["ap_xy"], c["ap_D"], c["ap_d"], c["pairs"])
    d = oracle.draw(c["p"], n_f=nf, n_real=R)
    f = np.hypot(d["f"][..., 0].astype(np.float64), d["f"][..., 1].astype(np.float64))
    A = an.airy(f.ravel(), 1.0).reshape(f.shape)
    sig = np.sqrt(2.0 * np.sum((d["F"] * A) ** 2, axis=1))  # two apertures of the same D
    got = c["delta"]
    assert np.isfinite(got).all()
    err = np.abs(got.astype(np.float64) - ref) / sig[:, None]
    print("plain piston, %d values: max err %.3g sigma, rms %.3g sigma"
          % (err.size, err.max(), np.sqrt(np.mean(err ** 2))))
    assert err.max() <= TOL_FIELD


def test_plain_piston_full_size_structure_function_within_3_sigma(plain_case):
    c = plain_case
    cfg = c["cfg"]
    a = c["acc"]
    assert np.all(a[:, 2] == cfg["n_real"])
    # the GPU's FP64 sums against numpy's of the same pair differences
    x = c["delta"].astype(np.float64)
    assert np.allclose(a[:, 0], np.sum(x ** 2, axis=0), rtol=1e-12, atol=0)
    assert np.allclose(a[:, 1], np.sum(x ** 4, axis=0), rtol=1e-12, atol=0)
    mean = a[:, 0] / a[:, 2]
    sem = np.sqrt((a[:, 1] / a[:, 2] - mean ** 2) / a[:, 2])
    ref = np.array([an.piston_sf(float(np.float32(b)), cfg["r0"], cfg["L0"], 1.0, 0.0, cfg["fmin"], cfg["fmax"])
                    for b in c["B"]])
    z = (mean - ref) / sem
    print("plain piston SF: z per baseline", np.round(z, 2))
    assert np.all(np.abs(z) < 3.0), z
    # the long-baseline limit: twice the piston variance of one aperture
    var = an.piston_variance(cfg["r0"], cfg["L0"], 1.0, 0.0, cfg["fmin"], cfg["fmax"])
    assert ref[-1] == pytest.approx(2 * var, rel=1e-3)
