"""Statistical acceptance of the tensor-core grid form at full size.

1000 phase screens of the 256^2 grid over 8 m (von Karman r0 = 0.15 m,
L0 = 30 m, N_f = 4096 log-polar R2 terms over [1e-3, 16] c/m, the phase-screen
workload) in each split precision; the structure function along x at 0.25, 1
and 4 m, one sample per realisation (the mean over its rows and positions),
against the annulus integral 4 pi int f W(f) (1 - J0(2 pi f r)) df over the
sampled band (Sec. 4.4; the draw is unbiased for it) within 3 standard
errors of the Monte Carlo.  The inputs are seeded, so the z values are fixed.
"""
import numpy as np
import pytest
import torch

import paper_2404_02978_gb300 as qrs
from oracle import analytic as an
from paper_2404_02978_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["gemm_3xtf32", "gemm_bf16x3"])
def test_grid_screens_structure_function(mode):
    h = qrs.Handle(0)
    cfg = wl.PHASE_SCREEN
    n, L, R = cfg["grid"], cfg["pupil"], cfg["n_real"]
    dx = L / n
    c = torch.from_numpy(((np.arange(n) + 0.5 - n / 2) * dx).astype(np.float32)).cuda()
    p = wl.method_params(dict(cfg, seed=31))
    out = qrs.qrs_synthesize_grid(h, p, cfg["n_f"], R, c, c, mode=mode)  # [R][n][n], x fastest
    lags = np.array([8, 32, 128], np.int32)
    acc = qrs.qrs_structure_fn(h, out.reshape(1, R * n, n), torch.from_numpy(lags).cuda())
    qrs.qrs_sync(h)
    a = acc.cpu().numpy().reshape(R, n, len(lags), 3)
    per_real = a[..., 0].sum(1) / a[..., 2].sum(1)  # [R][lags]: each realisation's mean squared difference
    mean = per_real.mean(0)
    sem = per_real.std(0, ddof=1) / np.sqrt(R)
    for li, lag in enumerate(lags):
        r = float(lag * dx)
        expect = an.phase_sf(r, p["r0"], p["L0"], 1e-3, 16.0)
        z = (mean[li] - expect) / sem[li]
        print("%s r=%.2f m: SF %.4f rad^2, annulus %.4f, z %.2f" % (mode, r, mean[li], expect, z))
        assert abs(z) < 3.0, (mode, r, z)
