"""Piston-PSD synthesis, pair differences and the Sec. 4.3-4.4 experiment on the GPU.

* The Eq. 7 aperture filter on the PSD: draws and syntheses (fused, shared-draw
  GEMM, separable grid) against the FP64 oracle, 1e-5 sigma per value (sigma^2
  = sum_k F_k^2 of the realisation, F carrying the filter); at aperture
  positions the filtered synthesis equals libqrs's own piston kernel.
* Pair differences: exact, and a bad index is caught on the device.
* The VLTI unit-telescope experiment of Sec. 4.3 (SQUARE domain, N = 44,
  delta_f = 0.25/22, D = 8 m, d = 1.1 m, B = 56.5 m, wind 10.2 m/s along the
  baseline, 1 ms sampling): the temporal structure function of the
  differential piston from synthesis -> pair differences -> FP64 lagged sums,
  against the expected value over the square (2-D quadrature), within the
  Monte-Carlo error across realisations; sampled series against the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2404_02978_gb300 as qrs
from oracle import analytic as an

pytestmark = pytest.mark.gpu
D1 = float(np.float32(1.1))  # the piston kernel takes FP32 diameters
VLTI = dict(r0=0.10, L0=22.0, D=8.0, d=D1, B=56.5, v=10.2, fmax=0.25, N=44)


@pytest.fixture(scope="module")
def h():
    from paper_2404_02978_gb300 import build as B
    B.build()
    return qrs.Handle(0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _sigma(p, n_f, n_real, off):
    d = oracle.draw(p, n_f=n_f, n_real=n_real, real_offset=off)
    return np.sqrt(np.sum(d["F"] ** 2, axis=1))


def _vlti_params(seed):
    return oracle.params(seed=seed, r0=VLTI["r0"], L0=VLTI["L0"], domain="square", fmax=VLTI["fmax"],
                         ap_D=VLTI["D"], ap_d=VLTI["d"])


DOMS = {"logpolar": dict(domain="logpolar", fmin=1e-3, fmax=10.0), "square": dict(domain="square", fmax=0.25)}


@pytest.mark.parametrize("dom", list(DOMS))
def test_filtered_draw_parity(h, dom):
    p = oracle.params(seed=31, r0=0.1, L0=22.0, ap_D=8.0, ap_d=D1, **DOMS[dom])
    n_f = 1936 if dom == "square" else 1024
    got = qrs.qrs_draw(h, p, n_f, 3, real_offset=4, outputs=("f_xy", "amp"))
    ref = oracle.draw(p, n_f=n_f, n_real=3, real_offset=4)
    F0 = oracle.draw(dict(p, ap_D=0.0, ap_d=0.0), n_f=n_f, n_real=3, real_offset=4)["F"]
    assert np.array_equal(got["f_xy"].cpu().numpy(), ref["f"])
    # the filter in FP32 (Taylor series / large-argument form) against FP64, relative to the
    # unfiltered amplitude: |A_gpu - A| <= 5e-7
    assert np.all(np.abs(got["amp"].cpu().numpy() - ref["F"]) <= 5e-7 * F0)


@pytest.mark.parametrize("mode", ["fused", "gemm_3xtf32", "grid"])
@pytest.mark.parametrize("dom", list(DOMS))
def test_filtered_synthesis_parity(h, mode, dom):
    rng = np.random.default_rng(32)
    p = oracle.params(seed=33, r0=0.1, L0=22.0, ap_D=8.0, ap_d=D1, **DOMS[dom])
    n_f, R, off = (1936 if dom == "square" else 1000), 3, 2
    if mode == "grid":
        x = np.sort(rng.uniform(-60, 60, 150)).astype(np.float32)
        y = np.sort(rng.uniform(-20, 20, 40)).astype(np.float32)
        got = qrs.qrs_synthesize_grid(h, p, n_f, R, _dev(x), _dev(y), real_offset=off)
        X, Y = np.meshgrid(x, y, indexing="xy")
        xy = np.stack([X.ravel(), Y.ravel()], -1).astype(np.float32)
        ref = oracle.synthesize(p, n_f, R, xy, real_offset=off)
        sig = _sigma(p, n_f, R, off)
    elif mode == "fused":
        xy = rng.uniform(-60, 60, size=(700, 2)).astype(np.float32)
        got = qrs.qrs_synthesize_points(h, p, n_f, R, _dev(xy), real_offset=off)
        ref = oracle.synthesize(p, n_f, R, xy, real_offset=off)
        sig = _sigma(p, n_f, R, off)
    else:
        xy = rng.uniform(-60, 60, size=(300, 2)).astype(np.float32)
        got = qrs.qrs_synthesize_points(h, p, n_f, R, _dev(xy), mode=mode, real_offset=off)
        ref = oracle.synthesize_shared(p, n_f, R, xy, real_offset=off)
        sig = np.full(R, _sigma(p, n_f, 1, off)[0])
    qrs.qrs_sync(h)
    g = got.cpu().numpy().reshape(R, -1).astype(np.float64)
    err = np.abs(g - ref) / sig[:, None]
    print("filtered %s %s: max err %.3g sigma" % (mode, dom, err.max()))
    assert np.isfinite(g).all() and err.max() <= 1e-5


def test_filtered_synthesis_equals_piston_kernel(h):
    rng = np.random.default_rng(34)
    ap = rng.uniform(-100, 100, size=(20, 2)).astype(np.float32)
    p_plain = qrs.params(seed=35, r0=0.1, L0=22.0, fmax=10.0)
    chi = qrs.qrs_synthesize_points(h, dict(p_plain, ap_D=8.0, ap_d=D1), 1024, 5, _dev(ap), real_offset=3)
    pis = torch.empty(5, 20, device="cuda")
    job = qrs.piston_job(p_plain, 1024, 5, _dev(ap), _dev(np.full(20, 8.0, np.float32)),
                         _dev(np.full(20, D1, np.float32)), None, pis, None, real_offset=3)
    qrs.qrs_diff_piston(h, [job])
    qrs.qrs_sync(h)
    sig = _sigma(dict(p_plain, ap_D=8.0, ap_d=D1), 1024, 5, 3)
    assert np.all(np.abs(chi.cpu().numpy() - pis.cpu().numpy()) <= 2e-5 * sig[:, None])
    with pytest.raises(qrs.QrsError):  # a piston job must not filter twice
        qrs.qrs_diff_piston(h, [qrs.piston_job(dict(p_plain, ap_D=8.0), 64, 1, _dev(ap), _dev(np.full(20, 8.0, np.float32)),
                                               None, None, pis, None)])


def test_pair_diff_exact_and_checked(h):
    v = torch.randn(7, 50, device="cuda")
    pairs = torch.tensor([[0, 1], [49, 3], [5, 5], [10, 20]], dtype=torch.int32, device="cuda")
    out = qrs.qrs_pair_diff(h, v, pairs)
    qrs.qrs_sync(h)
    assert torch.equal(out, v[:, pairs[:, 0].long()] - v[:, pairs[:, 1].long()])
    bad = torch.tensor([[0, 1], [50, 2]], dtype=torch.int32, device="cuda")
    o2 = qrs.qrs_pair_diff(h, v, bad)
    with pytest.raises(qrs.QrsError) as e:
        qrs.qrs_sync(h)
    assert e.value.status == -6
    assert torch.isnan(o2[:, 1]).all() and torch.equal(o2[:, 0], v[:, 0] - v[:, 1])
    qrs.qrs_sync(h)  # the error word was cleared


def vlti_series(h, R, M, dt, seed, real_offset=0):
    """Differential-piston series [R, M] of the VLTI pair: synthesis of the
    piston field (Eq. 7 PSD) at both telescopes' tracks, then pair differences."""
    v, B = VLTI["v"], VLTI["B"]
    t = np.arange(M) * dt
    xy = np.concatenate([np.stack([-v * t, 0 * t], -1), np.stack([B - v * t, 0 * t], -1)]).astype(np.float32)
    pairs = np.stack([np.arange(M), M + np.arange(M)], -1).astype(np.int32)
    p = _vlti_params(seed)
    chi = qrs.qrs_synthesize_points(h, p, VLTI["N"] ** 2, R, _dev(xy), real_offset=real_offset)
    return qrs.qrs_pair_diff(h, chi, _dev(pairs)), xy, p


def test_vlti_temporal_structure_function(h):
    R, M, dt = 500, 1024, 1e-3
    delta, xy, p = vlti_series(h, R, M, dt, seed=36)
    lags = np.array([1, 2, 5, 10, 20, 50, 100, 200, 500, 1000], np.int32)
    acc = qrs.qrs_structure_fn(h, delta.reshape(1, R, M), _dev(lags))  # one series per realisation
    qrs.qrs_sync(h)
    a = acc.cpu().numpy()
    per = a[:, :, 0] / a[:, :, 2]  # [R][lags]: the SF of each realisation
    mean, sem = per.mean(0), per.std(0, ddof=1) / np.sqrt(R)
    ref = an.square_temporal_piston_sf(lags * dt, VLTI["B"], VLTI["v"], VLTI["r0"], VLTI["L0"], VLTI["D"],
                                       VLTI["d"], VLTI["fmax"])
    z = (mean - ref) / sem
    print("VLTI temporal SF: z =", np.round(z, 2))
    assert np.all(np.abs(z) < 4)
    # sampled series against the oracle
    d_np = delta.cpu().numpy()
    for r in (0, 377):
        idx = np.arange(0, M, 97)
        chi = oracle.synthesize(p, VLTI["N"] ** 2, 1, np.concatenate([xy[idx], xy[M + idx]]), real_offset=r)
        ref_d = chi[0, :idx.size] - chi[0, idx.size:]
        sig = _sigma(p, VLTI["N"] ** 2, 1, r)[0] * np.sqrt(2)
        assert np.all(np.abs(d_np[r, idx] - ref_d) <= 1e-5 * sig)
