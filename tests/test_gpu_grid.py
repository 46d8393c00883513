"""GPU parity of the separable-grid form against the oracle.

On a tensor-product point set {x_i} x {y_j}, Eq. 3 factors into x-side and
y-side harmonics, and libqrs computes each realisation as one split-precision
tensor-core product.  The field is the same as the fused form's at those
points (realisation r from stream points (real_offset + r) N_f + k), so the
oracle is its plain Eq. 3 sum at the grid points.  Tolerance per value,
relative to the realisation's field standard deviation sigma_r
(sigma_r^2 = sum_k F_k^2): 3XTF32 1e-5, BF16X3 5e-5 (the measured error is
printed).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2404_02978_gb300 as qrs
from paper_2404_02978_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
TOL = {"gemm_3xtf32": 1e-5, "gemm_bf16x3": 5e-5}


@pytest.fixture(scope="module")
def h():
    from paper_2404_02978_gb300 import build as B
    B.build()
    return qrs.Handle(0)


def _sigma(p, n_f, n_real, off):
    d = oracle.draw(p, n_f=n_f, n_real=n_real, real_offset=off)
    return np.sqrt(np.sum(d["F"] ** 2, axis=1))


def _points(x, y):
    X, Y = np.meshgrid(x, y, indexing="xy")  # node (i, j) at row j, column i
    return np.stack([X.ravel(), Y.ravel()], -1).astype(np.float32)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _pupil_index(n, L):
    """Grid coordinates of wl.pupil_grid(n, L) and the node -> point map."""
    c = (np.arange(n, dtype=np.float64) + 0.5 - n / 2) * (L / n)
    X, Y = np.meshgrid(c, c, indexing="xy")
    inside = (X ** 2 + Y ** 2 <= (L / 2) ** 2).ravel()
    index = np.full(n * n, -1, np.int32)
    index[inside] = np.arange(int(inside.sum()), dtype=np.int32)
    return c.astype(np.float32), index.reshape(n, n)


CASES = {
    # fixed-point phase (fmax |x| <= 128); 2 x tiles and 2 y blocks, both
    # ragged; 1000 terms = 63 K chunks (ragged last segment and padded terms)
    "ragged-fixed": dict(x=(-3.9, 3.9, 200), y=(-3.7, 3.8, 300), p=dict(fmax=16.0), n_f=1000, n_real=3, off=5),
    # long coordinates: double-float phase path
    "wide-df": dict(x=(-40.0, 37.0, 130), y=(-21.0, 44.0, 70), p=dict(fmax=4.0), n_f=333, n_real=2, off=0),
    # square domain (Eq. 5), literal Eq. 3 coefficients
    "square-eq3": dict(x=(-2.0, 2.0, 129), y=(-2.5, 2.5, 257), p=dict(domain="square", fmax=4.0, coef="eq3"),
                       n_f=37 * 37, n_real=2, off=1),
    # a single node, a single term (one x tile: the single-CTA kernel)
    "one-node": dict(x=(0.3, 0.3, 1), y=(-1.1, -1.1, 1), p=dict(fmax=16.0), n_f=1, n_real=4, off=2),
    # three x tiles: the second CTA pair's odd CTA has no x tile of its own
    # (it still builds its half of the y rows); one ragged y block
    "odd-tiles": dict(x=(-3.0, 3.1, 300), y=(-2.0, 2.0, 100), p=dict(fmax=16.0), n_f=500, n_real=3, off=9),
}


@pytest.mark.parametrize("mode", ["gemm_3xtf32", "gemm_bf16x3"])
@pytest.mark.parametrize("case", list(CASES))
def test_grid_parity(h, mode, case):
    c = CASES[case]
    rng = np.random.default_rng(11)
    x = np.sort(rng.uniform(c["x"][0], c["x"][1], c["x"][2])).astype(np.float32)
    y = np.sort(rng.uniform(c["y"][0], c["y"][1], c["y"][2])).astype(np.float32)
    if c["x"][2] == 1:
        x, y = np.float32([c["x"][0]]), np.float32([c["y"][0]])
    p = oracle.params(seed=71, **c["p"])
    got = qrs.qrs_synthesize_grid(h, p, c["n_f"], c["n_real"], _dev(x), _dev(y), mode=mode, real_offset=c["off"])
    qrs.qrs_sync(h)
    assert got.shape == (c["n_real"], len(y), len(x))
    got = got.cpu().numpy().reshape(c["n_real"], -1).astype(np.float64)
    ref = oracle.synthesize(p, c["n_f"], c["n_real"], _points(x, y), real_offset=c["off"])
    sig = _sigma(p, c["n_f"], c["n_real"], c["off"])
    err = np.abs(got - ref) / sig[:, None]
    print("grid %s %s: max err %.3g sigma, rms %.3g sigma" % (mode, case, err.max(), np.sqrt(np.mean(err ** 2))))
    assert np.isfinite(got).all()
    assert err.max() <= TOL[mode]


@pytest.mark.parametrize("mode", ["gemm_3xtf32", "gemm_bf16x3"])
def test_grid_cta_pairs_and_single_ctas(h, monkeypatch, mode):
    """Grids of two or more x tiles run on CTA pairs (one MMA over two SMs);
    QRS_GRID_PAIR=0 at handle creation keeps every tile on its own CTA.  Both
    against the oracle at the same tolerance, and against each other."""
    monkeypatch.setenv("QRS_GRID_PAIR", "0")
    h1 = qrs.Handle(0)
    monkeypatch.delenv("QRS_GRID_PAIR")
    rng = np.random.default_rng(12)
    x = np.sort(rng.uniform(-3.0, 3.0, 390)).astype(np.float32)  # 4 x tiles, the last one ragged
    y = np.sort(rng.uniform(-2.5, 2.5, 520)).astype(np.float32)  # 3 y blocks, the last one ragged
    p = oracle.params(seed=74, fmax=16.0)
    n_f, R = 700, 2
    pair = qrs.qrs_synthesize_grid(h, p, n_f, R, _dev(x), _dev(y), mode=mode, real_offset=3)
    single = qrs.qrs_synthesize_grid(h1, p, n_f, R, _dev(x), _dev(y), mode=mode, real_offset=3)
    qrs.qrs_sync(h)
    qrs.qrs_sync(h1)
    sig = _sigma(p, n_f, R, 3)
    rows = rng.choice(len(y), 40, replace=False)
    pts = _points(x, y[rows])
    ref = oracle.synthesize(p, n_f, R, pts, real_offset=3)
    for name, got in (("pair", pair), ("single", single)):
        g = got[:, rows, :].cpu().numpy().reshape(R, -1).astype(np.float64)
        err = np.abs(g - ref) / sig[:, None]
        print("grid %s %s: max err %.3g sigma" % (mode, name, err.max()))
        assert err.max() <= TOL[mode], name
    d = (pair - single).abs().max().item()
    print("grid %s pair vs single: max |diff| %.3g (%s)" % (mode, d, "bit-identical" if d == 0 else "differ"))
    assert d <= 2 * TOL[mode] * sig.max()


def test_grid_pupil_index_equals_fused(h):
    """Masked output (the 48^2 pupil) in pupil-point order equals the fused
    form at the same points and the oracle."""
    c, index = _pupil_index(48, 8.0)
    xy = wl.pupil_grid(48, 8.0)
    assert index.max() + 1 == xy.shape[0]
    p = qrs.params(seed=72)
    out = torch.full((3, xy.shape[0]), float("nan"), device="cuda")
    qrs.qrs_synthesize_grid(h, p, 700, 3, _dev(c), _dev(c), index=_dev(index), n_points=xy.shape[0], out=out,
                            real_offset=4)
    fu = qrs.qrs_synthesize_points(h, p, 700, 3, _dev(xy), real_offset=4)
    qrs.qrs_sync(h)
    g, f = out.cpu().numpy().astype(np.float64), fu.cpu().numpy().astype(np.float64)
    op = oracle.params(seed=72)
    sig = _sigma(op, 700, 3, 4)
    ref = oracle.synthesize(op, 700, 3, xy, real_offset=4)
    assert np.all(np.abs(g - ref) <= 1e-5 * sig[:, None])
    assert np.all(np.abs(g - f) <= 2e-5 * sig[:, None])


def test_grid_slabs_and_offsets(h):
    """More realisations than one slab of draw records (N_f = 16384: 1024 per
    slab) and a nonzero offset: realisations on both sides of the slab
    boundary against the oracle; a split call equals one call."""
    x = np.linspace(-1.5, 1.5, 16).astype(np.float32)
    y = np.linspace(-1.0, 2.0, 8).astype(np.float32)
    p = qrs.params(seed=73)
    n_f, R, off = 16384, 1030, 7
    full = qrs.qrs_synthesize_grid(h, p, n_f, R, _dev(x), _dev(y), real_offset=off)
    tail = qrs.qrs_synthesize_grid(h, p, n_f, 10, _dev(x), _dev(y), real_offset=off + 1020)
    qrs.qrs_sync(h)
    op = oracle.params(seed=73)
    pts = _points(x, y)
    for r in (0, 1023, 1024, 1029):
        ref = oracle.synthesize(op, n_f, 1, pts, real_offset=off + r)
        sig = _sigma(op, n_f, 1, off + r)
        got = full[r].cpu().numpy().reshape(1, -1).astype(np.float64)
        assert np.all(np.abs(got - ref) <= 1e-5 * sig[:, None]), r
    assert torch.equal(full[1020:], tail)


def test_grid_phase_screen_full_size(h):
    """The 8 m / 256^2 pupil (51,468 points), N_f = 4096, 1000 realisations
    (2000 work items over the persistent grid): equal to the fused form
    everywhere, and 3 realisations x 300 sampled points against the oracle."""
    cfg = wl.PHASE_SCREEN
    c, index = _pupil_index(cfg["grid"], cfg["pupil"])
    xy = wl.pupil_grid(cfg["grid"], cfg["pupil"])
    p = wl.method_params(cfg)
    R = cfg["n_real"]
    g = qrs.qrs_synthesize_grid(h, p, cfg["n_f"], R, _dev(c), _dev(c), index=_dev(index), n_points=xy.shape[0])
    f = qrs.qrs_synthesize_points(h, p, cfg["n_f"], R, _dev(xy))
    qrs.qrs_sync(h)
    sig = _sigma(p, cfg["n_f"], R, 0)
    d = (g - f).abs().max(dim=1).values.cpu().numpy()
    print("grid vs fused, full size: max %.3g sigma" % (d / sig).max())
    assert np.all(d <= 2e-5 * sig)
    rng = np.random.default_rng(5)
    for r in (0, 517, 999):
        idx = rng.choice(xy.shape[0], 300, replace=False)
        ref = oracle.synthesize(p, cfg["n_f"], 1, xy[idx], real_offset=r)
        got = g[r, idx].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - ref[0]) <= 1e-5 * sig[r]), r


def test_grid_arguments(h):
    x = torch.zeros(4, device="cuda")
    p = qrs.params()
    with pytest.raises(qrs.QrsError):
        qrs.qrs_synthesize_grid(h, p, 16, 1, x, x, mode="fused")
    before = h.launch_count()
    qrs.qrs_synthesize_grid(h, p, 16, 0, x, x)  # no realisations: no launch
    assert h.launch_count() == before
