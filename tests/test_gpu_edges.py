"""Edge cases of every entry point on the GPU: empty inputs are no-ops that
launch nothing; out-of-range sizes are argument errors; the method's
degenerate cases have closed forms.

* N_f = 1: the field is F (a cos 2 pi f.x - b sin 2 pi f.x) of the one drawn
  term (from qrs_draw's export), at every point, fused and GEMM forms.
* The origin: chi(0) = sum_k F_k a_k (every phase is 0), from the export.
* One point, one realisation; ragged sizes are covered by the parity tests.
"""
import numpy as np
import pytest
import torch

import paper_2404_02978_gb300 as qrs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_2404_02978_gb300 import build as B
    B.build()
    return qrs.Handle(0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_empty_inputs_launch_nothing(h):
    p = qrs.params(seed=1)
    xy = torch.zeros(0, 2, device="cuda")
    x = torch.zeros(4, device="cuda")
    lags = torch.tensor([1], dtype=torch.int32, device="cuda")
    before = h.launch_count()
    qrs.qrs_synthesize_points(h, p, 64, 3, xy)                      # no points
    qrs.qrs_synthesize_points(h, p, 64, 0, _dev(np.zeros((5, 2), np.float32)))  # no realisations
    qrs.qrs_synthesize_points(h, p, 64, 0, _dev(np.zeros((5, 2), np.float32)), mode="gemm_3xtf32")
    qrs.qrs_synthesize_grid(h, p, 64, 0, x, x)
    qrs.qrs_synthesize_grid(h, p, 64, 2, torch.zeros(0, device="cuda"), x)
    qrs.qrs_draw(h, p, 64, 0)
    qrs.qrs_structure_fn(h, torch.zeros(0, 1, 8, device="cuda"), lags)
    qrs.qrs_pair_diff(h, torch.zeros(3, 5, device="cuda"), torch.zeros(0, 2, dtype=torch.int32, device="cuda"))
    qrs.qrs_diff_piston(h, [])
    assert h.launch_count() == before
    qrs.qrs_sync(h)


@pytest.mark.parametrize("call", ["n_f_zero", "n_f_huge", "negative_real", "negative_offset", "grid_too_wide",
                                  "stats_too_many", "lag_out_of_range", "fold_not_importance", "fold_three",
                                  "frame_not_finite"])
def test_size_limits_are_argument_errors(h, call):
    p = qrs.params(seed=2)
    xy = _dev(np.zeros((4, 2), np.float32))
    calls = {
        "n_f_zero": lambda: qrs.qrs_synthesize_points(h, p, 0, 1, xy),
        "n_f_huge": lambda: qrs.qrs_draw(h, p, 1 << 31, 1),
        "negative_real": lambda: qrs.qrs_synthesize_points(h, p, 16, -1, xy, out=torch.empty(1, 4, device="cuda")),
        "negative_offset": lambda: qrs.qrs_synthesize_points(h, p, 16, 1, xy, real_offset=-3),
        "grid_too_wide": lambda: qrs.qrs_synthesize_grid(h, p, 16, 1, torch.zeros((1 << 24) + 1, device="cuda"),
                                                        torch.zeros(1, device="cuda"),
                                                        out=torch.empty(1, device="cuda")),
        "stats_too_many": lambda: qrs.qrs_star_discrepancy(h, torch.zeros(1, 65537, 2, device="cuda")),
        "fold_not_importance": lambda: qrs.qrs_draw(h, qrs.params(seed=2, fold=4), 16, 1),
        "fold_three": lambda: qrs.qrs_draw(h, qrs.params(sampler="importance", n_rho=2, n_theta=2, fold=3,
                                                         cdf=torch.zeros(6, dtype=torch.int32, device="cuda")), 16, 1),
        "frame_not_finite": lambda: qrs.qrs_draw(h, qrs.params(sampler="importance", n_rho=2, n_theta=2,
                                                               frame=float("nan"),
                                                               cdf=torch.zeros(6, dtype=torch.int32, device="cuda")),
                                                 16, 1),
        "lag_out_of_range": None,
    }
    if call == "lag_out_of_range":  # a device-side check, reported by qrs_sync
        qrs.qrs_structure_fn(h, torch.zeros(2, 1, 8, device="cuda"), torch.tensor([8], dtype=torch.int32,
                                                                                 device="cuda"))
        with pytest.raises(qrs.QrsError) as e:
            qrs.qrs_sync(h)
        assert e.value.status == -6
        return
    with pytest.raises((qrs.QrsError, ValueError, RuntimeError)):
        calls[call]()


@pytest.mark.parametrize("mode", ["fused", "gemm_3xtf32"])
def test_single_term_closed_form(h, mode):
    """N_f = 1: chi_r(x) = F (a cos 2 pi f.x - b sin 2 pi f.x) of realisation
    r's single term; GEMM columns share realisation 0's frequency."""
    rng = np.random.default_rng(3)
    xy = rng.uniform(-3, 3, size=(257, 2)).astype(np.float32)
    p = qrs.params(seed=4, fmax=8.0)
    R = 5
    got = qrs.qrs_synthesize_points(h, p, 1, R, _dev(xy), mode=mode).cpu().numpy().astype(np.float64)
    d = qrs.qrs_draw(h, p, 1, R, outputs=("f_xy", "amp", "coef"))
    qrs.qrs_sync(h)
    f = d["f_xy"].cpu().numpy().astype(np.float64)[:, 0]
    F = d["amp"].cpu().numpy().astype(np.float64)[:, 0]
    ab = d["coef"].cpu().numpy().astype(np.float64)[:, 0]
    if mode == "gemm_3xtf32":  # shared frequency and amplitude of realisation 0, own coefficients
        f = np.repeat(f[:1], R, 0)
        F = np.repeat(F[:1], R, 0)
    ph = 2 * np.pi * (f[:, None, 0] * xy[None, :, 0] + f[:, None, 1] * xy[None, :, 1])
    ref = F[:, None] * (ab[:, None, 0] * np.cos(ph) - ab[:, None, 1] * np.sin(ph))
    assert np.allclose(got, ref, atol=2e-6 * np.abs(F).max(), rtol=0)


def test_field_at_origin_is_sum_of_weighted_a(h):
    """At x = 0 the Eq. 3 sum is sum_k F_k a_k.  The fused kernel evaluates
    each term as F amp cos 2 pi (f.x + u 2^-24) (the amplitude-phase form of
    Eq. 3, one cosine per term), so at the origin every term carries the
    hardware cosine's error at its offset angle, as it does at any other
    point: the tolerance is the field tolerance of the parity tests
    (1e-5 sigma; observed about 2e-6 sigma)."""
    p = qrs.params(seed=5)
    n_f, R = 3000, 4
    xy = _dev(np.zeros((3, 2), np.float32))
    got = qrs.qrs_synthesize_points(h, p, n_f, R, xy).cpu().numpy().astype(np.float64)
    d = qrs.qrs_draw(h, p, n_f, R, outputs=("amp", "coef"))
    qrs.qrs_sync(h)
    F = d["amp"].cpu().numpy().astype(np.float64)
    a = d["coef"].cpu().numpy().astype(np.float64)[..., 0]
    ref = np.sum(F * a, axis=1)
    sig = np.sqrt(np.sum(F ** 2, axis=1))
    assert np.all(np.abs(got - ref[:, None]) <= 1e-5 * sig[:, None])
