"""Error paths of the C ABI on the GPU, without faulting or hanging it.

* Host-side fault injection (QRS_FAULT read at qrs_create): "alloc" makes a
  workspace allocation fail with QRS_ERR_NOMEM, "launch" makes every compute
  call fail with QRS_ERR_CUDA before anything is launched; the handle stays
  usable, other handles are unaffected.
* Device-side index checks: a grid node index beyond n_points and a pair
  index beyond the values are not used; the device error word reports
  QRS_ERR_DEVICE_CHECK at the next qrs_sync, which clears it.
* Bounded waits: "timeout" makes the next tensor-core GEMM launch wait on an
  mbarrier that no thread arrives at, with a limit of about 1 ms; every CTA
  records QRS_ERR_TIMEOUT, lets its copies in flight land, frees its tensor
  memory and returns (no MMA has been issued).  The next call on the same
  handle runs normally and matches the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2404_02978_gb300 as qrs
from paper_2404_02978_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _pts(n=300):
    rng = np.random.default_rng(0)
    return torch.from_numpy(rng.uniform(-3, 3, size=(n, 2)).astype(np.float32)).cuda()


def test_injected_allocation_failure(monkeypatch):
    monkeypatch.setenv("QRS_FAULT", "alloc")
    h = qrs.Handle(0)
    p = qrs.params(seed=1)
    with pytest.raises(qrs.QrsError) as e:
        qrs.qrs_synthesize_points(h, p, 64, 4, _pts(), mode="gemm_3xtf32")
    assert e.value.status == -5 and "injected" in str(e.value)
    out = qrs.qrs_synthesize_points(h, p, 64, 4, _pts())  # the fused form needs no workspace
    qrs.qrs_sync(h)
    assert torch.isfinite(out).all()
    monkeypatch.delenv("QRS_FAULT")
    h2 = qrs.Handle(0)
    qrs.qrs_synthesize_points(h2, p, 64, 4, _pts(), mode="gemm_3xtf32")
    qrs.qrs_sync(h2)


def test_injected_launch_failure(monkeypatch):
    monkeypatch.setenv("QRS_FAULT", "launch")
    h = qrs.Handle(0)
    p = qrs.params(seed=2)
    before = h.launch_count()
    for call in (lambda: qrs.qrs_synthesize_points(h, p, 64, 2, _pts()),
                 lambda: qrs.qrs_draw(h, p, 64, 2),
                 lambda: qrs.qrs_structure_fn(h, torch.zeros(2, 1, 8, device="cuda"),
                                              torch.tensor([1], dtype=torch.int32, device="cuda"))):
        with pytest.raises(qrs.QrsError) as e:
            call()
        assert e.value.status == -2 and "injected launch failure" in str(e.value)
    assert h.launch_count() == before
    qrs.qrs_sync(h)  # nothing ran, nothing to report


@pytest.mark.parametrize("nx,ny", [(8, 8), (200, 40)])  # one x tile (single CTA) and two (CTA pair)
def test_grid_index_beyond_points_is_caught(nx, ny):
    h = qrs.Handle(0)
    x = torch.linspace(-1, 1, nx, device="cuda")
    y = torch.linspace(-1, 1, ny, device="cuda")
    P = nx * ny
    index = torch.arange(P, dtype=torch.int32, device="cuda").reshape(ny, nx)
    index[3, 5] = P + 1000  # beyond n_points
    out = torch.full((2, P), float("nan"), device="cuda")
    qrs.qrs_synthesize_grid(h, qrs.params(seed=3), 32, 2, x, y, index=index, n_points=P, out=out)
    with pytest.raises(qrs.QrsError) as e:
        qrs.qrs_sync(h)
    assert e.value.status == -6
    written = torch.isfinite(out)
    assert written.sum().item() == 2 * (P - 1) and not written[:, 3 * nx + 5].any()
    qrs.qrs_sync(h)  # cleared


@pytest.mark.parametrize("mode", ["gemm_3xtf32", "gemm_bf16x3"])
def test_injected_wait_timeout_then_normal_call(monkeypatch, mode):
    monkeypatch.setenv("QRS_FAULT", "timeout")
    h = qrs.Handle(0)
    monkeypatch.delenv("QRS_FAULT")
    xy_np = wl.pupil_grid(32, 8.0)[:300]
    xy = torch.from_numpy(xy_np).cuda()
    p = qrs.params(seed=5)
    n_f, R = 200, 20
    qrs.qrs_synthesize_points(h, p, n_f, R, xy, mode=mode)
    with pytest.raises(qrs.QrsError) as e:
        qrs.qrs_sync(h)
    assert e.value.status == -3
    qrs.qrs_sync(h)  # cleared
    # the same handle and context: a normal call against the oracle
    got = qrs.qrs_synthesize_points(h, p, n_f, R, xy, mode=mode)
    qrs.qrs_sync(h)
    op = oracle.params(seed=5)
    ref = oracle.synthesize_shared(op, n_f, R, xy_np)
    sig = np.sqrt(np.sum(oracle.draw(op, n_f=n_f, n_real=1)["F"] ** 2))
    tol = 1e-5 if mode == "gemm_3xtf32" else 5e-5
    assert np.abs(got.cpu().numpy().astype(np.float64) - ref).max() <= tol * sig
    # and the fused form on the same handle
    fu = qrs.qrs_synthesize_points(h, p, n_f, 2, xy)
    qrs.qrs_sync(h)
    assert torch.isfinite(fu).all()
