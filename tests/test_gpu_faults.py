"""Error paths of the C ABI on the GPU, without faulting or hanging it.

* Host-side fault injection (QRS_FAULT read at qrs_create): "alloc" makes a
  workspace allocation fail with QRS_ERR_NOMEM, "launch" makes every compute
  call fail with QRS_ERR_CUDA before anything is launched; the handle stays
  usable, other handles are unaffected.
* Device-side index checks: a grid node index beyond n_points and a pair
  index beyond the values are not used; the device error word reports
  QRS_ERR_DEVICE_CHECK at the next qrs_sync, which clears it.
"""
import numpy as np
import pytest
import torch

import paper_2404_02978_gb300 as qrs

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


def test_grid_index_beyond_points_is_caught():
    h = qrs.Handle(0)
    x = torch.linspace(-1, 1, 8, device="cuda")
    index = torch.arange(64, dtype=torch.int32, device="cuda").reshape(8, 8)
    index[3, 5] = 1000  # beyond n_points = 64
    out = torch.full((2, 64), float("nan"), device="cuda")
    qrs.qrs_synthesize_grid(h, qrs.params(seed=3), 32, 2, x, x, index=index, n_points=64, out=out)
    with pytest.raises(qrs.QrsError) as e:
        qrs.qrs_sync(h)
    assert e.value.status == -6
    written = torch.isfinite(out)
    assert written.sum().item() == 2 * 63 and not written[:, 3 * 8 + 5].any()
    qrs.qrs_sync(h)  # cleared
