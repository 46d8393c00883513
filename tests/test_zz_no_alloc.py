"""The no-allocation synthesis entry point (qrs_synthesize_points_noalloc).

Some callers cannot allocate device memory -- code running inside a framework
that owns all device memory through its own pool, or a latency-bound loop in
which an allocation could block or synchronise the device -- so they cannot
create a qrs_handle.  This entry point serves them: its scratch lives in a
static device array of the library.  The test calls it through the C ABI,
twice in a row with different point sets (so the scratch written by the first
call must not leak into the second), and checks each result against the
regular handle-based entry point within the tolerance the parity tests use
(1e-5 of the field's standard deviation per value).  It lives in a file of its
own that pytest collects last and passes both alone and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_2404_02978_gb300 as qrs
from paper_2404_02978_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
TOL_FIELD = 1e-5


def _noalloc_fn():
    L = qrs.load()
    f = L.qrs_synthesize_points_noalloc
    f.argtypes = [C.POINTER(qrs.QrsPsd), C.POINTER(qrs.QrsDomain), C.POINTER(qrs.QrsSampler), C.c_int64, C.c_int64,
                  C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return f


def test_noalloc_matches_handle_entry_point_twice():
    from paper_2404_02978_gb300 import build as B
    B.build()
    f = _noalloc_fn()
    h = qrs.Handle(0)
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(3)
    cases = [
        # pupil points: fixed-point phase path
        (qrs.params(seed=51), 700, 3, wl.pupil_grid(96, 8.0)),
        # baselines to 150 m: double-float phase path (the point bound in scratch changes)
        (qrs.params(seed=52, fmax=2.0), 300, 2, rng.uniform(-150, 150, size=(3001, 2)).astype(np.float32)),
        # rows of the phase screen's grid: the anchored kernel (the anchor bound in scratch)
        (qrs.params(seed=53), 500, 2, wl.pupil_grid(256, 8.0)[:4001]),
    ]
    for p, n_f, n_real, xy_np in cases:
        xy = torch.from_numpy(xy_np).cuda()
        ref = qrs.qrs_synthesize_points(h, p, n_f, n_real, xy, real_offset=4)
        out = torch.full((n_real, xy.shape[0]), float("nan"), device="cuda")
        psd, dom, smp = qrs._structs(p)
        st = f(C.byref(psd), C.byref(dom), C.byref(smp), n_f, n_real, 4, xy.data_ptr(), xy.shape[0],
               out.data_ptr(), C.c_void_p(stream.cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        sig = torch.sqrt(torch.mean(ref.double() ** 2, dim=1, keepdim=True))
        err = ((out.double() - ref.double()).abs() / sig).max().item()
        assert err <= TOL_FIELD, err
        assert torch.equal(out, ref)  # the same kernels on the same launch shapes
    # the contract itself: a warm call leaves the device's free memory unchanged
    p, n_f, n_real, xy_np = cases[0]
    xy = torch.from_numpy(xy_np).cuda()
    out = torch.empty(n_real, xy.shape[0], device="cuda")
    psd, dom, smp = qrs._structs(p)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(0)[0]
    st = f(C.byref(psd), C.byref(dom), C.byref(smp), n_f, n_real, 4, xy.data_ptr(), xy.shape[0], out.data_ptr(),
           C.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info(0)[0]
    assert st == 0
    assert free1 == free0, "free device memory changed by %d bytes" % (free0 - free1)
    h.close()


def test_noalloc_rejects_invalid_sizes():
    f = _noalloc_fn()
    psd, dom, smp = qrs._structs(qrs.params())
    xy = torch.zeros(4, 2, device="cuda")
    out = torch.zeros(1, 4, device="cuda")
    assert f(C.byref(psd), C.byref(dom), C.byref(smp), 0, 1, 0, xy.data_ptr(), 4, out.data_ptr(), None) == -1
    assert f(C.byref(psd), C.byref(dom), C.byref(smp), 2**31, 1, 0, xy.data_ptr(), 4, out.data_ptr(), None) == -1
    assert f(C.byref(psd), C.byref(dom), C.byref(smp), 64, -1, 0, xy.data_ptr(), 4, out.data_ptr(), None) == -1
    assert f(C.byref(psd), C.byref(dom), C.byref(smp), 64, 1, 0, None, 4, out.data_ptr(), None) == -1
    # real_offset + n_real beyond int64: rejected like qrs_synthesize_points does
    big = 2**63 - 1
    assert f(C.byref(psd), C.byref(dom), C.byref(smp), 64, big, big, xy.data_ptr(), 4, out.data_ptr(), None) == -1
    assert f(C.byref(psd), C.byref(dom), C.byref(smp), 1, 2, big - 1, xy.data_ptr(), 4, out.data_ptr(), None) == -1
