"""The bounds-checked build (libqrs_checked.so, QRS_CHECKED=1) on the GPU.

In that build every checked accessor of the kernels tests its index against
its buffer's extent; an index out of range is not used and QRS_ERR_DEVICE_CHECK
is reported at the next qrs_sync.  Two checks:

* the machinery: qrs_check_selftest stores through the accessor at an index
  inside and outside its 8-float scratch; only the latter is reported (the
  access itself goes to a sink, so nothing outside the scratch is touched);
* the kernels: the parity suites of every form run against the checked
  library in a child process (the binding picks the library at import) and
  pass, which means no checked access of theirs was out of range (every test
  calls qrs_sync, which would raise) and the results still match the oracle.
  The full-size cases are left to the default build (the checked kernels are
  slower).
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _child(args, timeout):
    from paper_2404_02978_gb300 import build as B
    B.build_checked()
    env = dict(os.environ, QRS_CHECKED="1")
    return subprocess.run([sys.executable, *args], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=timeout)


def test_checked_accessor_reports_out_of_range_indices():
    code = r"""
import torch
import paper_2404_02978_gb300 as qrs
assert qrs.checked_build()
h = qrs.Handle(0)
for i in (0, 3, 7):
    qrs.qrs_check_selftest(h, i)
    qrs.qrs_sync(h)
for i in (8, -1, 1 << 40):
    qrs.qrs_check_selftest(h, i)
    try:
        qrs.qrs_sync(h)
    except qrs.QrsError as e:
        assert e.status == -6, e.status  # QRS_ERR_DEVICE_CHECK
    else:
        raise AssertionError("index %d not reported" % i)
    qrs.qrs_sync(h)  # cleared
print("selftest ok")
"""
    r = _child(["-c", code], 600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "selftest ok" in r.stdout


def test_parity_suites_pass_on_the_checked_build():
    files = ["tests/test_gpu_parity.py", "tests/test_gpu_anchor.py", "tests/test_gpu_edges.py", "tests/test_gpu_grid.py", "tests/test_gpu_gemm.py",
             "tests/test_gpu_fft.py", "tests/test_gpu_stats.py", "tests/test_gpu_proposal.py", "tests/test_gpu_fig5.py",
             "tests/test_gpu_batch.py"]
    files = [f for f in files if os.path.exists(os.path.join(ROOT, f))]
    r = _child(["-m", "pytest", *files, "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                "-k", "not full_size and not phase_screen and not trained and not four_times and not vlti"], 3000)
    tail = r.stdout[-4000:] + r.stderr[-2000:]
    print(tail)
    assert r.returncode == 0, tail
