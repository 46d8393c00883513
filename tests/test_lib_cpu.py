"""CPU-side checks of the C ABI library (no GPU needed): it builds, loads, exports
every entry point include/*.h declares, the Python binding's ctypes layouts
match the C compiler's, and the synthetic workloads have the stated sizes."""
import ctypes as C
import glob
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(hdr).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\**(qrs_[A-Za-z0-9_]+)\s*\(", txt,
                             flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libqrs():
    from paper_2404_02978_gb300 import build as B
    path = B.build()
    return C.CDLL(path)


def test_library_exports_every_declared_symbol(libqrs):
    names = _declared()
    assert {"qrs_create", "qrs_draw", "qrs_synthesize_points", "qrs_diff_piston", "qrs_structure_fn"} <= names
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2404_02978_gb300", "libqrs.so")],
                         capture_output=True, text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = sorted(n for n in names if n not in exported)
    assert not missing, missing
    for n in names:
        getattr(libqrs, n)


def test_checked_build_exports_the_same_symbols(libqrs):
    """libqrs_checked.so (QRS_CHECKED=1) is the same library with its kernels'
    accesses bounds-checked: same exports; qrs_checked_build tells them apart
    (a host function, callable without a GPU); qrs_check_selftest refuses a
    null handle in both."""
    from paper_2404_02978_gb300 import build as B
    path = B.build_checked()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    missing = sorted(n for n in _declared() if n not in exported)
    assert not missing, missing
    checked = C.CDLL(path)
    for L, want in ((libqrs, 0), (checked, 1)):
        L.qrs_checked_build.restype = C.c_int32
        assert L.qrs_checked_build() == want
        L.qrs_check_selftest.argtypes = [C.c_void_p, C.c_int64, C.c_void_p]
        assert L.qrs_check_selftest(None, 0, None) == -1


def test_null_handle_is_rejected_without_a_device(libqrs):
    libqrs.qrs_sync.argtypes = [C.c_void_p, C.c_void_p]
    assert libqrs.qrs_sync(None, None) == -1
    libqrs.qrs_last_error.restype = C.c_char_p
    libqrs.qrs_last_error.argtypes = [C.c_void_p]
    assert libqrs.qrs_last_error(None) == b"null handle"


def test_ctypes_layouts_match_c(tmp_path):
    import paper_2404_02978_gb300 as qrs
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "qrs.h"
#include "qrs_proposal.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\\n", sizeof(qrs_psd), sizeof(qrs_domain), sizeof(qrs_sampler),
         sizeof(qrs_draw_out), sizeof(qrs_piston_job));
  printf("%zu %zu %zu %zu %zu %zu %zu\\n", offsetof(qrs_sampler, cell_cdf), offsetof(qrs_sampler, kind),
         offsetof(qrs_sampler, frame),
         offsetof(qrs_piston_job, n_f), offsetof(qrs_piston_job, ap_xy), offsetof(qrs_piston_job, n_ap),
         offsetof(qrs_piston_job, n_pairs));
  printf("%zu %zu %zu %zu\\n", sizeof(qrs_mlp_state), offsetof(qrs_mlp_state, step), offsetof(qrs_mlp_state, params),
         offsetof(qrs_mlp_state, v));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    sizes, offs, mlp = [list(map(int, l.split())) for l in subprocess.check_output([str(exe)]).decode().splitlines()]
    assert sizes == [C.sizeof(qrs.QrsPsd), C.sizeof(qrs.QrsDomain), C.sizeof(qrs.QrsSampler),
                     C.sizeof(qrs.QrsDrawOut), C.sizeof(qrs.QrsPistonJob)]
    assert offs == [qrs.QrsSampler.cell_cdf.offset, qrs.QrsSampler.kind.offset, qrs.QrsSampler.frame.offset,
                    qrs.QrsPistonJob.n_f.offset,
                    qrs.QrsPistonJob.ap_xy.offset, qrs.QrsPistonJob.n_ap.offset, qrs.QrsPistonJob.n_pairs.offset]
    assert mlp == [C.sizeof(qrs.QrsMlpState), qrs.QrsMlpState.step.offset, qrs.QrsMlpState.params.offset,
                   qrs.QrsMlpState.v.offset]


def test_workload_sizes():
    from paper_2404_02978_gb300 import workloads as wl
    assert wl.pupil_grid(256, 8.0).shape == (51468, 2)
    assert wl.pupil_grid(512, 16.0).shape == (205892, 2)
    B, xy, D, d, pairs = wl.piston_plain_apertures()
    assert xy.shape == (17, 2) and pairs.shape == (16, 2)
    assert B[0] == pytest.approx(1.0) and B[-1] == pytest.approx(100.0)
    inst = wl.batched_instances(50, seed=1)
    assert all(4 <= len(i["ap_D"]) <= 64 and 256 <= i["n_f"] <= 8192 for i in inst)
    assert all(np.max(np.hypot(*i["ap_xy"].T)) <= 100.0 for i in inst)


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2404_02978_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True) + \
            glob.glob(os.path.join(pkg, "csrc", "*")):
        txt = open(f, errors="ignore").read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, flags=re.M), f
        assert "qrs_oracle" not in txt and "liboracle" not in txt, f
