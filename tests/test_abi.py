"""The C-ABI library: loads without a GPU, exports what include/gmmnlse.h
declares, matches the ctypes layouts, and validates arguments on the host."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1708_05324_b300 import binding as B
from paper_1708_05324_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gmmnlse.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gmmnlse_\w+)\s*\(", txt)))


def test_library_exports_every_declared_function(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(B.EXPORTS) == names


def test_struct_layouts_match_the_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r"""
#include <stdio.h>
#include <stddef.h>
#include "gmmnlse.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(gmmnlse_params), offsetof(gmmnlse_params, stream),
         offsetof(gmmnlse_params, io_device), sizeof(gmmnlse_stats), offsetof(gmmnlse_stats, eps_max),
         sizeof(gmmnlse_step), offsetof(gmmnlse_step, trials));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [C.sizeof(B.Params), B.Params.stream.offset, B.Params.io_device.offset,
            C.sizeof(B.Stats), B.Stats.eps_max.offset, C.sizeof(B.Step), B.Step.trials.offset]
    assert got == want


def test_strerror_and_status_codes(lib):
    assert lib.gmmnlse_strerror(0) == b"ok"
    assert b"converge" in lib.gmmnlse_strerror(B.E_NOT_CONVERGED)
    assert lib.gmmnlse_strerror(12345) == b"unknown status"


def _create(prm, beta, SK, SR=None, fR=0.0, hR=None):
    h = C.c_void_p()
    rc = B.load().gmmnlse_create(C.byref(prm), beta.ctypes.data, SK.ctypes.data,
                                 None if SR is None else SR.ctypes.data, fR,
                                 None if hR is None else hR.ctypes.data, C.byref(h))
    return rc, h


def test_create_validates_on_the_host_before_any_cuda_call():
    """These fail in argument checking, which runs before the device is
    touched, so they also pass on a machine without a GPU."""
    N, Nt = 2, 64
    beta = np.zeros((N, Nt))
    S = I.grin_S_gauss_hermite(I.grin_mode_indices(N), 6.4e-6)
    good = B.Params(N, Nt, 1e-15, 1030e-9, 2.3e-20, 1, B.FP64, 0, 0, 0, None, 0)
    bad_nt = B.Params(N, 48, 1e-15, 1030e-9, 2.3e-20, 1, B.FP64, 0, 0, 0, None, 0)
    assert _create(bad_nt, beta, S)[0] == B.E_INVALID
    zero_n = B.Params(0, Nt, 1e-15, 1030e-9, 2.3e-20, 1, B.FP64, 0, 0, 0, None, 0)
    assert _create(zero_n, beta, S)[0] == B.E_INVALID
    nan_beta = beta.copy()
    nan_beta[1, 3] = np.nan
    assert _create(good, nan_beta, S)[0] == B.E_INVALID
    # Raman on without a response
    assert _create(good, beta, S, fR=0.18)[0] == B.E_INVALID
    # a coupling tensor that is not symmetric in m <-> n (not from Eq. 2)
    asym = S.copy()
    asym[0, 0, 0, 1] += 0.1 * abs(S).max()
    assert _create(good, beta, asym)[0] == B.E_UNSUPPORTED


def test_propagate_and_server_reject_null_handles(lib):
    assert lib.gmmnlse_propagate(None, None, 1.0, 0.1, 5, 1e-8, None, None) == B.E_INVALID
    assert lib.gmmnlse_poll(None, 1, None, None) == B.E_INVALID
    h = C.c_void_p()
    assert lib.gmmnlse_server_create(0, 1, C.byref(h)) == B.E_INVALID
    assert lib.gmmnlse_destroy(None) == 0
    assert lib.gmmnlse_server_destroy(None) == 0


def test_choose_m_rejects_bad_arguments_before_any_cuda_call(lib):
    cand = (C.c_int * 2)(1, 5)
    best = C.c_int(0)
    buf = (C.c_double * 4)()
    assert lib.gmmnlse_choose_m(None, buf, 1e-4, 1e-8, cand, 2, 10, buf, None, C.byref(best)) == B.E_INVALID


def test_rk4ip_rejects_null_handles(lib):
    assert lib.gmmnlse_propagate_rk4ip(None, None, 1e-3, 1e-4, None, None) == B.E_INVALID


def test_set_linear_coupling_rejects_a_null_handle(lib):
    assert lib.gmmnlse_set_linear_coupling(None, None) == B.E_INVALID


def test_set_gain_rejects_a_null_handle(lib):
    assert lib.gmmnlse_set_gain(None, None) == B.E_INVALID


def test_overlap_tensor_validates_on_the_host(lib):
    F = np.ones(6)
    S = np.empty(16)
    assert lib.gmmnlse_overlap_tensor(0, None, 2, 3, 1e-12, S.ctypes.data) == B.E_INVALID
    assert lib.gmmnlse_overlap_tensor(0, F.ctypes.data, 0, 3, 1e-12, S.ctypes.data) == B.E_INVALID
    assert lib.gmmnlse_overlap_tensor(0, F.ctypes.data, 2, 3, -1.0, S.ctypes.data) == B.E_INVALID
