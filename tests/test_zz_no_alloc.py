"""gmmnlse_propagate_noalloc: the propagation for callers that cannot let
the library allocate device memory (stream capture, latency-critical loops,
programs whose device memory belongs to their own pool).

Its output must equal that of gmmnlse_propagate on the same input, call
after call: the static scratch array keeps the previous call's contents, so
two consecutive calls also check that everything that must start from zero
is reset.  This file is collected last so that a first failure here comes
after every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1708_05324_b300 import binding as B
from paper_1708_05324_b300 import inputs as I

pytestmark = pytest.mark.gpu

BAR = {"fp64": 1e-10, "fp32": 1e-5}


def _problem(seed):
    return I.grin_problem("noalloc", N=3, Nt=1024, dt=2e-12 / 1024, kind="gaussian", fwhm=150e-15,
                          energy=20e-9, L=2.3e-3, dz=1e-4, M=5, tol=1e-12, seed=seed, fR=0.18, s_from="gh")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_propagate_on_consecutive_calls(precision):
    import torch
    lib = B.load()
    for seed in (21, 22):
        prob = _problem(seed)
        ctx = B.Context.from_problem(prob, precision=precision, io_device=True)
        a0 = torch.from_numpy(prob.A0).cuda()
        ref = torch.empty_like(a0)
        tol = prob.tol if precision == "fp64" else 1e-9
        _, st_ref, _ = ctx.propagate(a0, prob.L, prob.dz, prob.M, tol, out=ref)
        for _ in range(2):
            out = torch.full_like(a0, complex(float("nan"), float("nan")))
            st = B.Stats()
            rc = lib.gmmnlse_propagate_noalloc(ctx.handle, a0.data_ptr(), prob.L, prob.dz, prob.M, tol,
                                               out.data_ptr(), C.byref(st))
            torch.cuda.synchronize()
            assert rc == B.OK, lib.gmmnlse_last_error()
            r, o = ref.cpu().numpy(), out.cpu().numpy()
            assert np.linalg.norm(o - r) / np.linalg.norm(r) < BAR[precision]
            assert st.long_steps == st_ref["long_steps"] == 5
            assert st.energy_in == pytest.approx(st_ref["energy_in"], rel=1e-12)
        ctx.close()


def test_noalloc_rejects_a_workspace_beyond_the_static_array():
    import torch
    lib = B.load()
    prob = I.grin_problem("big", N=10, Nt=16384, dt=20e-12 / 16384, kind="gaussian", fwhm=500e-15,
                          energy=100e-9, L=2e-4, dz=1e-5, M=20, tol=1e-6, seed=3, fR=0.18, s_from="gh")
    ctx = B.Context.from_problem(prob, precision="fp32", io_device=True)
    a0 = torch.from_numpy(prob.A0).cuda()
    out = torch.empty_like(a0)
    rc = lib.gmmnlse_propagate_noalloc(ctx.handle, a0.data_ptr(), prob.L, prob.dz, prob.M, prob.tol,
                                       out.data_ptr(), None)
    assert rc == B.E_NOMEM
    assert b"32 MiB" in lib.gmmnlse_last_error()
    ctx.close()


def test_noalloc_rejects_fp64_2_14():
    """The no-alloc entry point has one-block transforms only: FP64 at 2^14 points is refused."""
    import torch
    lib = B.load()
    prob = I.grin_problem("big", N=2, Nt=16384, dt=20e-12 / 16384, kind="gaussian", fwhm=300e-15,
                          energy=50e-9, L=5e-5, dz=2.5e-5, M=2, tol=1e-10, seed=3, fR=0.18, s_from="gh")
    ctx = B.Context.from_problem(prob, precision="fp64", io_device=True)
    a0 = torch.from_numpy(prob.A0).cuda()
    out = torch.empty_like(a0)
    rc = lib.gmmnlse_propagate_noalloc(ctx.handle, a0.data_ptr(), prob.L, prob.dz, prob.M, prob.tol,
                                       out.data_ptr(), None)
    assert rc == B.E_UNSUPPORTED
    ctx.close()
