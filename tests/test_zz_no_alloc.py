"""gmmnlse_propagate_noalloc: the propagation for callers that cannot let
the library allocate device memory (latency-critical loops that cannot take
cudaMalloc's device-wide synchronisation, programs whose device memory all
belongs to their own pool allocator).

Its output must equal that of gmmnlse_propagate on the same input, call
after call: the static scratch array keeps the previous call's contents, so
two consecutive calls also check that everything that must start from zero
is reset.  The cases reach the register contraction (3 modes), the tiled
CUDA-core contraction (10 modes), the one-block 16384-point FP32 transforms
with the FP64 input / output transform in halves (1 mode), and a mixed-
precision context, which this entry point runs in FP32 on the CUDA cores.
This file is collected last so that a first failure here comes after every
other test has run.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1708_05324_b300 import binding as B
from paper_1708_05324_b300 import inputs as I

pytestmark = pytest.mark.gpu

# tolerance against gmmnlse_propagate: FP64 1e-10, FP32 1e-5; the mixed
# context's gmmnlse_propagate runs the low-rank tensor-core contraction, this
# entry point the dense FP32 one, so they meet at the FP32 bar
BAR = {"fp64": 1e-10, "fp32": 1e-5, "bf16": 1e-5}

CASES = [  # (precision, N, Nt, M, L)
    ("fp64", 3, 1024, 5, 2.3e-3),
    ("fp32", 3, 1024, 5, 2.3e-3),
    ("fp64", 10, 1024, 3, 1.1e-3),
    ("fp32", 10, 1024, 3, 1.1e-3),
    ("fp32", 1, 16384, 4, 1.0e-3),
    ("bf16", 10, 1024, 3, 1.1e-3),
]


def _problem(N, Nt, M, L, seed):
    return I.grin_problem("noalloc", N=N, Nt=Nt, dt=2e-12 / 1024, kind="gaussian", fwhm=150e-15,
                          energy=20e-9, L=L, dz=1e-4, M=M, tol=1e-12, seed=seed, fR=0.18, s_from="gh")


@pytest.mark.parametrize("precision,N,Nt,M,L", CASES)
def test_noalloc_matches_propagate_on_consecutive_calls(precision, N, Nt, M, L):
    import torch
    lib = B.load()
    for seed in (21, 22):
        prob = _problem(N, Nt, M, L, seed)
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
            assert st.long_steps == st_ref["long_steps"] == int(np.ceil(round(L / 1e-4) / M))
            assert st.energy_in == pytest.approx(st_ref["energy_in"], rel=1e-12)
            assert st.coupling_rank == N * (N + 1) // 2
        ctx.close()


def test_noalloc_rejects_host_pointers():
    import torch
    lib = B.load()
    prob = _problem(3, 1024, 5, 2.3e-3, 21)
    ctx = B.Context.from_problem(prob, precision="fp32", io_device=True)
    a0 = torch.from_numpy(prob.A0).cuda()
    out = torch.empty_like(a0)
    host_in = np.ascontiguousarray(prob.A0)
    host_out = np.empty_like(host_in)
    rc = lib.gmmnlse_propagate_noalloc(ctx.handle, host_in.ctypes.data, prob.L, prob.dz, prob.M, 1e-9,
                                       out.data_ptr(), None)
    assert rc == B.E_INVALID
    rc = lib.gmmnlse_propagate_noalloc(ctx.handle, a0.data_ptr(), prob.L, prob.dz, prob.M, 1e-9,
                                       host_out.ctypes.data, None)
    assert rc == B.E_INVALID
    assert b"device memory" in lib.gmmnlse_last_error()
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
