"""A bounded wait of the tensor-core GEMM that runs out (the failure path of
its mbarrier waits, tested without any GPU fault).

The test hook GMMNLSE_TC_STALL=1 (read when the context is created) makes the
MMA issuer of every single-CTA tensor-core GEMM wait on a barrier that nothing
completes; GMMNLSE_TC_WAIT_MS shortens the limit of every wait.  The wait must
run out, every role of the kernel stop, the kernel return, and the call report
GMMNLSE_E_CUDA with the tensor-core text; a context made afterwards on the same
device still propagates correctly.
"""
import time

import numpy as np
import pytest

import oracle as O
from paper_1708_05324_b300 import binding as B
from paper_1708_05324_b300 import inputs as I

pytestmark = pytest.mark.gpu


def low_rank_nine_modes():
    """Nine modes whose overlap tensor comes from ten grid cells: the pair
    matrix is a Gram matrix of rank <= 10, so the first GEMM of the low-rank
    coupling has one row block of 16 rows and runs on single CTAs."""
    prob = I.grin_problem("stall", N=9, Nt=256, dt=2e-12 / 256, kind="gaussian", fwhm=150e-15,
                          energy=20e-9, L=2e-4, dz=1e-4, M=2, tol=1e-12, seed=5, fR=0.18, s_from="gh")
    N = 9
    F = I.SplitMix64(77).normals(N * 10).reshape(N, 10)
    S = I.overlap_tensor_from_profiles(F, 1e-10)
    # exactly symmetric (as Eq. 2 makes it): the pair matrix made symmetric,
    # then spread over every index order
    pairs = [(m, n) for m in range(N) for n in range(m, N)]
    G = np.array([[S[p, l, m, n] for (m, n) in pairs] for (p, l) in pairs])
    G = (G + G.T) / 2
    row = {}
    for i, (m, n) in enumerate(pairs):
        row[(m, n)] = row[(n, m)] = i
    idx = np.array([[row[(a, b)] for b in range(N)] for a in range(N)])
    prob.SK = prob.SR = G[idx[:, :, None, None], idx[None, None, :, :]]
    return prob


def test_stalled_wait_times_out_and_reports(monkeypatch):
    prob = low_rank_nine_modes()
    monkeypatch.setenv("GMMNLSE_TC_STALL", "1")
    monkeypatch.setenv("GMMNLSE_TC_WAIT_MS", "20")
    ctx = B.Context.from_problem(prob, precision="bf16", fixed_iters=2)
    t0 = time.perf_counter()
    _, st, rc = ctx.propagate(prob.A0, prob.L, prob.dz, prob.M, prob.tol, check=False)
    took = time.perf_counter() - t0
    ctx.close()
    assert st["coupling_rank"] <= 10
    assert rc == B.E_CUDA
    assert "tensor-core" in B.load().gmmnlse_last_error().decode()
    assert took < 30.0
    # the device is still usable: a new context without the hook is correct
    monkeypatch.delenv("GMMNLSE_TC_STALL")
    monkeypatch.delenv("GMMNLSE_TC_WAIT_MS")
    ctx = B.Context.from_problem(prob, precision="bf16", fixed_iters=2)
    out, st, rc = ctx.propagate(prob.A0, prob.L, prob.dz, prob.M, prob.tol, check=False)
    ctx.close()
    assert rc == B.OK
    ref, _ = O.mpa_propagate(O.Fiber.from_problem(prob), prob.A0, prob.L, prob.dz, prob.M, prob.tol,
                             fixed_iters=2)
    assert float(np.linalg.norm(out - ref) / np.linalg.norm(ref)) < 1e-5
