"""K3 for N <= 8 as a nonzero list compiled for the context (nzlist.cu): the
coupling contraction of Eq. 1 with the nonzero entries of the reduced
coupling matrix written into the kernel, against the CPU FP64 oracle and
against the dense register kernel it replaces (GMMNLSE_NZ=0), which performs
the same operations in the same order with the zero entries included.

The graded-index Hermite-Gaussian couplings used here are 27-33% nonzero."""
import functools

import numpy as np
import pytest

import oracle as O
from paper_1708_05324_b300 import binding as B
from paper_1708_05324_b300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@functools.lru_cache(maxsize=None)
def case(N, fR, split_raman):
    prob = I.grin_problem("nz", N=N, Nt=512, dt=2e-12 / 512, kind="gaussian", fwhm=150e-15, energy=20e-9,
                          L=2e-3, dz=1e-4, M=5, tol=1e-13, seed=17, fR=fR, s_from="gh")
    if split_raman:
        # a separate (still fully symmetric) Raman tensor: the V = [U; h_R * U] form
        iso = np.zeros_like(prob.SK)
        for p in range(N):
            iso[p, p, p, p] = prob.SK[0, 0, 0, 0]
        prob.SR = 0.7 * prob.SK + 0.3 * iso
    ref, _ = O.mpa_propagate(O.Fiber.from_problem(prob), prob.A0, prob.L, prob.dz, prob.M, prob.tol)
    return prob, ref


def run(prob, precision, monkeypatch, nz):
    monkeypatch.setenv("GMMNLSE_NZ", nz)
    ctx = B.Context.from_problem(prob, precision=precision)
    try:
        out, st, rc = ctx.propagate(prob.A0, prob.L, prob.dz, prob.M, prob.tol, check=False)
    finally:
        ctx.close()
    assert rc == B.OK
    return out, st


@pytest.mark.parametrize("N", [1, 3, 6, 8])
@pytest.mark.parametrize("fR,split", [(0.0, False), (0.18, False), (0.18, True)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nonzero_list_contraction_matches_oracle_and_dense(N, fR, split, precision, monkeypatch):
    prob, ref = case(N, fR, split)
    nzl, st = run(prob, precision, monkeypatch, "require")  # the compiled kernel must be built
    dense, st_d = run(prob, precision, monkeypatch, "0")
    assert rel(nzl, ref) <= TOL[precision]
    # the same operations in the same order, minus the products with zeros
    assert rel(nzl, dense) <= (1e-14 if precision == "fp64" else 1e-7)
    if precision == "fp64":
        assert st["iters_total"] == st_d["iters_total"]
