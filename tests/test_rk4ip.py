"""gmmnlse_propagate_rk4ip: the split-step comparator of the MPA (Sec. III.D,
Fig. 3) on the GPU, element by element against the oracle's RK4IP."""
import functools

import numpy as np
import pytest

import oracle as O
from paper_1708_05324_b300 import inputs as I

pytestmark = pytest.mark.gpu

L, H = 1e-3, 1e-4  # ten steps


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def small(N, Nt, fR, split_raman=False, ss=1):
    prob = I.grin_problem("rk4", N=N, Nt=Nt, dt=2e-12 / Nt, kind="gaussian", fwhm=150e-15, energy=20e-9,
                          L=L, dz=H, M=5, tol=1e-13, seed=13, fR=fR, self_steepening=ss, s_from="gh")
    if split_raman:
        iso = np.zeros_like(prob.SK)
        for p in range(N):
            iso[p, p, p, p] = prob.SK[0, 0, 0, 0]
        prob.SR = 0.7 * prob.SK + 0.3 * iso
    return prob


@functools.lru_cache(maxsize=None)
def case(N, Nt, fR, split_raman=False, ss=1):
    prob = small(N, Nt, fR, split_raman, ss)
    ref = O.rk4ip_propagate(O.Fiber.from_problem(prob), prob.A0, L, H)
    return prob, ref


CASES = [(1, 128, 0.18), (3, 256, 0.0), (3, 1024, 0.18), (6, 512, 0.18), (6, 8192, 0.18), (10, 256, 0.18),
         (15, 256, 0.18)]


@pytest.mark.parametrize("N,Nt,fR", CASES)
@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_rk4ip_matches_the_oracle(N, Nt, fR, precision, bar):
    from paper_1708_05324_b300 import binding as B
    prob, ref = case(N, Nt, fR)
    ctx = B.Context.from_problem(prob, precision=precision, device=0)
    try:
        out, st, rc = ctx.propagate_rk4ip(prob.A0, L, H)
    finally:
        ctx.close()
    assert rc == B.OK
    assert st["long_steps"] == 10 and st["iters_total"] == 40
    assert rel(out, ref) < bar


@pytest.mark.parametrize("N,Nt", [(10, 256), (15, 256)])
@pytest.mark.parametrize("mixed", ["bf16", "fp16"])
def test_rk4ip_on_the_tensor_core_contraction(N, Nt, mixed):
    from paper_1708_05324_b300 import binding as B
    prob, ref = case(N, Nt, 0.18)
    ctx = B.Context.from_problem(prob, precision=mixed, device=0)
    try:
        out, _, rc = ctx.propagate_rk4ip(prob.A0, L, H)
    finally:
        ctx.close()
    assert rc == B.OK
    assert rel(out, ref) < 1e-3
    assert rel(out, ref) < 1e-5  # hi/lo operands keep it FP32-like


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_rk4ip_with_a_separate_raman_tensor_and_no_self_steepening(precision, bar):
    from paper_1708_05324_b300 import binding as B
    prob, ref = case(6, 256, 0.18, True, 0)
    ctx = B.Context.from_problem(prob, precision=precision, device=0)
    try:
        out, _, rc = ctx.propagate_rk4ip(prob.A0, L, H)
    finally:
        ctx.close()
    assert rc == B.OK
    assert rel(out, ref) < bar


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mpa_after_rk4ip_on_one_context_still_matches_the_oracle(precision):
    """The comparator takes the context's phase tables for (h/2, 1); the next
    MPA call must rebuild its own."""
    from paper_1708_05324_b300 import binding as B
    prob, ref = case(3, 1024, 0.18)
    fib = O.Fiber.from_problem(prob)
    ref_mpa, _ = O.mpa_propagate(fib, prob.A0, L, H, 5, 1e-13)
    bar = 1e-10 if precision == "fp64" else 1e-5
    ctx = B.Context.from_problem(prob, precision=precision, device=0)
    try:
        a, _, rc = ctx.propagate(prob.A0, L, H, 5, 1e-13)
        assert rc == B.OK and rel(a, ref_mpa) < bar
        b, _, rc = ctx.propagate_rk4ip(prob.A0, L, H)
        assert rc == B.OK and rel(b, ref) < bar
        c, _, rc = ctx.propagate(prob.A0, L, H, 5, 1e-13)
        assert rc == B.OK and rel(c, ref_mpa) < bar
        # two integrators of Eq. 1 (fourth and second order in h) sit as far
        # apart on the GPU as in the oracle: their step errors, not rounding
        d = rel(ref, ref_mpa)
        assert d > 10 * bar
        assert abs(rel(b, a) - d) < 3 * bar
    finally:
        ctx.close()


def test_rk4ip_rejects_bad_input():
    from paper_1708_05324_b300 import binding as B
    prob = small(3, 256, 0.18)
    ctx = B.Context.from_problem(prob, precision="fp32", device=0)
    try:
        bad = prob.A0.copy()
        bad[1, 7] = np.nan
        assert ctx.propagate_rk4ip(bad, L, H, check=False)[2] == B.E_INVALID
        assert ctx.propagate_rk4ip(prob.A0, 1.05e-3, 1e-4, check=False)[2] == B.E_INVALID
        assert ctx.propagate_rk4ip(prob.A0, L, -1e-4, check=False)[2] == B.E_INVALID
    finally:
        ctx.close()
