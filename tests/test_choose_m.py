"""gmmnlse_choose_m: the measured choice of substeps per long step (Sec. III.D,
the speed-up of the MPA as a function of M), on the GPU against the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1708_05324_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _problem():
    return I.grin_problem("choose_m", N=3, Nt=1024, dt=5e-12 / 1024, kind="sech", fwhm=100e-15,
                          energy=10e-9, L=2e-3, dz=1e-4, M=10, tol=1e-12, seed=11, fR=0.18, s_from="gh")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_choose_m_times_every_candidate_and_its_choice_propagates_to_the_oracle(precision):
    import torch
    from paper_1708_05324_b300 import binding as B
    assert torch.cuda.is_available()
    prob = _problem()
    ctx = B.Context.from_problem(prob, precision=precision, device=0)
    try:
        a0 = prob.A0.copy()
        cand = [1, 2, 5, 10, 20]
        best, sec = ctx.choose_m(a0, prob.dz, prob.tol, cand, trial_substeps=20)
        assert np.array_equal(a0, prob.A0)  # the starting field is not touched
        assert best in cand and set(sec) == set(cand)
        assert all(np.isfinite(t) and t > 0 for t in sec.values())
        assert sec[best] == min(sec.values())
        # one substep per fixed-point solve is far slower than ten at once
        assert sec[1] > 2.0 * sec[10]
        tol = 1e-10 if precision == "fp64" else 1e-5
        out, st, rc = ctx.propagate(prob.A0, prob.L, prob.dz, best, prob.tol)
        assert rc == B.OK
        ref, _ = O.mpa_propagate(O.Fiber.from_problem(prob), prob.A0, prob.L, prob.dz, best, prob.tol)
        assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < tol
        # every M reaches the same field (the implicit trapezoid substep after substep)
        out1, _, rc1 = ctx.propagate(prob.A0, prob.L, prob.dz, 1, prob.tol)
        assert rc1 == B.OK
        assert np.linalg.norm(out - out1) / np.linalg.norm(out1) < tol
    finally:
        ctx.close()


def test_choose_m_with_device_buffers_and_bad_candidates():
    import torch
    from paper_1708_05324_b300 import binding as B
    prob = _problem()
    ctx = B.Context.from_problem(prob, precision="fp32", device=0, io_device=True)
    try:
        a0 = torch.from_numpy(prob.A0).to("cuda:0")
        keep = a0.clone()
        best, sec = ctx.choose_m(a0, prob.dz, prob.tol, [4, 8], trial_substeps=16)
        assert best in (4, 8) and torch.equal(a0, keep)
        with pytest.raises(B.GmmnlseError):
            ctx.choose_m(a0, prob.dz, prob.tol, [0, 8], trial_substeps=16)
        with pytest.raises(B.GmmnlseError):
            ctx.choose_m(a0, prob.dz, prob.tol, [65], trial_substeps=16)
        bad = a0.clone()
        bad[0, 0] = float("nan")
        with pytest.raises(B.GmmnlseError):
            ctx.choose_m(bad, prob.dz, prob.tol, [4, 8], trial_substeps=16)
    finally:
        ctx.close()
