"""gmmnlse_choose_step: the substep dz and long step M from the length scales
of Sec. III.D (L_long = M dz << z_NL, dz << z_IM), refined to an accuracy
target by step doubling."""
import numpy as np
import pytest

import oracle as O
from paper_1708_05324_b300 import binding as B
from paper_1708_05324_b300 import inputs as I

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def fiber():
    return I.grin_problem("cs", N=6, Nt=512, dt=2e-12 / 512, kind="gaussian", fwhm=150e-15, energy=20e-9,
                          L=1e-2, dz=1e-4, M=5, tol=1e-12, seed=9, fR=0.18, s_from="gh")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_length_scales_match_the_oracle_and_the_rule(precision):
    prob = fiber()
    ctx = B.Context.from_problem(prob, precision=precision)
    try:
        ch = ctx.choose_step(prob.A0, prob.L, 0.0, 1e-12)
    finally:
        ctx.close()
    z_nl, z_im = O.length_scales(O.Fiber.from_problem(prob), prob.A0)
    assert ch["z_nl"] == pytest.approx(z_nl, rel=1e-12)
    assert ch["z_im"] == pytest.approx(z_im, rel=1e-12)
    assert ch["trials"] == 0
    # the rule, then L divided by a whole number
    dz = min(z_nl / 200, z_im / 10)
    n = int(np.ceil(prob.L / dz - 1e-9))
    assert ch["dz"] == pytest.approx(prob.L / n, rel=1e-12)
    assert ch["M"] == max(1, min(64, n, int(np.floor(z_nl / (10 * ch["dz"])))))
    assert ch["M"] * ch["dz"] <= z_nl / 10 * (1 + 1e-12)


def test_accuracy_target_is_met():
    """With rtol the chosen dz must give a field within about rtol of the
    converged (fine-step) one; a looser rtol gives a coarser dz."""
    prob = fiber()
    ctx = B.Context.from_problem(prob, precision="fp64")
    try:
        tight = ctx.choose_step(prob.A0, prob.L, 1e-6, 1e-12)
        loose = ctx.choose_step(prob.A0, prob.L, 1e-4, 1e-12)
        assert tight["trials"] >= 2 and tight["err_est"] <= 1e-6 * 1.001
        assert tight["dz"] < loose["dz"]
        out, _, rc = ctx.propagate(prob.A0, prob.L, tight["dz"], tight["M"], 1e-12)
        assert rc == B.OK
        # reference: the same scheme at a quarter of the step, Richardson-extrapolated
        d4 = prob.L / (4 * round(prob.L / tight["dz"]))
        f4, _, _ = ctx.propagate(prob.A0, prob.L, d4, tight["M"], 1e-12)
        f8, _, _ = ctx.propagate(prob.A0, prob.L, d4 / 2, tight["M"], 1e-12)
        ref = f8 + (f8 - f4) / 3
    finally:
        ctx.close()
    err = rel(out, ref)
    assert err < 3e-6
    # the estimate is of the right size, not merely an upper bound
    assert err > 1e-8


def test_rejections():
    prob = fiber()
    ctx = B.Context.from_problem(prob, precision="fp32")
    try:
        with pytest.raises(B.GmmnlseError):
            ctx.choose_step(prob.A0, -1.0, 0.0, 1e-9)
        with pytest.raises(B.GmmnlseError):
            ctx.choose_step(np.zeros_like(prob.A0), prob.L, 0.0, 1e-9)
    finally:
        ctx.close()
