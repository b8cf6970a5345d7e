"""Pins of the oracle's linear mode coupling C_p = i sum_n Q_np A_n (Sec. IV,
"Linear mode coupling including disorder"), an added term of Eq. 1's right-
hand side.  Without dispersion and nonlinearity the equation is the linear
system dA/dz = X A with X = i Q^T, and each integrator's step has a closed
form; with a per-mode propagation constant the exact field is a matrix
exponential."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle as O
from paper_1708_05324_b300 import inputs as I


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _linear_fiber(N=3, Nt=64, beta0=None, Q=None):
    prob = I.workload("C1", Nt=Nt, dt=2e-12 / Nt, fR=0.0, energy=1e-9)
    beta = np.zeros((prob.N, Nt)) if beta0 is None else np.repeat(np.asarray(beta0)[:, None], Nt, axis=1)
    fib = O.Fiber.from_problem(prob, beta=beta, n2=0.0, Q=Q)
    return prob, fib


Q3 = I.coupling_matrix(3, 40.0, seed=21, symmetric=False)  # not symmetric: a transpose shows


def test_converged_mpa_is_the_cayley_step_of_the_coupling():
    """The trapezoid rule on dA/dz = X A gives A_j = (1 - dz X/2)^-1 (1 + dz X/2) A_{j-1}."""
    prob, fib = _linear_fiber(Q=Q3)
    dz, steps = 1e-3, 12
    X = 1j * Q3.T
    C = np.linalg.solve(np.eye(3) - 0.5 * dz * X, np.eye(3) + 0.5 * dz * X)
    exact = np.linalg.matrix_power(C, steps) @ prob.A0
    out, st = O.mpa_propagate(fib, prob.A0, steps * dz, dz, 5, 1e-15)
    assert rel(out, exact) < 1e-12


def test_rk4ip_step_is_the_fourth_order_taylor_polynomial():
    prob, fib = _linear_fiber(Q=Q3)
    h, steps = 2e-3, 7
    Y = 1j * h * Q3.T
    T4 = np.eye(3) + Y + Y @ Y / 2 + Y @ Y @ Y / 6 + Y @ Y @ Y @ Y / 24
    exact = np.linalg.matrix_power(T4, steps) @ prob.A0
    assert rel(O.rk4ip_propagate(fib, prob.A0, steps * h, h), exact) < 1e-12


def test_coupling_with_dispersion_converges_to_the_matrix_exponential():
    """dA/dz = i (B + Q^T) A, B = diag(beta_p): the interaction picture must
    rotate the coupled modes by their own beta (a swapped phase fails); the
    MPA's error falls 4x per halving of dz, RK4IP's 16x."""
    b = np.array([0.0, 900.0, 2100.0])
    prob, fib = _linear_fiber(beta0=b, Q=Q3)
    L = 6e-3
    exact = sl.expm(1j * L * (np.diag(b) + Q3.T)) @ prob.A0
    e = [rel(O.mpa_propagate(fib, prob.A0, L, L / k, 4, 1e-15)[0], exact) for k in (24, 48)]
    assert e[0] < 1e-3
    assert e[0] / e[1] == pytest.approx(4.0, rel=0.05)
    r = [rel(O.rk4ip_propagate(fib, prob.A0, L, L / k), exact) for k in (12, 24)]
    assert r[0] / r[1] == pytest.approx(16.0, rel=0.1)


def test_symmetric_coupling_conserves_energy_with_kerr_and_a_skewed_one_does_not():
    """i Q^T is anti-Hermitian exactly when Q is symmetric: then Q moves energy
    between modes and keeps the total (Kerr without self-steepening conserves
    it too)."""
    prob = I.workload("C1", Nt=128, dt=2e-12 / 128, fR=0.0, energy=10e-9)
    e0 = O.energy_spectral(O.freq_from_time(prob.A0))
    Qs = I.coupling_matrix(3, 40.0, seed=22, symmetric=True)
    drift = {}
    for name, Q in (("none", None), ("sym", Qs), ("skew", Q3)):
        fib = O.Fiber.from_problem(prob, self_steepening=False, Q=Q)
        out, _ = O.mpa_propagate(fib, prob.A0, 4e-3, 1e-4, 10, 1e-14)
        drift[name] = abs(O.energy_spectral(O.freq_from_time(out)) / e0 - 1)
        if name == "sym":
            moved = out
    # the trapezoid's own step error with Kerr, not the coupling's
    assert drift["sym"] < 1e-5 and drift["sym"] < 3 * drift["none"] + 1e-9
    # energy moved between modes
    m0 = np.sum(abs(prob.A0) ** 2, axis=1)
    m1 = np.sum(abs(moved) ** 2, axis=1)
    assert np.max(abs(m1 - m0)) / np.sum(m0) > 1e-3
    assert drift["skew"] > 1e-3


G3 = np.array([3.0, -5.0, 11.0])  # per-mode field gain [1/m]; distinct, so a mode mix-up shows


def test_gain_steps_are_the_cayley_and_taylor_factors():
    """dA_p/dz = g_p A_p alone: the converged trapezoid multiplies mode p by
    (1 + g dz/2)/(1 - g dz/2) per substep, RK4IP by 1 + x + x^2/2 + x^3/6 +
    x^4/24 (x = g h) per step."""
    prob, fib = _linear_fiber()
    fib = O.Fiber.from_problem(prob, beta=fib.beta, n2=0.0, gain=G3)
    dz, steps = 1e-3, 10
    cay = ((1 + 0.5 * dz * G3) / (1 - 0.5 * dz * G3)) ** steps
    out, _ = O.mpa_propagate(fib, prob.A0, steps * dz, dz, 5, 1e-15)
    assert rel(out, cay[:, None] * prob.A0) < 1e-12
    x = G3 * dz
    tay = (1 + x + x ** 2 / 2 + x ** 3 / 6 + x ** 4 / 24) ** steps
    assert rel(O.rk4ip_propagate(fib, prob.A0, steps * dz, dz), tay[:, None] * prob.A0) < 1e-12


def test_gain_with_coupling_and_dispersion_converges_to_the_matrix_exponential():
    b = np.array([0.0, 900.0, 2100.0])
    prob, fib = _linear_fiber(beta0=b, Q=Q3)
    fib = O.Fiber.from_problem(prob, beta=fib.beta, n2=0.0, Q=Q3, gain=G3)
    L = 6e-3
    exact = sl.expm(L * (1j * np.diag(b) + 1j * Q3.T + np.diag(G3))) @ prob.A0
    e = [rel(O.mpa_propagate(fib, prob.A0, L, L / k, 4, 1e-15)[0], exact) for k in (24, 48)]
    assert e[0] < 1e-3
    assert e[0] / e[1] == pytest.approx(4.0, rel=0.05)


# ----------------------------------------------------------------------------
# Saturating gain (Sec. IV): g_p A_p - sat sum_lmn S^R_plmn A_l int A_m A_n^* dtau
# ----------------------------------------------------------------------------
def _single_mode(SR_factor=2.0, Nt=128):
    prob = I.grin_problem("sat", N=1, Nt=Nt, dt=2e-12 / Nt, kind="gaussian", fwhm=150e-15, energy=1e-9,
                          L=1e-3, dz=1e-4, M=5, tol=1e-14, seed=7, fR=0.0, s_from="gh")
    return prob, prob.SK * SR_factor


def test_saturated_gain_of_one_mode_follows_the_logistic_energy_law():
    """One mode, no dispersion, no Kerr: dA/dz = (g - sat S^R_1111 W) A with
    W = int |A|^2 dt, so dW/dz = 2 g W - 2 sat S^R W^2, solved by
    1/W = e^{-2gz}/W0 + (sat S^R/g)(1 - e^{-2gz}), and A keeps its shape and
    phase: A(z, t) = A0(t) sqrt(W/W0).  S^R is taken twice S^K, so that the
    Raman tensor (not the Kerr one) is the one that must saturate.  The MPA
    converges to it at second order."""
    prob, SR = _single_mode()
    g = 20.0
    W0 = prob.dt * float(np.sum(np.abs(prob.A0) ** 2))
    sat = 0.2 * g / (SR[0, 0, 0, 0] * W0)  # the energy saturates towards 5 W0
    fib = O.Fiber.from_problem(prob, beta=np.zeros_like(prob.beta), n2=0.0, SR=SR, fR=0.0, gain=np.array([g]),
                               sat=sat)
    L = 0.05
    W = 1.0 / (np.exp(-2 * g * L) / W0 + (sat * SR[0, 0, 0, 0] / g) * (1 - np.exp(-2 * g * L)))
    exact = prob.A0 * np.sqrt(W / W0)
    assert W / W0 > 1.5 and W / W0 < 0.5 * np.exp(2 * g * L)  # gained, and clearly saturated
    e = [rel(O.mpa_propagate(fib, prob.A0, L, L / k, 5, 1e-15)[0], exact) for k in (40, 80)]
    assert e[1] < 1e-4
    assert e[0] / e[1] == pytest.approx(4.0, rel=0.05)
    r = [rel(O.rk4ip_propagate(fib, prob.A0, L, L / k), exact) for k in (20, 40)]
    assert r[0] / r[1] == pytest.approx(16.0, rel=0.15)


def test_saturation_energy_rate_of_several_modes():
    """dW/dz of the total energy W = sum_p int |A_p|^2 dt under Eq. 1 plus the
    saturating gain, at any field: Kerr without self-steepening and the
    dispersion keep W, so dW/dz = 2 g W - 2 sat Re sum_plmn S^R_plmn E_mn E_lp
    with E_mn = int A_m A_n^* dt (equal gain g in every mode).  The oracle's
    operator, applied to a random three-mode field, against that sum written
    as explicit loops."""
    prob = I.workload("C1", Nt=64, dt=2e-12 / 64, fR=0.0, energy=2e-9)
    N, dt = prob.N, prob.dt
    g, sat = 7.0, 0.3
    fib = O.Fiber.from_problem(prob, self_steepening=False, gain=np.full(N, g), sat=sat)
    rng = np.random.default_rng(5)
    A = prob.A0 * (1 + 0.3 * (rng.standard_normal(prob.A0.shape) + 1j * rng.standard_normal(prob.A0.shape)))
    Aw = O.freq_from_time(A)
    rate = 2 * float(np.real(np.sum(np.conj(Aw) * O.nonlinear_operator(fib, Aw)))) * dt / prob.Nt
    E = np.zeros((N, N), dtype=complex)
    for m in range(N):
        for n in range(N):
            E[m, n] = dt * np.sum(A[m] * np.conj(A[n]))
    sat_sum = 0.0
    for p in range(N):
        for l in range(N):
            for m in range(N):
                for n in range(N):
                    sat_sum += prob.SK[p, l, m, n] * (E[m, n] * E[l, p]).real
    W = dt * float(np.sum(np.abs(A) ** 2))
    assert rate == pytest.approx(2 * g * W - 2 * sat * sat_sum, rel=1e-10)
    assert 2 * sat * sat_sum > 0.1 * 2 * g * W  # the saturation is a sizeable part of the rate


# ----------------------------------------------------------------------------
# Linear mode coupling with a longitudinal profile: Q_np(z) = Q_np f(z)
# ----------------------------------------------------------------------------
def test_coupling_profile_gives_the_integrated_coupling():
    """dA/dz = i f(z) Q^T A with f(z) = 1 + z/ell (tabulated, linearly
    interpolated: exact for a ramp) has A(z) = expm(i F(z) Q^T) A0,
    F(z) = z + z^2 / (2 ell).  The MPA takes f at every substep z_j (second
    order: 4x per halving of dz), RK4IP at its stage positions z, z + h/2,
    z + h (fourth order: 16x)."""
    ell = 2e-3
    zs_dz = 1e-4
    f = 1.0 + np.arange(200) * zs_dz / ell
    prob, fib = _linear_fiber()
    fib = O.Fiber.from_problem(prob, beta=fib.beta, n2=0.0, Q=Q3, Q_profile=f, Q_profile_dz=zs_dz)
    L = 6e-3
    F = L + L * L / (2 * ell)
    exact = sl.expm(1j * F * Q3.T) @ prob.A0
    e = [rel(O.mpa_propagate(fib, prob.A0, L, L / k, 4, 1e-15)[0], exact) for k in (24, 48)]
    assert e[0] < 1e-3
    assert e[0] / e[1] == pytest.approx(4.0, rel=0.05)
    r = [rel(O.rk4ip_propagate(fib, prob.A0, L, L / k), exact) for k in (12, 24)]
    assert r[0] / r[1] == pytest.approx(16.0, rel=0.1)
