"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each test names the passage of the paper (section / equation) or the piece of
mathematics it relies on.  None compares the oracle with itself: the expected
values are closed forms, invariants, a brute-force sum or an independent
integrator, chosen so that a dropped term, a sign error, a wrong index or a
transposed operand anywhere in oracle/gmmnlse.py fails at least one test.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1708_05324_b300 import inputs as I

LAM0 = 1030e-9
N2 = 2.3e-20
AEFF = 1.29e-10  # m^2, fundamental GRIN mode of the benchmark fiber


def single_mode(Nt, dt, beta1=0.0, beta2=0.0, beta3=0.0, fR=0.0, ss=False,
                n2=N2, s=1.0 / AEFF, hR=None):
    w = 2 * np.pi * np.fft.fftfreq(Nt, dt)
    beta = (beta1 * w + beta2 * w ** 2 / 2 + beta3 * w ** 3 / 6)[None, :]
    S = np.full((1, 1, 1, 1), s)
    if hR is None:
        hR = I.raman_response(Nt, dt)
    return O.Fiber(beta, S, S, fR, hR, dt, LAM0, n2, ss)


def gamma_of(s=1.0 / AEFF, n2=N2, lam0=LAM0):
    """gamma = n2 omega0 S / c with omega0 / c = 2 pi / lam0 (Eq. 1 prefactor),
    formed here independently of the oracle."""
    return n2 * 2.0 * math.pi / lam0 * s


def gaussian(Nt, dt, T0, P0, phase=0.0):
    t = I.time_grid(Nt, dt)
    return (math.sqrt(P0) * np.exp(-t ** 2 / (2 * T0 ** 2)) * np.exp(1j * phase))[None, :]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


# ----------------------------------------------------------------------------
# Fourier sign, phase bookkeeping, linear propagation (Sec. III.A, Eqs. 5, 8, "9")
# ----------------------------------------------------------------------------
def test_p5_walkoff_moves_pulse_to_later_time():
    """Eq. 8: with only delta beta_1 > 0 the envelope becomes S(t - db1 z).
    Choose db1 z = 8 dt so the exact answer is a shift by 8 samples."""
    Nt, dt = 256, 5e-15
    L, dz, M = 0.02, 1e-3, 5
    db1 = 8 * dt / L
    w = 2 * np.pi * np.fft.fftfreq(Nt, dt)
    beta = np.stack([0 * w, db1 * w])
    S = np.zeros((2, 2, 2, 2))
    fib = O.Fiber(beta, S, S, 0.0, None, dt, LAM0, N2, True)
    A0 = np.vstack([gaussian(Nt, dt, 40e-15, 1.0), gaussian(Nt, dt, 40e-15, 2.0, 0.4)])
    out, st = O.mpa_propagate(fib, A0, L, dz, M, 1e-12)
    assert st["status"] == O.gmmnlse.OK
    np.testing.assert_allclose(out[0], A0[0], atol=1e-14)
    np.testing.assert_allclose(out[1], np.roll(A0[1], 8), atol=1e-13 * abs(A0[1]).max())
    # pulse centroid moved to later t (not earlier)
    t = I.time_grid(Nt, dt)
    c0 = np.sum(t * abs(A0[1]) ** 2) / np.sum(abs(A0[1]) ** 2)
    c1 = np.sum(t * abs(out[1]) ** 2) / np.sum(abs(out[1]) ** 2)
    assert c1 - c0 == pytest.approx(8 * dt, rel=1e-9)


def test_p6_linear_phase_bookkeeping_over_a_long_fiber():
    """Eq. 5 / Eq. cov: with no nonlinearity the output is exactly
    F^-1{F{A0} exp(i beta L)}, also when beta L reaches ~1e5 rad.  The GRIN
    beta of the 15-mode benchmark fiber is used; dz = 2^-10 m and M = 8 make
    every z_j exactly representable, so the only error is the FP64 rounding of
    beta * (M dz) in each of the 100 long steps (<= 0.5 ulp of ~1e3 rad each,
    < 6e-12 rad in total); the reference phase is formed in long double."""
    prob = I.workload("C3", Nt=256, dt=20e-12 / 256, N=6, L=0.1)
    fib = O.Fiber.from_problem(prob, n2=0.0)
    dz, M = 2.0 ** -10, 8
    L = 100 * M * dz
    out, st = O.mpa_propagate(fib, prob.A0, L, dz, M, 1e-12)
    assert st["status"] == O.gmmnlse.OK and st["iters"][0] == 1
    arg = (fib.beta.astype(np.longdouble) * np.longdouble(L))
    ph = np.cos(arg).astype(np.float64) + 1j * np.sin(arg).astype(np.float64)
    assert float(np.max(np.abs(fib.beta * L))) > 5e3
    ref = O.time_from_freq(O.freq_from_time(prob.A0) * ph)
    assert np.max(np.abs(out - ref)) / np.max(np.abs(ref)) < 1e-11


def test_p7_gaussian_gvd_broadening():
    """Eq. "9" (Sec. III.A.3): T(z) = T0 sqrt(1 + (z |beta2| / T0^2)^2) for a
    transform-limited Gaussian, measured here by the RMS width."""
    Nt, dt = 2048, 4e-15
    T0, beta2 = 60e-15, 2e-26
    LD = T0 ** 2 / beta2
    fib = single_mode(Nt, dt, beta2=beta2, n2=0.0)
    A0 = gaussian(Nt, dt, T0, 1.0)
    L = 2 * LD
    out, _ = O.mpa_propagate(fib, A0, L, L / 20, 5, 1e-12)
    t = I.time_grid(Nt, dt)

    def rms(a):
        p = abs(a[0]) ** 2
        c = np.sum(t * p) / np.sum(p)
        return math.sqrt(np.sum((t - c) ** 2 * p) / np.sum(p))

    assert rms(out) / rms(A0) == pytest.approx(math.sqrt(1 + (L * beta2 / T0 ** 2) ** 2), rel=1e-9)


# ----------------------------------------------------------------------------
# Nonlinear sign and magnitude (Sec. III.C.1, Eq. 3; Sec. III.D)
# ----------------------------------------------------------------------------
def test_p8_spm_matches_discrete_and_continuum_closed_forms():
    """Dispersionless SPM, one mode, no self-steepening, f_R = 0:
    dA/dz = i gamma |A|^2 A with gamma = n2 w0 S_1111 / c (A_eff = 1/S_pppp,
    Sec. III.C.1).  The converged MPA is the interaction-picture trapezoid
    rule, which for this equation keeps |A| and advances the phase by
    2 atan(theta), theta = gamma |A|^2 dz / 2, per dz exactly.  It must match
    that to rounding and the continuum exp(i gamma |A|^2 z) to O(theta^3) per
    step."""
    Nt, dt = 64, 10e-15
    fib = single_mode(Nt, dt)
    gamma = gamma_of()
    A0 = gaussian(Nt, dt, 100e-15, 1e5, phase=0.3)
    L, dz, M = 0.01, 1e-4, 10
    out, st = O.mpa_propagate(fib, A0, L, dz, M, 1e-14)
    theta = gamma * abs(A0) ** 2 * dz / 2
    disc = A0 * np.exp(1j * 2 * round(L / dz) * np.arctan(theta))
    cont = A0 * np.exp(1j * gamma * abs(A0) ** 2 * L)
    peak = abs(A0).max()
    assert np.max(abs(out - disc)) / peak < 1e-13
    bound = round(L / dz) * (2 * theta.max() ** 3 / 3) * 1.01
    err_c = np.max(abs(out - cont)) / peak
    assert 0.5 * bound < err_c < bound
    assert gamma * 1e5 * L > 1.0  # a sizeable nonlinear phase


def test_p9_fundamental_soliton_second_order():
    """Fundamental soliton of Eq. 3 (N = 1, beta2 < 0): A = sqrt(P0) sech(t/T0)
    exp(i gamma P0 z / 2), P0 = |beta2| / (gamma T0^2) (Agrawal, cited in
    Sec. III.D as the analytic check).  A wrong relative sign between
    dispersion and nonlinearity, or in exp(-D z') of Eq. MPA_eq, destroys it.
    The error falls 4x per halving of dz (second order, Sec. III.D trapezoid)."""
    Nt, T0, beta2 = 1024, 100e-15, -2e-26
    dt = 40 * T0 / Nt
    fib = single_mode(Nt, dt, beta2=beta2)
    gamma = gamma_of()
    P0 = abs(beta2) / (gamma * T0 ** 2)
    LD = T0 ** 2 / abs(beta2)
    t = I.time_grid(Nt, dt)
    A0 = (math.sqrt(P0) / np.cosh(t / T0))[None, :].astype(complex)
    L = 0.5 * LD
    exact = A0 * np.exp(1j * gamma * P0 * L / 2)
    errs = []
    for dz in (LD / 50, LD / 100):
        out, _ = O.mpa_propagate(fib, A0, L, dz, 5, 1e-13)
        errs.append(np.max(abs(out - exact)) / math.sqrt(P0))
    assert errs[0] < 2e-4
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.05)


def test_self_steepening_delays_the_peak():
    """Sec. III.C.4: self-steepening forms a steep trailing edge (larger t).
    For dA/dz = i gamma (1 + (i/w0) d/dt)(|A|^2 A) the intensity centroid moves
    at d<t>/dz = (3 gamma / (2 w0)) int|A|^4 / int|A|^2 > 0 (integration by
    parts).  Checked over a short length where |A|^4 barely changes."""
    Nt, dt = 1024, 2e-15
    fib = single_mode(Nt, dt, ss=True)
    gamma = gamma_of()
    A0 = gaussian(Nt, dt, 30e-15, 1e5)
    L = 5e-3  # nonlinear phase gamma P0 L ~ 0.54 rad
    out, _ = O.mpa_propagate(fib, A0, L, L / 100, 10, 1e-14)
    t = I.time_grid(Nt, dt)
    p0, p1 = abs(A0[0]) ** 2, abs(out[0]) ** 2
    shift = np.sum(t * p1) / np.sum(p1) - np.sum(t * p0) / np.sum(p0)
    omega0 = 2 * math.pi * 299792458.0 / LAM0
    rate = 3 * gamma / (2 * omega0) * np.sum(p0 ** 2) / np.sum(p0)
    assert shift > 0
    assert shift == pytest.approx(rate * L, rel=1e-4)


# ----------------------------------------------------------------------------
# Raman (Sec. III.C.5, Eq. 1)
# ----------------------------------------------------------------------------
def test_p12_fft_convolution_equals_direct_sum():
    rng = np.random.default_rng(12)
    Nt, dt = 32, 3e-15
    h = rng.standard_normal(Nt)
    q = rng.standard_normal((3, Nt)) + 1j * rng.standard_normal((3, Nt))
    np.testing.assert_allclose(O.circular_convolution(h, q, dt),
                               O.circular_convolution_direct(h, q, dt), rtol=0, atol=1e-13 * dt * 40)


def test_p10_raman_is_transparent_for_cw_light():
    """With dt sum h_R = 1, h_R * U = U for a constant U, so a CW multimode
    field propagates identically with f_R = 0.18 and with f_R = 0 (Eq. 1: the
    Raman and Kerr brackets coincide when S^R = S^K)."""
    prob = I.workload("C1", Nt=64, dt=20e-15)
    w = I.random_mode_weights(3, 7)
    A0 = (w[:, None] * math.sqrt(5e4)) * np.ones((1, 64))
    hR = I.raman_response(64, 20e-15)
    f0 = O.Fiber.from_problem(prob, fR=0.0, hR=hR)
    f1 = O.Fiber.from_problem(prob, fR=0.18, hR=hR)
    o0, _ = O.mpa_propagate(f0, A0, 0.01, 5e-4, 5, 1e-14)
    o1, _ = O.mpa_propagate(f1, A0, 0.01, 5e-4, 5, 1e-14)
    assert rel(o1, o0) < 1e-13
    assert rel(o0, A0) > 1e-2  # the field did evolve (FWM + SPM + beating)


def test_p11_raman_red_shift_matches_gordon_rate():
    """Raman self-frequency shift (Sec. III.C.5: a spectral redshift) of a
    fundamental soliton.  Gordon's perturbative rate (Opt. Lett. 11, 662,
    1986): dOmega/dz = -(8/15) T_R |beta2| / T0^4, T_R = f_R int t h_R(t) dt,
    valid for T0 >> T_R (here T0 = 120 fs, T_R = 1.5 fs: within 5 percent).
    A reversed (acausal) response or a wrong Fourier sign gives a blue shift."""
    Nt, T0, beta2 = 2048, 120e-15, -2e-26
    dt = 60 * T0 / Nt
    hR = I.raman_response(Nt, dt)
    fib = single_mode(Nt, dt, beta2=beta2, fR=0.18, hR=hR)
    gamma = gamma_of()
    P0 = abs(beta2) / (gamma * T0 ** 2)
    t = I.time_grid(Nt, dt)
    A0 = (math.sqrt(P0) / np.cosh(t / T0))[None, :].astype(complex)
    LD = T0 ** 2 / abs(beta2)
    L = 0.4 * LD
    out, _ = O.mpa_propagate(fib, A0, L, L / 40, 5, 1e-12)
    Aw = O.freq_from_time(out)
    w = 2 * np.pi * np.fft.fftfreq(Nt, dt)
    shift = np.sum(w * abs(Aw[0]) ** 2) / np.sum(abs(Aw[0]) ** 2)
    TR = 0.18 * dt * np.sum(np.arange(Nt) * dt * hR)
    gordon = -(8.0 / 15.0) * TR * abs(beta2) / T0 ** 4 * L
    assert shift < 0
    assert shift == pytest.approx(gordon, rel=0.06)
    f0 = single_mode(Nt, dt, beta2=beta2, fR=0.0, hR=hR)
    o0, _ = O.mpa_propagate(f0, A0, L, L / 40, 5, 1e-12)
    Aw0 = O.freq_from_time(o0)
    assert abs(np.sum(w * abs(Aw0[0]) ** 2) / np.sum(abs(Aw0[0]) ** 2)) < 1e-3 * abs(gordon)


# ----------------------------------------------------------------------------
# Conservation laws (Sec. III.C.2: SPM/XPM carry no energy; Eq. 2 symmetry)
# ----------------------------------------------------------------------------
def _drift(fib, A0, L, dz, M, fn):
    out, _ = O.mpa_propagate(fib, A0, L, dz, M, 1e-14)
    a = fn(O.freq_from_time(A0))
    b = fn(O.freq_from_time(out))
    return abs(b - a) / a


@pytest.mark.parametrize("ss,fR", [(True, 0.0), (False, 0.18)])
def test_p13_energy_is_conserved_to_second_order(ss, fR):
    """Energy sum_p int |A_p|^2 is a continuum invariant of Eq. 1 when S is
    real and fully symmetric (Eq. 2) and f_R = 0 (with or without
    self-steepening), or f_R != 0 without self-steepening (h_R real).  The
    trapezoid scheme keeps it to O(dz^2): drift falls ~4x per dz halving."""
    prob = I.workload("C1", Nt=256, dt=2e-12 / 256, fR=fR, energy=10e-9)
    fib = O.Fiber.from_problem(prob, self_steepening=ss, hR=I.raman_response(256, 2e-12 / 256))
    d1 = _drift(fib, prob.A0, 2e-3, 1e-4, 5, O.energy_spectral)
    d2 = _drift(fib, prob.A0, 2e-3, 5e-5, 5, O.energy_spectral)
    assert d1 < 1e-5
    assert 3.0 < d1 / d2 < 5.0


def test_p14_photon_number_conserved_with_raman_and_self_steepening():
    """With Raman and self-steepening the energy is not conserved (Raman
    hands energy to the medium) but the photon number sum |A~|^2/(w0 + w) is.
    The oracle's energy must drift at first order in z while the photon
    number drifts only at O(dz^2)."""
    prob = I.workload("C1", Nt=256, dt=2e-12 / 256, fR=0.18, energy=10e-9, fwhm=40e-15)
    fib = O.Fiber.from_problem(prob, self_steepening=True, hR=I.raman_response(256, 2e-12 / 256))
    pn = lambda Aw: O.photon_number(fib, Aw)  # noqa: E731
    d1 = _drift(fib, prob.A0, 2e-3, 1e-4, 5, pn)
    d2 = _drift(fib, prob.A0, 2e-3, 5e-5, 5, pn)
    e1 = _drift(fib, prob.A0, 2e-3, 5e-5, 5, O.energy_spectral)
    assert 3.0 < d1 / d2 < 5.0
    assert e1 > 100 * d2


# ----------------------------------------------------------------------------
# Contraction: brute force (Eq. 1)
# ----------------------------------------------------------------------------
def test_p18_bracket_equals_brute_force_loops():
    """The Kerr and Raman sums of Eq. 1 against explicit Python loops over
    (p, l, m, n, t, tau) with a random, *non-symmetric* S (so that any
    transposition of indices or misplaced conjugate is caught)."""
    rng = np.random.default_rng(18)
    N, Nt, dt = 3, 8, 2e-15
    SK = rng.standard_normal((N, N, N, N))
    SR = rng.standard_normal((N, N, N, N))
    A = rng.standard_normal((N, Nt)) + 1j * rng.standard_normal((N, Nt))
    h = rng.random(Nt)
    fR = 0.3
    fib = O.Fiber(np.zeros((N, Nt)), SK, SR, fR, h, dt, LAM0, N2, False)
    got = O.nonlinear_bracket(fib, A)
    want = np.zeros((N, Nt), dtype=complex)
    for p in range(N):
        for t in range(Nt):
            kerr = 0j
            ram = 0j
            for l in range(N):
                for m in range(N):
                    for n in range(N):
                        kerr += SK[p, l, m, n] * A[l, t] * A[m, t] * A[n, t].conjugate()
                        conv = 0j
                        for tau in range(Nt):
                            conv += h[tau] * A[m, (t - tau) % Nt] * A[n, (t - tau) % Nt].conjugate()
                        ram += SR[p, l, m, n] * A[l, t] * conv * dt
            want[p, t] = (1 - fR) * kerr + fR * ram
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13 * abs(want).max())


def test_integrand_against_explicit_dft():
    """Eq. MPA_eq's integrand with explicitly summed DFTs in the e^{-i w t}
    convention (no FFT library), a random fiber and self-steepening on."""
    rng = np.random.default_rng(5)
    N, Nt, dt = 2, 16, 3e-15
    S = rng.standard_normal((N, N, N, N))
    beta = rng.standard_normal((N, Nt)) * 1e3
    fib = O.Fiber(beta, S, S, 0.0, None, dt, LAM0, N2, True)
    psi = rng.standard_normal((N, Nt)) + 1j * rng.standard_normal((N, Nt))
    z = 3.7e-4
    w = 2 * np.pi * np.fft.fftfreq(Nt, dt)
    tk = np.arange(Nt) * dt
    E = np.exp(1j * beta * z)
    A = np.array([[sum(psi[p, q] * E[p, q] * np.exp(-1j * w[q] * tk[k]) for q in range(Nt)) / Nt
                   for k in range(Nt)] for p in range(N)])
    NL = np.array([[sum(S[p, l, m, n] * A[l, k] * A[m, k] * np.conj(A[n, k])
                        for l in range(N) for m in range(N) for n in range(N))
                    for k in range(Nt)] for p in range(N)])
    F = np.array([[sum(NL[p, k] * np.exp(1j * w[q] * tk[k]) for k in range(Nt))
                   for q in range(Nt)] for p in range(N)])
    omega0 = 2 * math.pi * 299792458.0 / LAM0
    want = 1j * gamma_of(1.0) * (1 + w / omega0) * F * np.exp(-1j * beta * z)
    np.testing.assert_allclose(O.integrand(fib, psi, z), want, rtol=1e-12, atol=1e-12 * abs(want).max())


# ----------------------------------------------------------------------------
# The MPA iteration itself (Sec. III.D)
# ----------------------------------------------------------------------------
def _small_grin(fR=0.18, energy=10e-9, Nt=256):
    prob = I.workload("C1", Nt=Nt, dt=2e-12 / Nt, fR=fR, energy=energy)
    return prob, O.Fiber.from_problem(prob, hR=I.raman_response(Nt, 2e-12 / Nt))


def test_p2_converged_mpa_is_the_sequential_ip_trapezoid():
    """The fixed point of the MPA satisfies psi_j - psi_{j-1} =
    (dz/2)(I_{j-1} + I_j), i.e. the interaction-picture trapezoid rule
    A_j = e^{D dz}(A_{j-1} + dz/2 N(A_{j-1})) + dz/2 N(A_j) solved one step at a
    time.  Both must agree to the iteration tolerance."""
    prob, fib = _small_grin()
    a, st = O.mpa_propagate(fib, prob.A0, 3e-3, 1e-4, 10, 1e-14)
    b = O.iptrap_propagate(fib, prob.A0, 3e-3, 1e-4)
    assert rel(a, b) < 1e-12
    assert rel(a, prob.A0) > 1e-3


def test_p1_converged_mpa_does_not_depend_on_M():
    prob, fib = _small_grin()
    outs = [O.mpa_propagate(fib, prob.A0, 4e-3, 1e-4, M, 1e-14)[0] for M in (1, 4, 8, 20)]
    for o in outs[1:]:
        assert rel(o, outs[0]) < 1e-12


def test_p4_rk4ip_and_mpa_converge_to_the_same_solution():
    """Two different integrators of Eq. 1 (RK4 in the interaction picture and
    the MPA trapezoid) approach one continuum solution; the MPA's distance to
    a fine RK4IP run falls 4x per halving of dz."""
    prob, fib = _small_grin(Nt=128)
    L = 4e-3
    ref = O.rk4ip_propagate(fib, prob.A0, L, L / 400)
    e1 = rel(O.mpa_propagate(fib, prob.A0, L, L / 40, 10, 1e-14)[0], ref)
    e2 = rel(O.mpa_propagate(fib, prob.A0, L, L / 80, 10, 1e-14)[0], ref)
    assert e1 < 1e-3
    assert e1 / e2 == pytest.approx(4.0, rel=0.1)


def test_p19_iteration_error_falls_geometrically():
    """Sec. III.D: the error after n iterations ~ (L/z_NL)^(n+1), so eps
    shrinks per iteration by a factor proportional to L/z_NL: halving the long
    step halves the mean contraction factor.  At L = z_NL/10 a loose
    tolerance (1e-3) is met within 2-3 iterations."""
    Nt, dt = 256, 2e-12 / 256
    prob = I.workload("C1", Nt=Nt, dt=dt, fR=0.0)
    fib = O.Fiber.from_problem(prob)
    P0 = float(np.max(np.sum(abs(prob.A0) ** 2, axis=0)))
    zNL = 1.0 / (gamma_of(prob.SK[0, 0, 0, 0], prob.n2, prob.lam0) * P0)
    psi0 = O.freq_from_time(prob.A0)
    factor = {}
    traces = {}
    for div in (5, 10, 20):  # L = z_NL / div
        M, dz = 10, zNL / (10 * div)
        _, n, trace, status = O.mpa_long_step(fib, psi0, dz, M, 1e-300, max_iter=6)
        assert status == O.gmmnlse.E_NOT_CONVERGED and n == 6
        assert all(trace[i + 1] < trace[i] for i in range(5))
        factor[div] = (trace[5] / trace[0]) ** (1 / 5)
        traces[div] = trace
    assert factor[5] / factor[10] == pytest.approx(2.0, rel=0.15)
    assert factor[10] / factor[20] == pytest.approx(2.0, rel=0.15)
    assert factor[10] < 0.1
    assert traces[10][2] < 1e-3


def test_not_converged_and_nonfinite_statuses():
    prob, fib = _small_grin()
    _, st = O.mpa_propagate(fib, prob.A0, 2e-3, 1e-4, 10, 1e-300, max_iter=3)
    assert st["status"] == O.gmmnlse.E_NOT_CONVERGED and st["z"] == 0.0
    bad = prob.A0.copy()
    bad[0, 5] = np.nan
    _, st = O.mpa_propagate(fib, bad, 2e-3, 1e-4, 10, 1e-10)
    assert st["status"] == O.gmmnlse.E_NONFINITE


def test_substep_schedule():
    assert O.substep_schedule(0.05, 0.5e-3, 5) == [5] * 20
    assert O.substep_schedule(1.2e-3, 1e-4, 5) == [5, 5, 2]
    with pytest.raises(ValueError):
        O.substep_schedule(1.25e-3, 1e-4, 5)


# ----------------------------------------------------------------------------
# Length scales of the two step sizes (Sec. III.D)
# ----------------------------------------------------------------------------
def test_length_scales_of_a_soliton_and_of_the_grin_mode_groups():
    """z_NL of the fundamental soliton is the dispersion length (gamma P0 L_D
    = 1, Agrawal), formed here from gamma = n2 omega0 S / c; z_IM of a GRIN
    fiber is set by its highest mode group: the groups are spaced by
    delta beta0 = NA / (a n) to first order (Sec. III.A, equally spaced
    groups), so with groups 0-2 z_IM = 1 / (2 delta beta0), and a single mode
    has none."""
    Nt, T0, beta2 = 256, 100e-15, -2e-26
    dt = 40 * T0 / Nt
    fib = single_mode(Nt, dt, beta2=beta2)
    P0 = abs(beta2) / (gamma_of() * T0 ** 2)
    t = I.time_grid(Nt, dt)
    A0 = (math.sqrt(P0) / np.cosh(t / T0))[None, :].astype(complex)
    z_nl, z_im = O.length_scales(fib, A0)
    assert z_nl == pytest.approx(T0 ** 2 / abs(beta2), rel=1e-12)
    assert z_im == math.inf
    prob = I.grin_problem("ls", N=6, Nt=256, dt=2e-12 / 256, kind="gaussian", fwhm=150e-15, energy=10e-9,
                          L=1e-3, dz=1e-4, M=5, tol=1e-12, seed=3, fR=0.0, s_from="gh")
    g6 = O.Fiber.from_problem(prob)
    z_nl, z_im = O.length_scales(g6, prob.A0)
    db0 = 0.2 / (25e-6 * float(I.silica_index(LAM0)))
    assert z_im == pytest.approx(1.0 / (2 * db0), rel=2e-2)
    P0 = float(np.max(np.sum(np.abs(prob.A0) ** 2, axis=0)))
    w = I.grin_mode_width(25e-6, 0.2, LAM0)
    assert z_nl == pytest.approx(1.0 / (gamma_of(s=1.0 / (math.pi * w * w)) * P0), rel=1e-9)


# ----------------------------------------------------------------------------
# Complex coupling tensors (Eq. 1 without the single-polarization, real-
# profile simplification of Eq. 2)
# ----------------------------------------------------------------------------
def test_p20_complex_bracket_equals_brute_force_loops():
    """The bracket of Eq. 1 with complex, unsymmetric S^K and S^R against
    explicit loops over (p, l, m, n, t, tau)."""
    rng = np.random.default_rng(20)
    N, Nt, dt = 3, 8, 2e-15
    SK = rng.standard_normal((N, N, N, N)) + 1j * rng.standard_normal((N, N, N, N))
    SR = rng.standard_normal((N, N, N, N)) + 1j * rng.standard_normal((N, N, N, N))
    A = rng.standard_normal((N, Nt)) + 1j * rng.standard_normal((N, Nt))
    h = rng.random(Nt)
    fR = 0.3
    fib = O.Fiber(np.zeros((N, Nt)), SK, SR, fR, h, dt, LAM0, N2, False)
    got = O.nonlinear_bracket(fib, A)
    want = np.zeros((N, Nt), dtype=complex)
    for p in range(N):
        for t in range(Nt):
            for l in range(N):
                for m in range(N):
                    for n in range(N):
                        conv = sum(h[tau] * A[m, (t - tau) % Nt] * np.conj(A[n, (t - tau) % Nt])
                                   for tau in range(Nt)) * dt
                        want[p, t] += A[l, t] * ((1 - fR) * SK[p, l, m, n] * A[m, t] * np.conj(A[n, t])
                                                 + fR * SR[p, l, m, n] * conv)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13 * abs(want).max())


def test_p21_complex_single_mode_cw_closed_form():
    """One mode, no dispersion, a complex self-coupling s: dA/dz = i gamma0 s
    |A|^2 A (Eq. 1 with N = 1, f_R = 0, no self-steepening) gives for CW light
    |A(z)|^2 = I0 / (1 + 2 gamma0 Im(s) I0 z) and the phase
    Re(s) / (2 Im(s)) ln(1 + 2 gamma0 Im(s) I0 z).  The MPA reaches it to
    its O(dz^2) trapezoid error."""
    Nt, dt = 32, 1e-14
    s = (1.0 + 0.35j) / AEFF
    fib = single_mode(Nt, dt, s=s)
    I0, L = 2.0e4, 0.5
    A0 = np.full((1, Nt), math.sqrt(I0), dtype=complex)
    g = fib.gamma0
    x = 1.0 + 2.0 * g * s.imag * I0 * L
    want = math.sqrt(I0 / x) * np.exp(1j * s.real / (2.0 * s.imag) * math.log(x))
    assert abs(I0 / x - 1.0) > 0.05  # the loss is visible
    errs = []
    for dz in (1e-3, 5e-4):
        A, st = O.mpa_propagate(fib, A0, L, dz, 10, 1e-14, max_iter=200)
        assert st["status"] == 0
        errs.append(rel(A, np.full((1, Nt), want)))
    assert errs[0] < 4e-4
    assert 3.5 < errs[0] / errs[1] < 4.5  # second order in dz


def test_p22_complex_mode_basis_is_a_unitary_change_of_variables():
    """A unitary mixing T of a degenerate pair of GRIN modes (HG10, HG01 ->
    (HG10 +- i HG01)/sqrt(2)) turns the real S of Eq. 2 into the complex,
    m <-> n unsymmetric S'_plmn = sum T_pa T*_lb T*_mc T_nd S_abcd, and the
    same for S^R (Eq. 1's A_l A_m A_n^* and A_l (h_R * A_m A_n^*) transform
    alike).  The dispersion is diagonal and equal on the pair, so it commutes
    with T: the MPA in the mixed basis, from T A0, gives T times the MPA in
    the original basis, with Raman and self-steepening."""
    p = I.grin_problem("cx", N=3, Nt=256, dt=20e-15, kind="gaussian", fwhm=300e-15, energy=20e-9,
                       L=4e-3, dz=1e-4, M=8, tol=1e-12, seed=2, fR=0.18, s_from="gh")
    beta = p.beta.copy()
    beta[2] = beta[1]  # exactly degenerate pair
    r = 1.0 / math.sqrt(2.0)
    T = np.array([[1, 0, 0], [0, r, 1j * r], [0, r, -1j * r]], dtype=complex)
    np.testing.assert_allclose(T @ T.conj().T, np.eye(3), atol=1e-15)
    Sp = np.einsum("pa,lb,mc,nd,abcd->plmn", T, T.conj(), T.conj(), T, p.SK)
    assert np.abs(Sp - Sp.transpose(0, 1, 3, 2)).max() > 1e-3 * np.abs(Sp).max()  # m <-> n broken
    fib = O.Fiber(beta, p.SK, p.SR, p.fR, p.hR, p.dt, p.lam0, p.n2, True)
    fibp = O.Fiber(beta, Sp, Sp, p.fR, p.hR, p.dt, p.lam0, p.n2, True)
    A, st = O.mpa_propagate(fib, p.A0, p.L, p.dz, p.M, 0.0, fixed_iters=5)
    Ap, stp = O.mpa_propagate(fibp, T @ p.A0, p.L, p.dz, p.M, 0.0, fixed_iters=5)
    assert st["status"] == stp["status"] == 0
    assert rel(A, p.A0) > 1e-2  # the nonlinearity did something
    assert rel(Ap, T @ A) < 1e-11
