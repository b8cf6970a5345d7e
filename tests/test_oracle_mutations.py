"""Planted mistakes in the oracle must be caught by the pins.

Each case rewrites one line of oracle/gmmnlse.py (on the CPU, in a fresh
module object), swaps the mutated functions into the `oracle` package for the
duration of the case, and runs every pin of tests/test_oracle_pins.py.  At
least one pin must fail, otherwise the pins would not distinguish that
plausible mistake from the paper's method.
"""
import os
import types
import warnings

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "gmmnlse.py")

MUTATIONS = {
    "fourier_sign_swapped": [
        ("return np.fft.ifft(a, axis=-1) * a.shape[-1]", "return np.fft.fft(a, axis=-1)"),
        ("return np.fft.fft(af, axis=-1) / af.shape[-1]", "return np.fft.ifft(af, axis=-1)"),
    ],
    "forward_scale_dropped": [
        ("return np.fft.ifft(a, axis=-1) * a.shape[-1]", "return np.fft.ifft(a, axis=-1)"),
    ],
    "trapezoid_weight": [
        ("acc = acc + 0.5 * dz * (I[j - 1] + I[j])", "acc = acc + dz * (I[j - 1] + I[j])"),
    ],
    "left_rectangle_rule": [
        ("acc = acc + 0.5 * dz * (I[j - 1] + I[j])", "acc = acc + dz * I[j - 1]"),
    ],
    "integrand_phase_sign": [
        ("return nonlinear_operator(fib, psi_j * E, z0 + zrel) * np.conj(E)",
         "return nonlinear_operator(fib, psi_j * E, z0 + zrel) * E"),
    ],
    "interaction_picture_phase_dropped": [
        ("return nonlinear_operator(fib, psi_j * E, z0 + zrel) * np.conj(E)",
         "return nonlinear_operator(fib, psi_j, z0 + zrel) * np.conj(E)"),
    ],
    "substep_index_shift": [
        ("zrel = [j * dz for j in range(M + 1)]", "zrel = [(j + 1) * dz for j in range(M + 1)]"),
    ],
    "long_step_phase_dropped": [
        ("return psi[M] * phase_factor(fib, zrel[M]), n, trace, status",
         "return psi[M], n, trace, status"),
    ],
    "conjugate_on_wrong_field": [
        ("return A[:, None, :] * np.conj(A)[None, :, :]", "return np.conj(A)[:, None, :] * A[None, :, :]"),
    ],
    "kerr_tensor_transposed": [
        ("T = (np.asarray(SK).reshape(N * N, N * N) @ Q).reshape(N, N, -1)  # T[p,l,t]",
         "T = (np.asarray(SK).transpose(0, 3, 2, 1).reshape(N * N, N * N) @ Q).reshape(N, N, -1)"),
    ],
    "complex_coupling_dropped": [
        ("return S.astype(np.complex128) if np.iscomplexobj(S) else S.astype(np.float64)",
         "return np.real(S).astype(np.float64)"),
    ],
    "complex_coupling_conjugated": [
        ("return S.astype(np.complex128) if np.iscomplexobj(S) else S.astype(np.float64)",
         "return np.conj(S).astype(np.complex128) if np.iscomplexobj(S) else S.astype(np.float64)"),
    ],
    "raman_acausal": [
        ("return dt * np.fft.ifft(np.fft.fft(h) * np.fft.fft(q, axis=-1), axis=-1)",
         "return dt * np.fft.ifft(np.conj(np.fft.fft(h)) * np.fft.fft(q, axis=-1), axis=-1)"),
    ],
    "raman_fraction_not_removed_from_kerr": [
        ("out = (1.0 - fib.fR) * kerr_sum(fib.SK, A)", "out = kerr_sum(fib.SK, A)"),
    ],
    "self_steepening_sign": [
        ("self.shock = (1.0 + self.omega / self.omega0) if self.self_steepening",
         "self.shock = (1.0 - self.omega / self.omega0) if self.self_steepening"),
    ],
    "gamma_missing_omega0": [
        ("self.gamma0 = self.n2 * self.omega0 / C_LIGHT", "self.gamma0 = self.n2 * 1.8e15 / C_LIGHT * 1.01"),
    ],
    "nonlinear_sign": [
        ("out = 1j * fib.gamma0 * fib.shock * freq_from_time(NL)",
         "out = -1j * fib.gamma0 * fib.shock * freq_from_time(NL)"),
    ],
    "eps_not_relative": [
        ("eps = math.sqrt(diff / size) if (finite and size > 0)", "eps = math.sqrt(diff) if (finite and size > 0)"),
    ],
    "initial_integrand_reused": [
        ("I[0] = integrand(fib, psi0, zrel[0], z0)", "I[0] = 0.0 * psi0"),
    ],
}

PIN_TESTS = [getattr(pins, name) for name in dir(pins) if name.startswith("test_")
             and callable(getattr(pins, name))]


def _mutated_module(edits):
    src = open(SRC).read()
    for old, new in edits:
        assert old in src, f"mutation target vanished from the oracle: {old!r}"
        src = src.replace(old, new)
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = SRC
    exec(compile(src, SRC, "exec"), mod.__dict__)
    return mod


def _run_pin(fn):
    import inspect
    params = inspect.signature(fn).parameters
    if not params:
        fn()
        return
    # parametrised pins: run every parameter set recorded on the function
    marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
    names = [s.strip() for s in marks[0].args[0].split(",")]
    for values in marks[0].args[1]:
        fn(**dict(zip(names, values if isinstance(values, tuple) else (values,))))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    mod = _mutated_module(MUTATIONS[name])
    for attr in dir(oracle):
        if not attr.startswith("_") and hasattr(mod, attr) and attr != "gmmnlse":
            monkeypatch.setattr(oracle, attr, getattr(mod, attr))
    monkeypatch.setattr(oracle, "gmmnlse", mod)
    caught = []
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        with np.errstate(all="ignore"):
            for fn in PIN_TESTS:
                try:
                    _run_pin(fn)
                except Exception as e:  # AssertionError, or a blow-up
                    caught.append((fn.__name__, type(e).__name__))
    assert caught, f"no pin detects the planted mistake {name!r}"


# Planted mistakes in the added right-hand-side terms of Sec. IV (mode
# coupling with its longitudinal profile, gain and its saturation), run
# against the pins of tests/test_oracle_coupling.py.
import test_oracle_coupling as coupling_pins  # noqa: E402

Q_LINE = "out = out + 1j * coupling_factor(fib, z) * (fib.Q.T @ Aw)"
COUPLING_MUTATIONS = {
    "coupling_transposed": [(Q_LINE, "out = out + 1j * coupling_factor(fib, z) * (fib.Q @ Aw)")],
    "coupling_sign": [(Q_LINE, "out = out - 1j * coupling_factor(fib, z) * (fib.Q.T @ Aw)")],
    "gain_on_the_wrong_modes": [("out = out + fib.gain[:, None] * Aw", "out = out + fib.gain[::-1, None] * Aw")],
    "saturation_sign": [("out = out - fib.sat * freq_from_time(saturation_term(fib, At))",
                         "out = out + fib.sat * freq_from_time(saturation_term(fib, At))")],
    "saturation_integral_without_dt": [("E = fib.dt * (A @ np.conj(A).T)", "E = A @ np.conj(A).T")],
    "saturation_on_the_kerr_tensor": [("SR = fib.SK if fib.SR is None else fib.SR", "SR = fib.SK")],
    "profile_taken_at_the_long_step_origin": [
        ("return nonlinear_operator(fib, psi_j * E, z0 + zrel) * np.conj(E)",
         "return nonlinear_operator(fib, psi_j * E, z0) * np.conj(E)")],
    "rk4ip_midpoint_stage_at_the_step_start": [
        ("k2 = Nop(AI + 0.5 * h * k1, z + 0.5 * h)", "k2 = Nop(AI + 0.5 * h * k1, z)")],
}

COUPLING_PIN_TESTS = [getattr(coupling_pins, name) for name in dir(coupling_pins)
                      if name.startswith("test_") and callable(getattr(coupling_pins, name))]


@pytest.mark.parametrize("name", sorted(COUPLING_MUTATIONS))
def test_planted_mistake_in_an_added_term_is_caught(name, monkeypatch):
    mod = _mutated_module(COUPLING_MUTATIONS[name])
    for attr in dir(oracle):
        if not attr.startswith("_") and hasattr(mod, attr) and attr != "gmmnlse":
            monkeypatch.setattr(oracle, attr, getattr(mod, attr))
    monkeypatch.setattr(oracle, "gmmnlse", mod)
    caught = []
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        with np.errstate(all="ignore"):
            for fn in COUPLING_PIN_TESTS:
                try:
                    _run_pin(fn)
                except Exception as e:
                    caught.append((fn.__name__, type(e).__name__))
    assert caught, f"no pin detects the planted mistake {name!r}"
