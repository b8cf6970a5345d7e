"""Pins of the seeded input generators (fiber, modes, coupling tensor, pulses)."""
import itertools
import math

import numpy as np
import pytest

from paper_1708_05324_b300 import inputs as I


def test_splitmix64_reference_vector():
    """First outputs of SplitMix64 for seed 1234567, as produced by the
    reference C implementation of the algorithm."""
    g = I.SplitMix64(1234567)
    assert [g.next_u64() for _ in range(3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


def test_mode_weights_and_pulse_energy():
    w = I.random_mode_weights(6, 2)
    assert np.sum(abs(w) ** 2) == pytest.approx(1.0, abs=1e-15)
    dt = 10e-12 / 8192
    A = I.launch_field(6, 8192, dt, "gaussian", 200e-15, 50e-9, 2)
    assert dt * np.sum(abs(A) ** 2) == pytest.approx(50e-9, rel=1e-14)
    # intensity FWHM of the launched envelope
    p = np.sum(abs(A) ** 2, axis=0)
    above = np.nonzero(p >= p.max() / 2)[0]
    assert (above[-1] - above[0] + 1) * dt == pytest.approx(200e-15, abs=2 * dt)
    assert np.argmax(p) == 8192 // 2


def test_raman_response_normalisation_and_causality():
    dt = 1e-15
    h = I.raman_response(4096, dt)
    assert dt * h.sum() == pytest.approx(1.0, abs=1e-14)
    assert h[0] == 0.0 and h[1] > 0  # causal, starts at t = 0


def test_p15_S_is_fully_permutation_symmetric():
    """Eq. 2's integrand is symmetric in (p, l, m, n): all 24 permutations."""
    modes = I.grin_mode_indices(6)
    S = I.grin_S_grid(modes, I.grin_mode_width(25e-6, 0.2, 1030e-9), 25e-6)
    for perm in itertools.permutations(range(4)):
        np.testing.assert_allclose(S.transpose(perm), S, rtol=0, atol=1e-15 * abs(S).max())


@pytest.mark.parametrize("N,nnz,unique", [(3, 21, 6), (6, 336, 42), (10, 2512, 199), (15, 12717, 819)])
def test_p16_grin_S_closed_form_and_selection_rule(N, nnz, unique):
    """GRIN Hermite-Gauss modes: S_0000 = 1/(pi w^2) (a Gaussian overlap),
    S vanishes unless the x- and y-index sums are both even (parity of the
    Hermite functions), and the 128x128 grid integral of Eq. 2 equals exact
    Gauss-Hermite quadrature."""
    radius, na, lam0 = 25e-6, 0.2, 1030e-9
    w = I.grin_mode_width(radius, na, lam0)
    assert w == pytest.approx(6.40e-6, rel=1e-3)
    modes = I.grin_mode_indices(N)
    Sgh = I.grin_S_gauss_hermite(modes, w)
    assert Sgh[0, 0, 0, 0] == pytest.approx(1 / (math.pi * w * w), rel=1e-14)
    Sgrid = I.grin_S_grid(modes, w, radius)
    assert np.max(abs(Sgrid - Sgh)) < 1e-12 * Sgh.max()
    allowed = np.zeros(Sgh.shape, dtype=bool)
    for idx in itertools.product(range(N), repeat=4):
        sx = sum(modes[i][0] for i in idx)
        sy = sum(modes[i][1] for i in idx)
        allowed[idx] = (sx % 2 == 0) and (sy % 2 == 0)
    assert np.all(abs(Sgh[~allowed]) < 1e-14 * Sgh.max())
    assert int(np.count_nonzero(allowed)) == nnz
    assert int(np.count_nonzero(abs(Sgh) > 1e-12 * Sgh.max())) == nnz
    uniq = {tuple(sorted(i)) for i in zip(*np.nonzero(allowed))}
    assert len(uniq) == unique


def test_grin_mode_groups_are_equally_spaced():
    """Sec. III.A.1: in a parabolic fiber delta beta_0 = n P with one spacing
    P between consecutive mode groups; modes of one group are degenerate."""
    prob = I.workload("C3", Nt=64, dt=20e-12 / 64, L=1e-3)
    c = np.array(prob.extra["coeffs"])
    groups = [m[0] + m[1] for m in prob.extra["modes"]]
    db0 = c[:, 0] - c[0, 0]
    P = db0[1]
    assert -6e3 < P < -5e3
    for g, d in zip(groups, db0):
        assert d == pytest.approx(g * P, rel=2e-3)
    # silica GVD at 1030 nm: beta2 ~ 19 fs^2/mm (normal dispersion)
    assert 17e-27 < c[0, 2] < 21e-27
    # mode-1 frame: the first mode has zero delta beta_0 and delta beta_1
    np.testing.assert_allclose(prob.beta[0, 0], 0.0, atol=1e-9)


def test_p17_step_index_modes_are_orthogonal_on_the_grid():
    """LP modes of the step-index fiber (Sec. III.B.2), solved from the weakly
    guiding characteristic equation, are orthogonal: int F_p F_q ~ 0."""
    radius, na, lam0 = 25e-6, 0.22, 1030e-9
    modes, info = I.step_index_modes(radius, na, lam0, 12)
    assert info["V"] == pytest.approx(33.55, abs=0.05)
    betas = [m["beta"] for m in modes]
    assert all(betas[i] >= betas[i + 1] for i in range(len(betas) - 1))
    npts = 400
    x = (np.arange(npts) - npts / 2 + 0.5) * (3 * radius / npts)
    X, Y = np.meshgrid(x, x, indexing="ij")
    F = np.array([I.step_index_profile(m, radius, X, Y).ravel() for m in modes])
    F /= np.linalg.norm(F, axis=1)[:, None]
    G = F @ F.T
    off = G - np.diag(np.diag(G))
    assert np.max(abs(off)) < 1e-3
    S = I.overlap_tensor_from_profiles(F, (x[1] - x[0]) ** 2)
    for perm in [(1, 0, 2, 3), (2, 1, 0, 3), (3, 1, 2, 0)]:
        np.testing.assert_allclose(S.transpose(perm), S, atol=1e-12 * abs(S).max())
