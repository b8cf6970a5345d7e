"""Pins of the oracle's mode overlap tensor S_plmn (Eq. 2) on a grid."""
import numpy as np

import oracle as O
from paper_1708_05324_b300 import inputs as I


def _hg_grid(modes, w, npts=160, extent=5.0):
    x = (np.arange(npts) - npts / 2 + 0.5) * (2 * extent * w / npts)
    dx = x[1] - x[0]
    X, Y = np.meshgrid(x, x, indexing="ij")
    F = np.stack([(I.hg_profile_1d(m, X, w) * I.hg_profile_1d(n, Y, w)).ravel() for m, n in modes])
    return F, dx * dx


def test_fundamental_gaussian_gives_one_over_pi_w2():
    """F = exp(-r^2/w^2): int F^4 / (int F^2)^2 = (pi w^2/4) / (pi w^2/2)^2 = 1/(pi w^2)."""
    w = 10e-6
    F, dA = _hg_grid([(0, 0)], w)
    S = O.overlap_tensor(F, dA)
    assert abs(S[0, 0, 0, 0] * np.pi * w * w - 1.0) < 1e-10


def test_hermite_gauss_grid_sums_match_gauss_hermite_quadrature():
    """On a fine grid the Eq. 2 sums of Hermite-Gauss modes reach the exact
    Gauss-Hermite values (the integrands are Gaussians times polynomials)."""
    w = 10e-6
    modes = I.grin_mode_indices(6)
    F, dA = _hg_grid(modes, w)
    S = O.overlap_tensor(F, dA)
    exact = I.grin_S_gauss_hermite(modes, w)
    assert np.max(np.abs(S - exact)) / np.max(np.abs(exact)) < 1e-10


def test_symmetries_and_scale_invariance():
    rng = np.random.default_rng(3)
    F = rng.standard_normal((4, 300))
    S = O.overlap_tensor(F, 2.5e-12)
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (0, 2, 1, 3)]:
        assert np.allclose(S, S.transpose(perm), rtol=1e-13, atol=0)
    # each profile's own scale cancels in Eq. 2's normalisation
    assert np.allclose(O.overlap_tensor(F * np.array([[2.0], [0.5], [7.0], [1.0]]), 2.5e-12), S, rtol=1e-12)
    # brute force at one index
    nrm = np.sum(F * F, axis=1) * 2.5e-12
    b = np.sum(F[0] * F[1] * F[2] * F[3]) * 2.5e-12 / np.sqrt(np.prod(nrm))
    assert abs(S[0, 1, 2, 3] - b) < 1e-13 * abs(b)
