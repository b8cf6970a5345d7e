"""gmmnlse_overlap_tensor (Eq. 2 on the GPU) against the oracle's grid sums."""
import numpy as np
import pytest

import oracle as O
from paper_1708_05324_b300 import inputs as I

pytestmark = pytest.mark.gpu


def maxrel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("N,G", [(1, 1), (3, 17), (12, 1001), (13, 4096)])
def test_overlap_tensor_matches_the_oracle_on_ragged_sizes(N, G):
    """K = N(N+1)/2 pair rows across one or two 64-row tiles, grid cells
    not a multiple of the 16-cell chunk."""
    from paper_1708_05324_b300 import binding as B
    F = np.random.default_rng(N * 7 + G).standard_normal((N, G))
    S = B.overlap_tensor(F, 3.0e-12)
    assert maxrel(S, O.overlap_tensor(F, 3.0e-12)) < 1e-12


def test_overlap_tensor_of_hermite_gauss_modes():
    from paper_1708_05324_b300 import binding as B
    w = 10e-6
    modes = I.grin_mode_indices(10)
    x = (np.arange(160) - 80 + 0.5) * (10 * w / 160)
    X, Y = np.meshgrid(x, x, indexing="ij")
    F = np.stack([(I.hg_profile_1d(m, X, w) * I.hg_profile_1d(n, Y, w)).ravel() for m, n in modes])
    S = B.overlap_tensor(F, (x[1] - x[0]) ** 2)
    assert maxrel(S, O.overlap_tensor(F, (x[1] - x[0]) ** 2)) < 1e-12
    assert maxrel(S, I.grin_S_gauss_hermite(modes, w)) < 1e-10
    for perm in [(1, 0, 2, 3), (2, 3, 0, 1), (0, 2, 1, 3)]:
        assert maxrel(S, S.transpose(perm)) < 1e-13


def test_overlap_tensor_of_the_42_mode_step_index_fiber_on_400x400():
    """The 42-mode setup: 903 pair rows (15 tiles, ragged) over 160000 cells;
    sampled entries against the oracle one by one."""
    from paper_1708_05324_b300 import binding as B
    radius, npts, extent = 25e-6, 400, 1.5
    modes, _ = I.step_index_modes(radius, 0.22, 1030e-9, 42)
    x = (np.arange(npts) - npts / 2 + 0.5) * (2 * extent * radius / npts)
    X, Y = np.meshgrid(x, x, indexing="ij")
    F = np.array([I.step_index_profile(m, radius, X, Y).ravel() for m in modes])
    dA = (x[1] - x[0]) ** 2
    S = B.overlap_tensor(F, dA)
    rng = np.random.default_rng(5)
    idx = [tuple(rng.integers(0, 42, 4)) for _ in range(24)] + [(0, 0, 0, 0), (41, 41, 41, 41), (3, 17, 29, 40)]
    scale = np.max(np.abs(S))
    for p, l, m, n in idx:
        ref = O.overlap_tensor(F[[p, l, m, n]], dA)[0, 1, 2, 3]
        assert abs(S[p, l, m, n] - ref) < 1e-12 * scale
    assert maxrel(S, S.transpose(2, 3, 0, 1)) < 1e-13


def test_overlap_tensor_rejections():
    from paper_1708_05324_b300 import binding as B
    F = np.ones((3, 10))
    F[1, 4] = np.nan
    with pytest.raises(B.GmmnlseError):
        B.overlap_tensor(F, 1e-12)
    F = np.ones((3, 10))
    F[2] = 0.0
    with pytest.raises(B.GmmnlseError):
        B.overlap_tensor(F, 1e-12)
