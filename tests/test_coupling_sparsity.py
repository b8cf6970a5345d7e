"""The structure of the graded-index Hermite-Gaussian coupling that the
compiled nonzero-list contraction (N <= 8) relies on: the overlap integral
of Eq. 2 factorises into x and y integrals of products of four Hermite-
Gaussians, each of which vanishes when the four indices sum to an odd number
(an odd integrand), so S_plmn = 0 unless the x parities and the y parities of
the four modes each sum to an even number.  In the reduced matrix
G[(p,l)][(m,n)] that makes the rows and columns fall into four parity
classes, with zeros between different classes."""
import numpy as np
import pytest

from paper_1708_05324_b300 import inputs as I


def reduced(S, N):
    pairs = [(p, l) for p in range(N) for l in range(p, N)]
    return pairs, np.array([[S[p, l, m, n] for (m, n) in pairs] for (p, l) in pairs])


@pytest.mark.parametrize("N,nnz", [(3, 12), (6, 129), (8, 346)])
def test_grin_coupling_is_block_diagonal_by_parity(N, nnz):
    modes = I.grin_mode_indices(N)
    S = I.grin_S_gauss_hermite(modes, I.grin_mode_width(25e-6, 0.2, 1030e-9))
    pairs, G = reduced(S, N)
    tiny = 1e-12 * np.abs(G).max()
    cls = [((modes[a][0] + modes[b][0]) % 2, (modes[a][1] + modes[b][1]) % 2) for a, b in pairs]
    for r in range(len(pairs)):
        for k in range(len(pairs)):
            if cls[r] != cls[k]:
                assert abs(G[r, k]) <= tiny, (pairs[r], pairs[k], G[r, k])
    # every entry inside a class block is nonzero for these modes: the count
    # is the sum of the squared class sizes
    sizes = {}
    for c in cls:
        sizes[c] = sizes.get(c, 0) + 1
    assert sum(v * v for v in sizes.values()) == nnz
    assert int((np.abs(G) > tiny).sum()) == nnz
