"""The general coupling on the GPU (gmmnlse_create_general): complex S^K and
S^R with no symmetry (Eq. 1 without the real, single-polarization S of
Eq. 2), element by element against the oracle, which sums S_plmn A_m A_n^*
over every (m, n) as written."""
import functools
import math

import numpy as np
import pytest

import oracle as O
from paper_1708_05324_b300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-13


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def mixed_basis(N=3, Nt=256, fR=0.18):
    """A GRIN problem whose degenerate HG10 / HG01 pair is rotated into the
    complex modes (HG10 +- i HG01)/sqrt(2): S' = T S T^* T^* T, complex and
    unsymmetric in m <-> n; returns (problem with beta made exactly
    degenerate on the pair, S', T)."""
    p = I.grin_problem("gx", N=N, Nt=Nt, dt=20e-15, kind="gaussian", fwhm=300e-15, energy=20e-9,
                       L=2e-3, dz=1e-4, M=5, tol=TOL, seed=2, fR=fR, s_from="gh")
    p.beta[2] = p.beta[1]
    r = 1.0 / math.sqrt(2.0)
    T = np.eye(N, dtype=complex)
    T[1:3, 1:3] = [[r, 1j * r], [r, -1j * r]]
    Sp = np.einsum("pa,lb,mc,nd,abcd->plmn", T, T.conj(), T.conj(), T, p.SK)
    return p, Sp, T


def random_complex(N, Nt, fR, seed, separate_raman):
    """A GRIN problem with random complex unsymmetric S^K (and S^R when
    separate_raman) of the size of its real S."""
    p = I.grin_problem("gr", N=N, Nt=Nt, dt=2e-12 / Nt, kind="gaussian", fwhm=150e-15, energy=10e-9,
                       L=1e-3, dz=1e-4, M=5, tol=TOL, seed=seed, fR=fR, s_from="gh")
    rng = np.random.default_rng(seed)
    s0 = float(np.abs(p.SK).max())

    def draw():
        return s0 * (rng.uniform(-0.5, 1.0, (N,) * 4) + 0.3j * rng.standard_normal((N,) * 4))

    SK = draw()
    SR = draw() if separate_raman else SK
    return p, SK, SR


def context(p, SK, SR, precision):
    from paper_1708_05324_b300 import binding as B
    return B.Context(p.N, p.Nt, p.dt, p.lam0, p.n2, p.beta, SK, None if SR is SK else SR, p.fR,
                     p.hR if p.fR else None, p.self_steepening, precision, device=0)


@functools.lru_cache(maxsize=None)
def oracle_mixed(fixed):
    p, Sp, T = mixed_basis()
    fib = O.Fiber(p.beta, Sp, Sp, p.fR, p.hR, p.dt, p.lam0, p.n2, True)
    return O.mpa_propagate(fib, T @ p.A0, p.L, p.dz, p.M, 0.0 if fixed else TOL, fixed_iters=fixed)[0]


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_complex_mode_basis_matches_the_oracle(precision, bar):
    """S complex through a unitary mixing of a degenerate pair, with Raman and
    self-steepening: the GPU result equals the oracle's in the mixed basis,
    and T times the real-basis GPU result."""
    p, Sp, T = mixed_basis()
    ref = oracle_mixed(0)
    ctx = context(p, Sp, Sp, precision)
    try:
        out, st, rc = ctx.propagate(T @ p.A0, p.L, p.dz, p.M, TOL if precision == "fp64" else 1e-9)
        assert rc == 0 and st["z"] == pytest.approx(p.L)
        assert rel(out, ref) < bar
    finally:
        ctx.close()
    real = context(p, p.SK, p.SK, precision)
    try:
        A, _, _ = real.propagate(p.A0, p.L, p.dz, p.M, TOL if precision == "fp64" else 1e-9)
        assert rel(out, T @ A) < 10 * bar
    finally:
        real.close()


CASES = [(2, 128, 0.0, False), (4, 256, 0.18, False), (4, 256, 0.18, True), (10, 256, 0.18, True)]


@functools.lru_cache(maxsize=None)
def oracle_random(N, Nt, fR, sep):
    p, SK, SR = random_complex(N, Nt, fR, 40 + N, sep)
    fib = O.Fiber(p.beta, SK, SR, p.fR, p.hR, p.dt, p.lam0, p.n2, True)
    return O.mpa_propagate(fib, p.A0, p.L, p.dz, p.M, TOL)[0]


@pytest.mark.parametrize("N,Nt,fR,sep", CASES)
@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_random_complex_coupling_matches_the_oracle(N, Nt, fR, sep, precision, bar):
    """Random complex S^K (Kerr only, and with Raman), and a separate random
    complex S^R: the GPU MPA against the oracle's."""
    p, SK, SR = random_complex(N, Nt, fR, 40 + N, sep)
    ref = oracle_random(N, Nt, fR, sep)
    assert rel(ref, p.A0) > 1e-3  # the nonlinearity shows at this bar
    ctx = context(p, SK, SR, precision)
    try:
        out, st, rc = ctx.propagate(p.A0, p.L, p.dz, p.M, TOL if precision == "fp64" else 1e-9)
        assert rc == 0
        assert rel(out, ref) < bar
    finally:
        ctx.close()


def test_real_symmetric_coupling_through_the_general_path():
    """A real, symmetric S given as complex takes the general path and
    gives what gmmnlse_create's symmetric path gives."""
    p = I.grin_problem("gs", N=6, Nt=512, dt=4e-15, kind="gaussian", fwhm=150e-15, energy=15e-9,
                       L=1e-3, dz=1e-4, M=5, tol=TOL, seed=5, fR=0.18, s_from="gh")
    a = context(p, p.SK.astype(complex), p.SK.astype(complex), "fp64")
    b = context(p, p.SK, p.SK, "fp64")
    try:
        x = a.propagate(p.A0, p.L, p.dz, p.M, TOL)[0]
        y = b.propagate(p.A0, p.L, p.dz, p.M, TOL)[0]
        assert rel(x, y) < 1e-12
    finally:
        a.close()
        b.close()


def test_rk4ip_with_complex_coupling_matches_the_oracle():
    p, SK, SR = random_complex(4, 256, 0.18, 44, True)
    fib = O.Fiber(p.beta, SK, SR, p.fR, p.hR, p.dt, p.lam0, p.n2, True)
    ref = O.rk4ip_propagate(fib, p.A0, p.L, p.dz)
    ctx = context(p, SK, SR, "fp64")
    try:
        out, st, rc = ctx.propagate_rk4ip(p.A0, p.L, p.dz)
        assert rc == 0
        assert rel(out, ref) < 1e-10
    finally:
        ctx.close()


def test_packed_requests_with_complex_coupling():
    """Requests on a general context through the server (packed): each equals
    the same propagation alone."""
    from paper_1708_05324_b300 import binding as B
    p, SK, SR = random_complex(4, 256, 0.18, 46, True)
    ctx = context(p, SK, SR, "fp64")
    try:
        reqs = [(p.A0 * (1 + 0.1 * k), (2 + k) * p.M * p.dz) for k in range(4)]
        alone = [ctx.propagate(A0, L, p.dz, p.M, TOL)[0] for A0, L in reqs]
        srv = B.Server(hbm_budget=2 << 30, max_inflight=4)
        tickets = [srv.submit(ctx, A0, L, p.dz, p.M, TOL) for A0, L in reqs]
        got = {}
        while len(got) < len(tickets):
            for t in tickets:
                if t not in got:
                    rc, a, st = srv.poll(t, p.N, p.Nt)
                    if rc != B.PENDING:
                        got[t] = (rc, a)
        srv.close()
        for t, ref in zip(tickets, alone):
            assert got[t][0] == B.OK
            assert rel(got[t][1], ref) < 1e-12
    finally:
        ctx.close()


def test_general_coupling_rejections():
    from paper_1708_05324_b300 import binding as B
    p, SK, SR = random_complex(4, 256, 0.18, 47, False)
    with pytest.raises(B.GmmnlseError) as e:
        context(p, SK, SR, "bf16")
    assert e.value.status == B.E_UNSUPPORTED
    ctx = context(p, SK, SR, "fp64")
    try:
        with pytest.raises(B.GmmnlseError) as e:
            ctx.set_gain_saturation(0.1)
        assert e.value.status == B.E_UNSUPPORTED
    finally:
        ctx.close()
