"""Linear mode coupling C_p = i sum_n Q_np A_n (Sec. IV) on the GPU: the MPA
and the RK4IP comparator with gmmnlse_set_linear_coupling, element by element
against the oracle."""
import functools

import numpy as np
import pytest

import oracle as O
from paper_1708_05324_b300 import inputs as I

pytestmark = pytest.mark.gpu

L, DZ, M, TOL = 1e-3, 1e-4, 5, 1e-13


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def problem(N, Nt, fR):
    return I.grin_problem("lc", N=N, Nt=Nt, dt=2e-12 / Nt, kind="gaussian", fwhm=150e-15, energy=20e-9,
                          L=L, dz=DZ, M=M, tol=TOL, seed=17, fR=fR, s_from="gh")


def coupling(N):
    # not symmetric, so that a transposed Q or a swapped phase shows
    return I.coupling_matrix(N, 40.0, seed=31 + N, symmetric=False)


@functools.lru_cache(maxsize=None)
def oracle_mpa(N, Nt, fR, with_q=True):
    prob = problem(N, Nt, fR)
    fib = O.Fiber.from_problem(prob, Q=coupling(N) if with_q else None)
    return O.mpa_propagate(fib, prob.A0, L, DZ, M, TOL)[0]


@functools.lru_cache(maxsize=None)
def oracle_rk4(N, Nt, fR):
    prob = problem(N, Nt, fR)
    return O.rk4ip_propagate(O.Fiber.from_problem(prob, Q=coupling(N)), prob.A0, L, DZ)


def context(prob, precision):
    from paper_1708_05324_b300 import binding as B
    return B.Context.from_problem(prob, precision=precision, device=0)


CASES = [(1, 128, 0.18), (3, 256, 0.18), (6, 1024, 0.18), (10, 256, 0.18), (15, 256, 0.0)]


@pytest.mark.parametrize("N,Nt,fR", CASES)
@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_mpa_with_linear_coupling_matches_the_oracle(N, Nt, fR, precision, bar):
    from paper_1708_05324_b300 import binding as B
    prob = problem(N, Nt, fR)
    ref = oracle_mpa(N, Nt, fR)
    assert rel(ref, oracle_mpa(N, Nt, fR, False)) > 100 * bar  # the term matters at this bar
    ctx = context(prob, precision)
    try:
        ctx.set_linear_coupling(coupling(N))
        out, _, rc = ctx.propagate(prob.A0, L, DZ, M, TOL)
    finally:
        ctx.close()
    assert rc == B.OK
    assert rel(out, ref) < bar


@pytest.mark.parametrize("N", [10, 15])
def test_linear_coupling_beside_the_tensor_core_contraction(N):
    from paper_1708_05324_b300 import binding as B
    fR = 0.18 if N == 10 else 0.0
    prob = problem(N, 256, fR)
    ctx = context(prob, "bf16")
    try:
        ctx.set_linear_coupling(coupling(N))
        out, _, rc = ctx.propagate(prob.A0, L, DZ, M, TOL)
    finally:
        ctx.close()
    assert rc == B.OK
    assert rel(out, oracle_mpa(N, 256, fR)) < 1e-5


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_rk4ip_with_linear_coupling_matches_the_oracle(precision, bar):
    from paper_1708_05324_b300 import binding as B
    prob = problem(6, 1024, 0.18)
    ctx = context(prob, precision)
    try:
        ctx.set_linear_coupling(coupling(6))
        out, _, rc = ctx.propagate_rk4ip(prob.A0, L, DZ)
    finally:
        ctx.close()
    assert rc == B.OK
    assert rel(out, oracle_rk4(6, 1024, 0.18)) < bar


def test_setting_and_removing_q_between_propagations_retires_the_graphs():
    from paper_1708_05324_b300 import binding as B
    prob = problem(3, 256, 0.18)
    with_q, without = oracle_mpa(3, 256, 0.18), oracle_mpa(3, 256, 0.18, False)
    ctx = context(prob, "fp64")
    try:
        a, _, rc = ctx.propagate(prob.A0, L, DZ, M, TOL)  # builds the graph without the term
        assert rc == B.OK and rel(a, without) < 1e-10
        ctx.set_linear_coupling(coupling(3))
        b, _, rc = ctx.propagate(prob.A0, L, DZ, M, TOL)
        assert rc == B.OK and rel(b, with_q) < 1e-10
        ctx.set_linear_coupling(None)
        c, _, rc = ctx.propagate(prob.A0, L, DZ, M, TOL)
        assert rc == B.OK and rel(c, without) < 1e-10
    finally:
        ctx.close()


def test_linear_coupling_rejections():
    import ctypes as C
    from paper_1708_05324_b300 import binding as B
    prob = problem(3, 256, 0.18)
    ctx = context(prob, "fp32")
    try:
        bad = coupling(3)
        bad[1, 2] = np.inf
        with pytest.raises(B.GmmnlseError):
            ctx.set_linear_coupling(bad)
        ctx.set_linear_coupling(coupling(3))
        import torch
        a0 = torch.from_numpy(prob.A0).cuda()
        out = torch.empty_like(a0)
        st = B.Stats()
        rc = ctx.lib.gmmnlse_propagate_noalloc(ctx.handle, a0.data_ptr(), L, DZ, M, TOL,
                                               out.data_ptr(), C.byref(st))
        assert rc == B.E_UNSUPPORTED
    finally:
        ctx.close()


GAIN = {3: np.array([4.0, -6.0, 9.0]), 6: np.linspace(-8.0, 8.0, 6), 10: np.linspace(-5.0, 12.0, 10)}


@functools.lru_cache(maxsize=None)
def oracle_gain(N, Nt, fR, with_q):
    prob = problem(N, Nt, fR)
    fib = O.Fiber.from_problem(prob, Q=coupling(N) if with_q else None, gain=GAIN[N])
    return O.mpa_propagate(fib, prob.A0, L, DZ, M, TOL)[0], O.rk4ip_propagate(fib, prob.A0, L, DZ)


@pytest.mark.parametrize("N,Nt,fR,with_q", [(3, 256, 0.18, False), (6, 1024, 0.18, True), (10, 256, 0.18, True)])
@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_gain_matches_the_oracle_in_the_mpa_and_rk4ip(N, Nt, fR, with_q, precision, bar):
    from paper_1708_05324_b300 import binding as B
    prob = problem(N, Nt, fR)
    ref_mpa, ref_rk = oracle_gain(N, Nt, fR, with_q)
    assert rel(ref_mpa, oracle_mpa(N, Nt, fR, with_q)) > 100 * bar
    ctx = context(prob, precision)
    try:
        ctx.set_gain(GAIN[N])
        if with_q:
            ctx.set_linear_coupling(coupling(N))
        out, _, rc = ctx.propagate(prob.A0, L, DZ, M, TOL)
        assert rc == B.OK and rel(out, ref_mpa) < bar
        out, _, rc = ctx.propagate_rk4ip(prob.A0, L, DZ)
        assert rc == B.OK and rel(out, ref_rk) < bar
        ctx.set_gain(None)  # back to the coupling alone (or nothing)
        out, _, rc = ctx.propagate(prob.A0, L, DZ, M, TOL)
        assert rc == B.OK and rel(out, oracle_mpa(N, Nt, fR, with_q)) < bar
    finally:
        ctx.close()


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_served_requests_take_the_linear_terms(precision, bar):
    """Server requests build their own graphs from the context: with Q and a
    gain set, each served result equals the oracle, in a mix with a context
    that has neither."""
    import time
    from paper_1708_05324_b300 import binding as B
    pq, p0 = problem(6, 1024, 0.18), problem(3, 256, 0.18)
    cq, c0 = context(pq, precision), context(p0, precision)
    srv = B.Server(hbm_budget=1 << 30, max_inflight=4)
    try:
        cq.set_linear_coupling(coupling(6))
        cq.set_gain(GAIN[6])
        jobs = []
        for _ in range(2):
            jobs.append((srv.submit(cq, pq.A0, L, DZ, M, TOL), 6, 1024, oracle_gain(6, 1024, 0.18, True)[0]))
            jobs.append((srv.submit(c0, p0.A0, L, DZ, M, TOL), 3, 256, oracle_mpa(3, 256, 0.18, False)))
        t0 = time.time()
        left = list(jobs)
        while left:
            for job in list(left):
                t, N, Nt, ref = job
                rc, a, _ = srv.poll(t, N, Nt)
                if rc == B.PENDING:
                    continue
                assert rc == B.OK and rel(a, ref) < bar
                left.remove(job)
            assert time.time() - t0 < 120, "requests did not finish"
            time.sleep(0.002)
    finally:
        srv.close()
        cq.close()
        c0.close()


@pytest.mark.parametrize("mixed", ["fp16", "bf16"])
def test_fp16_scale_follows_an_energy_that_a_gain_raises_tenfold(mixed):
    """MIXED_FP16 scales its tensor-core operands by a power of two from an
    energy bound; with a gain that raises the energy 10x over the fiber
    (exp(2 g L) = 10) a bound taken once at the input would overflow FP16.
    The bound is taken anew at every long step, so the result matches the
    oracle at the mixed-precision bar."""
    from paper_1708_05324_b300 import binding as B
    N, Nt, fR = 10, 256, 0.18
    prob = problem(N, Nt, fR)
    g = np.full(N, np.log(10.0) / (2 * L))
    fib = O.Fiber.from_problem(prob, gain=g)
    ref = O.mpa_propagate(fib, prob.A0, L, DZ, M, TOL)[0]
    e_in = float(np.sum(np.abs(prob.A0) ** 2))
    assert float(np.sum(np.abs(ref) ** 2)) > 9.0 * e_in  # the energy grew about tenfold
    ctx = context(prob, mixed)
    try:
        ctx.set_gain(g)
        out, st, rc = ctx.propagate(prob.A0, L, DZ, M, 1e-9, check=False)
    finally:
        ctx.close()
    assert rc == B.OK
    assert rel(out, ref) < 1e-3


def saturation_for(prob, g):
    """A saturation coefficient that brings the energy's fixed point to about
    five times the input energy (a clearly saturated gain)."""
    W0 = prob.dt * float(np.sum(np.abs(prob.A0) ** 2))
    return 0.2 * float(np.max(g)) / (prob.SK[0, 0, 0, 0] * W0)


@functools.lru_cache(maxsize=None)
def oracle_saturated(N, Nt, fR, with_profile):
    prob = problem(N, Nt, fR)
    g = GAIN.get(N, np.full(N, 6.0)) + 40.0
    sat = saturation_for(prob, g)
    kw = dict(gain=g, sat=sat)
    if with_profile:
        kw.update(Q=coupling(N), Q_profile=PROFILE, Q_profile_dz=PROFILE_DZ)
    fib = O.Fiber.from_problem(prob, **kw)
    return (O.mpa_propagate(fib, prob.A0, L, DZ, M, TOL)[0], O.rk4ip_propagate(fib, prob.A0, L, DZ), g, sat,
            O.mpa_propagate(O.Fiber.from_problem(prob, gain=g), prob.A0, L, DZ, M, TOL)[0])


# a grating-like profile of the coupling: f(z) = 1 + 0.8 sin(2 pi z / 0.4 mm)
PROFILE_DZ = 2e-5
PROFILE = 1.0 + 0.8 * np.sin(2 * np.pi * np.arange(80) * PROFILE_DZ / 4e-4)


@pytest.mark.parametrize("N,Nt,fR,with_profile", [(1, 128, 0.18, False), (3, 256, 0.18, True),
                                                  (10, 256, 0.18, True)])
@pytest.mark.parametrize("precision,bar", [("fp64", 1e-10), ("fp32", 1e-5), ("bf16", 1e-3)])
def test_saturated_gain_matches_the_oracle_in_the_mpa_and_rk4ip(N, Nt, fR, with_profile, precision, bar):
    """The saturation (per substep: FP64 time integrals of the pair
    products, R = S^R Ubar, the term in the integrand) beside the small-signal
    gain, with a z-dependent linear coupling Q f(z) for 3 and 10 modes (the
    MPA takes f at every substep, RK4IP at its stage positions); 10 modes in
    BF16 run the contraction on the tensor cores."""
    from paper_1708_05324_b300 import binding as B
    prob = problem(N, Nt, fR)
    ref_mpa, ref_rk, g, sat, unsat = oracle_saturated(N, Nt, fR, with_profile)
    assert rel(ref_mpa, unsat) > 1e-3  # the saturation changes the field
    ctx = context(prob, precision)
    tol = TOL if precision == "fp64" else 1e-9
    try:
        ctx.set_gain(g)
        ctx.set_gain_saturation(sat)
        if with_profile:
            ctx.set_linear_coupling(coupling(N))
            ctx.set_coupling_profile(PROFILE, PROFILE_DZ)
        out, _, rc = ctx.propagate(prob.A0, L, DZ, M, tol)
        assert rc == B.OK and rel(out, ref_mpa) < bar
        out, _, rc = ctx.propagate_rk4ip(prob.A0, L, DZ)
        assert rc == B.OK and rel(out, ref_rk) < bar
        # removing the saturation and the profile (and Q) gives the gain alone
        ctx.set_gain_saturation(0.0)
        ctx.set_coupling_profile(None)
        ctx.set_linear_coupling(None)
        out, _, rc = ctx.propagate(prob.A0, L, DZ, M, tol)
        assert rc == B.OK and rel(out, unsat) < bar
    finally:
        ctx.close()


def test_profile_and_saturation_rejections():
    from paper_1708_05324_b300 import binding as B
    prob = problem(3, 256, 0.18)
    ctx = context(prob, "fp32")
    try:
        for bad in (-1.0, float("inf"), float("nan")):
            with pytest.raises(B.GmmnlseError):
                ctx.set_gain_saturation(bad)
        with pytest.raises(B.GmmnlseError):
            ctx.set_coupling_profile(np.array([1.0, np.nan]), 1e-4)
        with pytest.raises(B.GmmnlseError):
            ctx.set_coupling_profile(np.array([1.0, 2.0]), 0.0)
    finally:
        ctx.close()
