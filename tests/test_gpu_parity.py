"""CUDA path (through the C ABI) against the CPU FP64 oracle.

Bars (relative L2 over all modes and samples): FP64 <= 1e-10, FP32 <= 1e-5.
Sizes span several FFT passes (the leading radix-2/4/8 pass and radix-16
passes), odd pair counts, a separate Raman tensor, ragged long steps and the
largest transform (Nt = 2^14).
"""
import functools
import math

import numpy as np
import pytest

import oracle as O
from paper_1708_05324_b300 import binding as B
from paper_1708_05324_b300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_run(prob, precision, L=None, dz=None, M=None, tol=None, **kw):
    ctx = B.Context.from_problem(prob, precision=precision, **{k: v for k, v in kw.items()
                                                              if k in ("max_iter", "fixed_iters")})
    try:
        out, st, rc = ctx.propagate(prob.A0, L or prob.L, dz or prob.dz, M or prob.M,
                                    prob.tol if tol is None else tol, check=False)
    finally:
        ctx.close()
    return out, st, rc


def oracle_run(prob, L=None, dz=None, M=None, tol=None, **kw):
    fib = O.Fiber.from_problem(prob)
    return O.mpa_propagate(fib, prob.A0, L or prob.L, dz or prob.dz, M or prob.M,
                           prob.tol if tol is None else tol, **kw)


@functools.lru_cache(maxsize=None)
def small(name, N, Nt, fR, ss=1, seed=11, energy=20e-9, split_raman=False):
    prob = I.grin_problem(name, N=N, Nt=Nt, dt=2e-12 / Nt, kind="gaussian", fwhm=150e-15,
                          energy=energy, L=2e-3, dz=1e-4, M=5, tol=1e-13, seed=seed, fR=fR,
                          self_steepening=ss, s_from="gh")
    if split_raman:
        # a different (still fully symmetric) Raman tensor: S^R = 0.7 S^K + 0.3 S_iso
        iso = np.zeros_like(prob.SK)
        for p in range(N):
            iso[p, p, p, p] = prob.SK[0, 0, 0, 0]
        prob.SR = 0.7 * prob.SK + 0.3 * iso
    return prob


@functools.lru_cache(maxsize=None)
def oracle_small(key):
    prob = small(*key)
    return oracle_run(prob)


# ----------------------------------------------------------------------------
def test_linear_propagation_fp64_matches_oracle():
    """n2 = 0: the output is the input times exp(i beta L), with beta L ~ 1e4
    rad at the grid edge; dz = 2^-10 m and M = 8 make every z_j exact."""
    lin = I.grin_problem("lin", N=3, Nt=256, dt=2e-12 / 256, kind="gaussian", fwhm=150e-15,
                         energy=20e-9, L=0.1, dz=2.0 ** -10, M=8, tol=1e-13, seed=11, s_from="gh")
    lin.n2 = 0.0
    L = 100 * 8 * 2.0 ** -10
    out, st, rc = gpu_run(lin, "fp64", L=L)
    assert rc == B.OK and st["iters_max"] == 1
    ref, _ = O.mpa_propagate(O.Fiber.from_problem(lin), lin.A0, L, 2.0 ** -10, 8, 1e-13)
    assert rel(out, ref) < 1e-12


@pytest.fixture(params=["one_block", "cluster"])
def fft_variant(request, monkeypatch):
    """Run with one block per transform (default) and with transforms of small
    launches spread over 2- or 4-block clusters (GMMNLSE_CLUSTER_FFT=1)."""
    if request.param == "cluster":
        monkeypatch.setenv("GMMNLSE_CLUSTER_FFT", "1")
    return request.param


@pytest.mark.parametrize("Nt", [16, 32, 64, 128, 1024])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_every_fft_pass_structure(Nt, precision, fft_variant):
    """Nt = 16 (one radix-16 pass), 32/64/128 (leading radix 2/4/8), 1024."""
    key = ("p", 3, Nt, 0.18)
    prob = small(*key)
    ref, sref = oracle_small(key)
    out, st, rc = gpu_run(prob, precision, tol=1e-13 if precision == "fp64" else 1e-9)
    assert rc == B.OK
    assert rel(out, ref) < TOL[precision]


@pytest.mark.parametrize("N,fR,ss,split", [(1, 0.0, 1, False), (1, 0.18, 0, False), (2, 0.18, 1, False),
                                           (4, 0.0, 0, False), (4, 0.18, 1, True), (6, 0.18, 1, False)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_modes_raman_and_steepening_variants(N, fR, ss, split, precision, fft_variant):
    key = ("v", N, 256, fR, ss, 11, 20e-9, split)
    prob = small(*key)
    ref, sref = oracle_small(key)
    out, st, rc = gpu_run(prob, precision, tol=1e-13 if precision == "fp64" else 1e-9)
    assert rc == B.OK
    assert rel(out, ref) < TOL[precision]
    if precision == "fp64":
        assert st["iters_total"] == sum(sref["iters"])


@pytest.mark.parametrize("N,Nt,fR,split", [(10, 256, 0.18, False), (15, 256, 0.18, False), (10, 64, 0.18, True),
                                            (15, 32, 0.0, False), (9, 128, 0.18, False)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tiled_contraction_many_modes(N, Nt, fR, split, precision):
    """N > 8 takes the tiled CUDA-core contraction (mode groups 0-3 and 0-4
    of the GRIN fiber, as in the 15-mode workload).  Nt = 64 and 32 make the
    128-point (FP32) and 64-point (FP64) tiles straddle substeps, so the z0
    points of later iterations are skipped point by point; the separate
    Raman tensor and the Kerr-only case cover the other two forms of V."""
    key = ("m", N, Nt, fR, 1, 11, 20e-9, split)
    prob = small(*key)
    ref, _ = oracle_small(key)
    out, st, rc = gpu_run(prob, precision, tol=1e-13 if precision == "fp64" else 1e-9)
    assert rc == B.OK
    assert rel(out, ref) < TOL[precision]


def test_ragged_last_long_step_and_M1():
    key = ("p", 3, 128, 0.18)
    prob = small(*key)
    for L, M in ((2.3e-3, 5), (7e-4, 1), (1.2e-3, 7)):
        ref, sref = oracle_run(prob, L=L, M=M)
        out, st, rc = gpu_run(prob, "fp64", L=L, M=M)
        assert rc == B.OK
        assert rel(out, ref) < 1e-10
        assert st["long_steps"] == len(sref["iters"])
        assert st["z"] == pytest.approx(L, rel=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_largest_transform_2_14(precision, fft_variant):
    """Nt = 2^14; in FP64 every transform of the iterates spans a 4-block cluster."""
    prob = I.grin_problem("big", N=2, Nt=16384, dt=20e-12 / 16384, kind="gaussian", fwhm=300e-15,
                          energy=50e-9, L=5e-4, dz=2.5e-5, M=10, tol=1e-13, seed=3, fR=0.18, s_from="gh")
    ref, _ = oracle_run(prob)
    out, st, rc = gpu_run(prob, precision, tol=1e-9)
    assert rc == B.OK
    assert rel(out, ref) < TOL[precision]


@functools.lru_cache(maxsize=None)
def ten_modes_8192():
    prob = I.grin_problem("m10", N=10, Nt=8192, dt=10e-12 / 8192, kind="gaussian", fwhm=200e-15,
                          energy=30e-9, L=30 * 2e-5, dz=2e-5, M=30, tol=1e-13, seed=5, fR=0.18, s_from="gh")
    ref, _ = oracle_run(prob, fixed_iters=3)
    return prob, ref


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("dense", [False, True])
def test_8192_point_transforms_at_32_per_thread(precision, dense, monkeypatch):
    """10 modes x 31 substeps: K1, K2 (pair products, or the rows of Z) and K4
    launch at least two blocks per SM, so their 8192-point transforms take
    32 elements per thread and the 32 x 16 x 16 schedule."""
    if dense:
        monkeypatch.setenv("GMMNLSE_DENSE", "1")
    prob, ref = ten_modes_8192()
    out, st, rc = gpu_run(prob, precision, fixed_iters=3)
    assert rc == B.OK
    assert (st["coupling_rank"] == 55) == dense
    assert rel(out, ref) < TOL.get(precision, 1e-3)


@functools.lru_cache(maxsize=None)
def c2_prefix():
    prob = I.workload("C2", L=4 * 10 * 25e-6)  # 4 long steps of the 0.5 m run
    ref, sref = oracle_run(prob, tol=1e-13)
    return prob, ref, sref


def test_c2_prefix_fp64():
    """Kerr + Raman, N = 6, Nt = 2^13: the benchmark workload, 4 long steps."""
    prob, ref, sref = c2_prefix()
    out, st, rc = gpu_run(prob, "fp64", tol=1e-13)
    assert rc == B.OK
    assert rel(out, ref) < 1e-10
    assert st["long_steps"] == 4


def test_c2_prefix_fp32(fft_variant):
    prob, ref, sref = c2_prefix()
    out, st, rc = gpu_run(prob, "fp32", tol=1e-8)
    assert rc == B.OK
    assert rel(out, ref) < 1e-5


def test_c1_full_length_fp64():
    """Kerr only, N = 3, Nt = 2^10, 5 cm in 20 long steps of M = 5."""
    prob = I.workload("C1")
    ref, sref = oracle_run(prob)
    out, st, rc = gpu_run(prob, "fp64")
    assert rc == B.OK
    assert rel(out, ref) < 1e-10
    assert st["long_steps"] == 20
    assert st["iters_total"] == sum(sref["iters"])


# ----------------------------------------------------------------------------
def test_not_converged_returns_field_of_last_completed_step():
    prob = small("p", 3, 128, 0.18)
    out, st, rc = gpu_run(prob, "fp64", tol=1e-300, max_iter=2)
    assert rc == B.E_NOT_CONVERGED
    assert st["z"] == 0.0 and st["long_steps"] == 0
    assert rel(out, prob.A0) < 1e-14


def test_nonfinite_input_is_rejected():
    prob = small("p", 3, 128, 0.18)
    bad = prob.A0.copy()
    bad[1, 7] = np.nan
    ctx = B.Context.from_problem(prob, precision="fp32")
    _, _, rc = ctx.propagate(bad, prob.L, prob.dz, prob.M, 1e-8, check=False)
    ctx.close()
    assert rc == B.E_INVALID


def test_fixed_iterations_match_oracle():
    key = ("p", 3, 256, 0.18)
    prob = small(*key)
    ref, sref = oracle_run(prob, fixed_iters=3)
    out, st, rc = gpu_run(prob, "fp64", fixed_iters=3)
    assert rc == B.OK and st["iters_min"] == st["iters_max"] == 3
    assert rel(out, ref) < 1e-10


def test_statistics_energy_and_photon_number():
    prob = small("p", 3, 256, 0.18)
    out, st, rc = gpu_run(prob, "fp64")
    assert st["energy_in"] == pytest.approx(prob.dt * np.sum(abs(prob.A0) ** 2), rel=1e-12)
    assert st["energy_out"] == pytest.approx(prob.dt * np.sum(abs(out) ** 2), rel=1e-12)
    fib = O.Fiber.from_problem(prob)
    assert st["photons_in"] == pytest.approx(O.photon_number(fib, O.freq_from_time(prob.A0)), rel=1e-12)
    assert sum(st["iter_hist"]) == st["long_steps"]


@pytest.mark.parametrize("N,fR", [(6, 0.18), (3, 0.0), (4, 0.18)])
def test_long_step_kernel_matches_the_kernel_chain(N, fR, monkeypatch):
    """The opt-in cooperative long-step kernel (GMMNLSE_PERSIST=1) runs the
    same arithmetic as the kernel-per-step chain: equal results and
    iteration counts, and the oracle's within the FP32 bar."""
    prob = I.grin_problem("ls", N=N, Nt=2048, dt=4e-12 / 2048, kind="gaussian", fwhm=150e-15,
                          energy=20e-9, L=2e-3, dz=1e-4, M=5, tol=1e-9, seed=11, fR=fR, s_from="gh")
    chain, st_chain, rc = gpu_run(prob, "fp32")
    assert rc == B.OK
    monkeypatch.setenv("GMMNLSE_PERSIST", "1")
    fused, st_fused, rc = gpu_run(prob, "fp32")
    assert rc == B.OK
    assert st_fused["iters_total"] == st_chain["iters_total"]
    assert rel(fused, chain) < 1e-6
    ref, _ = oracle_run(prob)
    assert rel(fused, ref) < TOL["fp32"]


def test_graph_and_host_loop_agree_bitwise(monkeypatch):
    prob = small("p", 3, 256, 0.18)
    a, sa, _ = gpu_run(prob, "fp64")
    monkeypatch.setenv("GMMNLSE_NO_GRAPH", "1")
    b, sb, _ = gpu_run(prob, "fp64")
    assert np.array_equal(a, b)
    assert sa["iter_hist"] == sb["iter_hist"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_one_context_many_step_sizes(precision):
    """A context (and its cached launch graphs) reused with different dz, M
    and L gives the same result as a fresh context for each call."""
    prob = small("p", 3, 256, 0.18)
    ctx = B.Context.from_problem(prob, precision=precision)
    calls = [(2e-3, 1e-4, 5), (2e-3, 2e-4, 5), (1.2e-3, 1e-4, 7), (2e-3, 1e-4, 5), (8e-4, 4e-5, 5)]
    for L, dz, M in calls:
        a, _, rc = ctx.propagate(prob.A0, L, dz, M, prob.tol, check=False)
        b, _, rcb = gpu_run(prob, precision, L=L, dz=dz, M=M)
        assert rc == rcb == B.OK
        assert np.array_equal(a, b)
    ctx.close()


def test_repeat_is_deterministic():
    prob = small("p", 4, 256, 0.18)
    ctx = B.Context.from_problem(prob, precision="fp64")
    a, _, _ = ctx.propagate(prob.A0, prob.L, prob.dz, prob.M, prob.tol)
    b, _, _ = ctx.propagate(prob.A0, prob.L, prob.dz, prob.M, prob.tol)
    ctx.close()
    assert np.array_equal(a, b)


def test_device_pointers_and_torch_stream():
    import torch
    prob = small("p", 3, 256, 0.18)
    ref, _ = oracle_small(("p", 3, 256, 0.18))
    s = torch.cuda.Stream()
    ctx = B.Context(prob.N, prob.Nt, prob.dt, prob.lam0, prob.n2, prob.beta, prob.SK, None, prob.fR,
                    prob.hR, True, "fp64", stream=s.cuda_stream, io_device=True)
    a0 = torch.from_numpy(prob.A0).cuda()
    out = torch.empty_like(a0)
    torch.cuda.synchronize()
    ctx.propagate(a0, prob.L, prob.dz, prob.M, prob.tol, out=out)
    ctx.close()
    assert rel(out.cpu().numpy(), ref) < 1e-10


# ----------------------------------------------------------------------------
# Mixed precision: contraction on the tensor cores (BF16 hi/lo, FP32 accumulate)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("N,Nt,fR", [(3, 256, 0.18), (6, 512, 0.18), (9, 256, 0.0), (10, 256, 0.18),
                                     (12, 128, 0.18), (15, 1024, 0.18), (16, 256, 0.0), (1, 128, 0.18)])
@pytest.mark.parametrize("mixed", ["bf16", "fp16", "tf32"])
def test_mixed_tensor_core_contraction(N, Nt, fR, mixed):
    """The mixed paths (FFTs in FP32, coupling contraction as a tcgen05 GEMM
    on BF16, scaled FP16 or TF32 hi/lo operands for N >= 9, the FP32
    register contraction below) against the FP64 oracle: <= 1e-3 relative
    L2."""
    key = ("t", N, Nt, fR)
    prob = small(*key)
    ref, sref = oracle_small(key)
    out, st, rc = gpu_run(prob, mixed, tol=1e-9)
    assert rc == B.OK
    err = rel(out, ref)
    assert err < 1e-3
    # the hi/lo split keeps it far below the bar: FP32-like accuracy
    assert err < 1e-5


@functools.lru_cache(maxsize=None)
def wide_grin(N):
    """GRIN fibers of 20, 30 and 64 Hermite-Gauss modes (the last mode group
    partly filled) on a 128-point grid, one long step of M = 4 with three
    fixed updates (the oracle's N^2 x N^2 products stay at seconds)."""
    prob = I.grin_problem("w", N=N, Nt=128, dt=2e-12 / 128, kind="gaussian", fwhm=150e-15,
                          energy=20e-9, L=4e-4, dz=1e-4, M=4, tol=1e-13, seed=13, fR=0.18, s_from="gh")
    ref, _ = oracle_run(prob, fixed_iters=3)
    return prob, ref


@pytest.mark.parametrize("N", [20, 30, 64])
@pytest.mark.parametrize("mixed", ["bf16", "fp16", "tf32"])
def test_mixed_tensor_core_any_mode_count(N, mixed):
    """Every N from 9 to 64 takes the tensor cores: 20 and 30 modes on the
    low-rank coupling (and 64 modes with TF32), 64 modes with 16-bit operands
    on the dense one (2080 x 2080 reduced matrix, nine row blocks of 256),
    against the FP64 oracle at the mixed bar."""
    prob, ref = wide_grin(N)
    out, st, rc = gpu_run(prob, mixed, fixed_iters=3)
    assert rc == B.OK
    assert rel(out, ref) < 1e-3
    assert rel(out, ref) < 1e-5


@pytest.mark.parametrize("mixed", ["bf16", "fp16", "tf32"])
def test_mixed_c2_prefix(mixed):
    prob, ref, sref = c2_prefix()
    out, st, rc = gpu_run(prob, mixed, tol=1e-8)
    assert rc == B.OK
    assert rel(out, ref) < 1e-3


def test_mixed_rejects_what_the_tensor_core_tile_cannot_hold():
    prob = small("p", 10, 64, 0.18)  # Nt not a multiple of the 128-point tile
    with pytest.raises(B.GmmnlseError) as e:
        B.Context.from_problem(prob, precision="bf16")
    assert e.value.status == B.E_UNSUPPORTED
    prob = small("p", 3, 64, 0.18)  # N <= 8: the register contraction, any Nt
    B.Context.from_problem(prob, precision="bf16").close()


@functools.lru_cache(maxsize=None)
def c4_small():
    """The 42-mode step-index fiber of the dense-contraction workload on a
    small grid (Nt = 256): 903 x 903 reduced coupling matrix, four row blocks
    of the tensor-core tile.  One long step of M = 4 with 3 fixed updates
    keeps the oracle's naive N^4 sums to seconds."""
    prob = I.workload("C4", Nt=256, dt=4e-12 / 256, L=4 * 37.5e-6, M=4, npts=160)
    ref, sref = oracle_run(prob, fixed_iters=3)
    return prob, ref


@pytest.mark.parametrize("mixed", ["bf16", "fp16", "tf32"])
def test_mixed_dense_42_mode_contraction(mixed):
    prob, ref = c4_small()
    out, st, rc = gpu_run(prob, mixed, fixed_iters=3)
    assert rc == B.OK
    assert rel(out, ref) < 1e-3


@pytest.mark.parametrize("mixed", ["bf16", "fp16"])
def test_42_mode_low_rank_gemms_match_dense(mixed, monkeypatch):
    """The 42-mode coupling on the low-rank path (GEMM 1 forms U in the
    kernel, K2 writes GEMM 2's operand, GEMM 2 runs four 256-row blocks over
    K = r) against the oracle and the dense tensor-core contraction."""
    prob, ref = c4_small()
    low, st_low, rc = gpu_run(prob, mixed, fixed_iters=3)
    assert rc == B.OK
    assert st_low["coupling_rank"] <= 224
    monkeypatch.setenv("GMMNLSE_DENSE", "1")
    dense, st_dense, rc = gpu_run(prob, mixed, fixed_iters=3)
    assert rc == B.OK
    assert st_dense["coupling_rank"] == 903
    assert rel(low, ref) < 1e-3
    assert rel(dense, ref) < 1e-3
    assert rel(low, dense) < 1e-5


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16", "fp16", "tf32"])
def test_low_rank_coupling_matches_dense(precision, monkeypatch):
    """The 15-mode GRIN fiber: the pair matrix of S is the Gram matrix of the
    products of Hermite-Gauss modes of total order <= 4, which span the 45
    monomials x^i y^j, i + j <= 8, times one Gaussian: rank 45 of K = 120.
    The low-rank path (Z = W U, h_R * Z, R = X V') against the oracle and
    against the dense contraction (GMMNLSE_DENSE=1)."""
    key = ("m", 15, 256, 0.18)
    prob = small(*key)
    ref, _ = oracle_small(key)
    tol = 1e-13 if precision == "fp64" else 1e-9
    low, st_low, rc = gpu_run(prob, precision, tol=tol)
    assert rc == B.OK
    assert st_low["coupling_rank"] == 45
    monkeypatch.setenv("GMMNLSE_DENSE", "1")
    dense, st_dense, rc = gpu_run(prob, precision, tol=tol)
    assert rc == B.OK
    assert st_dense["coupling_rank"] == 120
    bar = TOL.get(precision, 1e-3)
    assert rel(low, ref) < bar
    assert rel(dense, ref) < bar
    assert rel(low, dense) < (1e-11 if precision == "fp64" else 1e-5)


@functools.lru_cache(maxsize=None)
def fifteen_modes_2_14():
    prob = I.grin_problem("m", N=15, Nt=16384, dt=2e-12 / 16384, kind="gaussian", fwhm=150e-15,
                          energy=20e-9, L=5e-4, dz=1e-4, M=5, tol=1e-13, seed=11, fR=0.18, s_from="gh")
    ref, sref = oracle_run(prob)
    return prob, ref, sref


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_15_modes_2_14_low_rank_and_dense(precision, fft_variant, monkeypatch):
    """One long step of the 15-mode fiber at Nt = 2^14: the Raman convolution of
    the low-rank rows (h_R * Z) and of the pair products, each through the
    cluster transforms in FP64 (and in FP32 under the cluster variant)."""
    prob, ref, sref = fifteen_modes_2_14()
    tol = 1e-13 if precision == "fp64" else 1e-9
    low, st_low, rc = gpu_run(prob, precision, tol=tol)
    assert rc == B.OK
    assert st_low["coupling_rank"] == 45
    monkeypatch.setenv("GMMNLSE_DENSE", "1")
    dense, st_dense, rc = gpu_run(prob, precision, tol=tol)
    assert rc == B.OK
    assert st_dense["coupling_rank"] == 120
    assert rel(low, ref) < TOL[precision]
    assert rel(dense, ref) < TOL[precision]
    assert st_low["long_steps"] == st_dense["long_steps"] == len(sref["iters"]) == 1


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_dense_42_mode_contraction_cuda_cores(precision):
    """The FP32 and FP64 paths of the 42-mode workload: the tiled CUDA-core
    contraction over eight 128-row blocks of the 903 x 903 matrix."""
    prob, ref = c4_small()
    out, st, rc = gpu_run(prob, precision, fixed_iters=3)
    assert rc == B.OK
    assert rel(out, ref) < TOL[precision]
