"""Benchmark of the MPA hot path: mode * sample * z-steps per second.

Headline workload (the largest single-GPU configuration, the dense-contraction
stress case): step-index fiber (a = 25 um, NA = 0.22, 1030 nm, n2 = 2.3e-20
m^2/W), the first N = 42 LP modes with both orientations solved from the LP
characteristic equation, S_plmn on a 400 x 400 grid (computed on the GPU by
gmmnlse_overlap_tensor), Nt = 2^13 over 10 ps, Kerr + Raman (f_R = 0.18,
tau1 = 12.2 fs, tau2 = 32 fs), self-steepening, 100 fs Gaussian pulse of
100 nJ with seeded random complex mode weights, L = 0.3 m, dz = 37.5 um,
M = 16, tol = 1e-6, MIXED_BF16 (coupling contraction on the tensor cores,
BF16 hi/lo operands, FP32 accumulate).  One bench step = one full
propagation over the 0.3 m fiber (8000 substeps, 500 long steps) through
the C ABI with device buffers.  Synthetic inputs (no dataset).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload C4|C3|C2]
                    [--precision bf16|fp16|tf32|fp32|fp64] [--length L]
    python bench.py --impl reference     # the CPU oracle on a bounded sample
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1708_05324_b300 import inputs as I  # noqa: E402

METRIC = "mode*sample*z-steps/s"
WORKLOADS = {
    "C4": ("step-index a=25um NA=0.22 1030nm, N=42 LP modes (both orientations, S from a 400^2 grid), "
           "Nt=2^13 over 10 ps, Kerr+Raman fR=0.18, self-steepening, 100 fs Gaussian 100 nJ seeded weights, "
           "L=0.3 m, dz=37.5 um, M=16, tol=1e-6"),
    "C3": ("GRIN a=25um NA=0.2 1030nm, N=15 HG modes (groups 0-4), Nt=2^14 over 20 ps, Kerr+Raman fR=0.18, "
           "self-steepening, 500 fs Gaussian 200 nJ seeded weights, L=1 m, dz=12.5 um, M=20, tol=1e-6"),
    "C2": ("GRIN a=25um NA=0.2 1030nm, N=6 HG modes, Nt=2^13 over 10 ps, Kerr+Raman fR=0.18, "
           "self-steepening, 200 fs Gaussian 50 nJ seeded weights, L=0.5 m, dz=25 um, M=10, tol=1e-8"),
}
FULL_LENGTH = {"C4": 0.3, "C3": 1.0, "C2": 0.5}
SEED = {"C4": 4, "C3": 3, "C2": 2}
# the precision's error against the FP64 GPU path is measured on this prefix
ERR_PREFIX = {"C4": (16 * 37.5e-6, "one long step (0.6 mm)"), "C3": (2e-3, "2 mm (8 long steps)"),
              "C2": (5e-3, "5 mm (20 long steps)")}
# DRAM bytes of the dominant kernel slot per iteration from one ncu capture
# (the kernels unchanged since), keyed (workload, precision, kernel slot):
# the 42-mode MIXED_BF16 contraction is its two GEMM launches, 302.7 MB for
# 17 live substeps, scaled to the profile's 16
TRAFFIC = {("C4", "bf16", "contract"): 284.9e6}
FP32_ALU_TFLOPS = 148 * 128 * 2 * 2.032 / 1e3  # SMs x FP32 lanes x 2 (FMA) x max SM clock [GHz]
# nominal dense TF32 : BF16 tensor rate (1.1 : 2.25 PFLOP/s)
TF32_OVER_BF16 = 1.1 / 2.25

_PROBLEMS = {}


def problem(name="C4", L=None, seed=None, dev=0, gpu_overlap=True):
    """The named workload with fiber length L (default: its full length).
    The 42-mode fiber's overlap tensor comes from the 400^2 grid, on the GPU
    through gmmnlse_overlap_tensor (gpu_overlap) or by the numpy sums (for
    the oracle's inputs, which never come from the CUDA path)."""
    L = FULL_LENGTH[name] if L is None else L
    seed = SEED[name] if seed is None else seed
    key = (name, seed, gpu_overlap and name == "C4")
    if key not in _PROBLEMS:
        if name == "C4":
            over = None
            if gpu_overlap:
                from paper_1708_05324_b300 import binding as B
                over = lambda F, dA: B.overlap_tensor(F, dA, dev)  # noqa: E731
            _PROBLEMS[key] = I.workload("C4", seed=seed, npts=400, overlap=over)
        elif name == "C3":
            _PROBLEMS[key] = I.workload("C3", seed=seed, s_from="gh")
        else:
            _PROBLEMS[key] = I.workload(name, seed=seed)
    return dataclasses.replace(_PROBLEMS[key], L=L)


def units(prob, L=None):
    return prob.N * prob.Nt * int(round((L or prob.L) / prob.dz))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows)}


def max_over_ranks(seconds, dist=None, device="cpu"):
    """The largest of a per-rank time over the ranks of the job (the rank's
    own without a process group): the job's time is that of its slowest
    replica."""
    if dist is None:
        return float(seconds)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank_step, steps, world, seconds):
    """Whole-job throughput: the units every rank processed over the job's
    (slowest rank's) time; each rank runs its own replica (weak scaling)."""
    return units_per_rank_step * steps * world / seconds


def launches_per_step(st, raman, mixed=False, fp64=False, graph=True, N=1, Nt=8192, tf32=False):
    """Kernel launches of one propagate call, from its statistics."""
    per_iter = 5 if raman else 4   # K1 [K2] K3 K4 K5 (decision in K5's last block)
    tc = mixed and N > 8           # the tensor cores run the contraction from 9 modes
    lowrank = st.get("coupling_rank", 0) < N * (N + 1) // 2
    if lowrank:
        per_iter += 1              # two GEMMs (Z = W U, then X V')
    if tc and not lowrank:
        per_iter += 1              # the operand pack of V
    elif tc:
        # 16-bit operands: GEMM 1 forms U itself and, with Raman, K2 writes
        # GEMM 2's operand V'; TF32 packs both operands
        per_iter += (1 if tf32 else 0) + (1 if tf32 or not raman else 0)
    fft = 1 if Nt <= 8192 else 2  # FP64 input/output transforms (halves + combine above 8192)
    n = 1 + fft + 1          # non-finite check, forward transform, input sums
    if not fp64:
        n += 1               # psi0 rounded to the working precision
    n += 1 + fft             # output sums, inverse transform
    # per long step: the advance (bookkeeping in its last block)
    n += st["iters_total"] * per_iter + st["long_steps"]
    return n


def contraction_flops_per_point(prob, coupling_rank, mixed):
    """Algorithmic flops of the coupling contraction per point (substep x
    sample) and MPA iteration, unpadded: with the low-rank coupling (rank r)
    the two GEMMs 2 r (K + P), else the dense reduced GEMM 2 P KK; x3 for the
    hi/lo products on the tensor cores."""
    P = prob.N * (prob.N + 1) // 2
    KK = P if prob.fR == 0 or prob.SR is None or prob.SR is prob.SK else 2 * P
    per = 2.0 * coupling_rank * (P + P) if coupling_rank < P else 2.0 * P * KK
    return per * (3 if mixed else 1)


# ----------------------------------------------------------------------------
# Error along the fiber and the M sweep (separate modes of bench.py)
# ----------------------------------------------------------------------------
def run_error_curve(args, dev):
    """Relative L2 difference between this precision and the FP64 GPU path
    along the fiber.  Both propagate the same input in SEGMENTS pieces of
    whole long steps, each piece continuing from its own previous output
    (the field between long steps is kept in FP64 on both paths, so the
    pieces add only FP64 transforms); the difference is printed at the end
    of each piece.  Over long, strongly nonlinear fibers rounding differences
    grow, so this is the curve that says how far a prefix parity carries."""
    from paper_1708_05324_b300 import binding as B
    prob = problem(args.workload, L=args.length, dev=dev)
    lstep = prob.M * prob.dz
    nlong = int(round(prob.L / lstep))
    nseg = max(1, min(args.error_curve, nlong))
    per = nlong // nseg
    c64 = B.Context.from_problem(prob, precision="fp64", device=dev)
    cx = B.Context.from_problem(prob, precision=args.precision, device=dev)
    a64, ax = np.ascontiguousarray(prob.A0), np.ascontiguousarray(prob.A0)
    curve, done = [], 0
    t0 = time.perf_counter()
    for sgm in range(nseg):
        nl = per if sgm < nseg - 1 else nlong - done
        a64, _, _ = c64.propagate(a64, nl * lstep, prob.dz, prob.M, prob.tol)
        ax, _, _ = cx.propagate(ax, nl * lstep, prob.dz, prob.M, prob.tol)
        done += nl
        curve.append([round(done * lstep, 9), float(np.linalg.norm(ax - a64) / np.linalg.norm(a64))])
    c64.close()
    cx.close()
    print(json.dumps({"error_curve": curve, "vs": "fp64 gpu", "precision": args.precision,
                      "workload": args.workload, "length_m": prob.L, "long_steps": nlong,
                      "wall_s": time.perf_counter() - t0}))


def run_m_sweep(args, dev):
    """Speed-up of the MPA over a solver that takes one substep at a time, on
    the same kernels (Sec. III.D, Fig. 3).  At convergence the M coupled
    equations of a long step are the implicit trapezoid rule applied substep
    after substep in the interaction picture, whatever the long step's origin,
    so every M reaches the same field up to the iteration tolerance; M = 1 is
    that sequential integrator, one dz per fixed-point solve.  Each M
    propagates the same fiber prefix with the same dz; the line reports the
    rate, the iterations per long step, the speed-up over M = 1 and the
    relative L2 difference from the M = 1 field."""
    import torch
    from paper_1708_05324_b300 import binding as B
    prob = problem(args.workload, L=args.length, dev=dev)
    Ms = sorted({int(x) for x in args.m_sweep.split(",")} | {1})
    stream = torch.cuda.Stream(device=dev)
    ctx = B.Context.from_problem(prob, precision=args.precision, device=dev, stream=stream.cuda_stream,
                                 io_device=True)
    a0 = torch.from_numpy(prob.A0).to(f"cuda:{dev}")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
    u = units(prob)
    rows, ref = [], None
    for M in Ms:
        out = torch.empty_like(a0)

        def once():
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st, rc = ctx.propagate(a0, prob.L, prob.dz, M, prob.tol, out=out, check=False)
            e1.record(stream)
            e1.synchronize()
            if rc != B.OK:
                raise B.GmmnlseError(rc, f"propagate (M={M})")
            return e0.elapsed_time(e1), st
        for _ in range(max(args.warmup, 1)):
            once()
        ms = []
        for _ in range(max(args.steps, 1)):
            t, st = once()
            ms.append(t)
        torch.cuda.synchronize()
        field = out.cpu().numpy()
        if ref is None:
            ref = field
        t = float(np.median(ms))
        rows.append({"M": M, "ms": round(t, 4), "units_per_s": u / (t / 1e3),
                     "iters_per_long_step": st["iters_total"] / max(st["long_steps"], 1),
                     "long_steps": st["long_steps"],
                     "rel_l2_vs_M1": float(np.linalg.norm(field - ref) / np.linalg.norm(ref))})
    # the split-step comparator (RK4IP, four evaluations of N per step of dz)
    # on the same kernels, timed the same way
    rk_out = torch.empty_like(a0)
    rk_ms = []
    for it in range(max(args.warmup, 1) + max(args.steps, 1)):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, rk_st, rc = ctx.propagate_rk4ip(a0, prob.L, prob.dz, out=rk_out, check=False)
        e1.record(stream)
        e1.synchronize()
        if rc != B.OK:
            raise B.GmmnlseError(rc, "propagate_rk4ip")
        if it >= max(args.warmup, 1):
            rk_ms.append(e0.elapsed_time(e1))
    rk_t = float(np.median(rk_ms))
    rk_field = rk_out.cpu().numpy()
    rk4ip = {"h": prob.dz, "ms": round(rk_t, 4), "units_per_s": u / (rk_t / 1e3),
             "evaluations_of_N": rk_st["iters_total"],
             "rel_l2_vs_mpa_M1": float(np.linalg.norm(rk_field - ref) / np.linalg.norm(ref))}
    auto_M, auto_sec = ctx.choose_m(a0, prob.dz, prob.tol, Ms, trial_substeps=2 * max(Ms),
                                    scratch=torch.empty_like(a0))
    ctx.close()
    base = rows[0]["ms"]
    for r in rows:
        r["speedup_vs_M1"] = round(base / r["ms"], 3)
        r["speedup_vs_rk4ip"] = round(rk_t / r["ms"], 3)
    print(json.dumps({"m_sweep": rows, "rk4ip": rk4ip, "workload": args.workload, "precision": args.precision,
                      "length_m": prob.L, "dz": prob.dz, "tol": prob.tol, "unit": METRIC,
                      "choose_m": {"M": auto_M, "trial_substeps": 2 * max(Ms),
                                   "us_per_substep": {m: round(1e6 * t, 3) for m, t in auto_sec.items()}},
                      "timing": "CUDA events per propagation, median of --steps, L2 flushed before each"}))


# ----------------------------------------------------------------------------
# The CPU oracle: reference arm and cpu_baseline
# ----------------------------------------------------------------------------
# MPA iterations per long step of the 42-mode workload at tol = 1e-6 over the
# whole 0.3 m fiber (3.334, measured on the GPU; 5.0 on the first
# centimetre, 3 to 4 later), used to turn the oracle's time per integrand
# into a rate when no GPU run of the same workload gives the count
C4_ITERS_PER_LONG_STEP = 3.334


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        return max([d.get("num_threads", 1) for d in info] or [1])
    except Exception:
        return os.cpu_count() or 1


def _oracle_integrand_seconds(fib, psi, count, budget_s):
    """Seconds per integrand evaluation (Eq. MPA_eq at one substep: the
    oracle's unit of work) over up to `count` evaluations within budget_s."""
    import oracle as O
    times = []
    t_all = time.perf_counter()
    for k in range(count):
        t0 = time.perf_counter()
        O.integrand(fib, psi, (k % 16) * 37.5e-6)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_all > budget_s:
            break
    return float(np.median(times)), len(times)


def _oracle_rate(prob, sec_per_integrand, iters_per_long_step):
    """Units per second of the oracle's MPA: a long step of M substeps takes
    iters x M integrand evaluations (plus I_0 once), all in the oracle's
    plain sums; everything else of the step is negligible beside them."""
    per_long_step = prob.N * prob.Nt * prob.M
    evals = iters_per_long_step * prob.M + 1
    return per_long_step / (sec_per_integrand * evals)


_ONE_THREAD_CHILD = """
import sys, time
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle as O
z = np.load(sys.argv[2])
fR, dt, lam0, n2, ss = z["scal"]
fib = O.Fiber(z["beta"], z["SK"], z["SK"], fR, z["hR"], dt, lam0, n2, bool(ss))
psi = O.freq_from_time(z["A0"])
O.integrand(fib, psi, 0.0)
t0 = time.perf_counter()
O.integrand(fib, psi, 37.5e-6)
print(time.perf_counter() - t0)
"""


def _one_thread_integrand_seconds(prob):
    """Seconds per integrand evaluation on one host thread: timed in a child
    process whose BLAS thread counts are set to 1 before numpy loads (the
    inputs handed over in a temporary file)."""
    import subprocess
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        f = os.path.join(d, "fiber.npz")
        np.savez(f, beta=prob.beta, SK=prob.SK, hR=prob.hR, A0=prob.A0,
                 scal=np.array([prob.fR, prob.dt, prob.lam0, prob.n2, float(prob.self_steepening)]))
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
                   CUDA_VISIBLE_DEVICES="")
        out = subprocess.run([sys.executable, "-c", _ONE_THREAD_CHILD, ROOT, f], env=env, capture_output=True,
                             text=True, timeout=600, check=True)
        return float(out.stdout.strip().splitlines()[-1])


def cpu_baseline(seconds=15.0, iters_per_long_step=C4_ITERS_PER_LONG_STEP):
    """Oracle rate on the host cores on a bounded sample of the 42-mode
    workload: integrand evaluations at full size (N = 42, Nt = 2^13) with
    every BLAS thread, then one with a single thread; iters_per_long_step
    (the GPU run's count on the same fiber) turns them into a rate."""
    import oracle as O
    prob = problem("C4", gpu_overlap=False)
    fib = O.Fiber.from_problem(prob)
    psi = O.freq_from_time(prob.A0)
    O.integrand(fib, psi, 0.0)  # warm-up
    sec, count = _oracle_integrand_seconds(fib, psi, 64, seconds)
    rate = _oracle_rate(prob, sec, iters_per_long_step)
    try:
        sec1 = _one_thread_integrand_seconds(prob)
        one = {"value": _oracle_rate(prob, sec1, iters_per_long_step), "unit": METRIC, "cores": 1,
               "sec_per_integrand": sec1}
    except Exception as e:  # the figure is then missing, and says why
        one = {"value": None, "error": f"{type(e).__name__}: {e}"}
    return {"value": rate, "unit": METRIC, "cores": _blas_threads(), "kind": "oracle",
            "sample": (f"{count} integrand evaluations of the 42-mode field at full size (median {sec:.2f} s each), "
                       f"scaled to the rate by {iters_per_long_step:.3f} iterations x 16 substeps + 1 per long "
                       f"step (the GPU run's iteration count on the same fiber)"),
            "one_core": one}


def run_reference(args):
    """The CPU oracle as it stands, on a bounded sample of the workload: each
    step is one integrand evaluation of the 42-mode field at full size, the
    rate scaled as in cpu_baseline."""
    import oracle as O
    prob = problem("C4", gpu_overlap=False)
    fib = O.Fiber.from_problem(prob)
    psi = O.freq_from_time(prob.A0)
    for _ in range(max(args.warmup, 0)):
        O.integrand(fib, psi, 0.0)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        O.integrand(fib, psi, (k % 16) * prob.dz)
        times.append(time.perf_counter() - t0)
    sec = sum(times) / len(times)
    value = _oracle_rate(prob, sec, C4_ITERS_PER_LONG_STEP)
    cores = _blas_threads()
    sample = (f"one integrand evaluation of the 42-mode field at full size per step ({sec:.2f} s), scaled to "
              f"the rate by {C4_ITERS_PER_LONG_STEP} iterations x 16 substeps + 1 per long step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS["C4"], "precision": "fp64-cpu-oracle"},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------------------------
# Serving (continuous batching through gmmnlse_submit / gmmnlse_poll)
# ----------------------------------------------------------------------------
SERVE_NS = (1, 3, 6, 10, 15)
SERVE_NTS = (1024, 2048, 4096, 8192, 16384)


def serving_requests(count, seed=5, max_substeps=2000, M=10):
    """Seeded requests with the C5 mix: N in {1,3,6,10,15} and Nt in 2^10..2^14
    (uniform), dt = 4.8828125 fs, Gaussian FWHM log-uniform 100-500 fs, energy
    log-uniform 1-200 nJ, L log-uniform 1 cm - 1 m, M = 10,
    dz = L / (M ceil(L / (M z_NL / 200))).  A request longer than max_substeps
    substeps is cut to that many (same dz); max_substeps = 0 keeps every
    request whole."""
    g = I.SplitMix64(seed)
    dt = 4.8828125e-15
    reqs = []
    for i in range(count):
        N = SERVE_NS[min(int(g.uniform() * 5), 4)]
        Nt = SERVE_NTS[min(int(g.uniform() * 5), 4)]
        fwhm = 100e-15 * 5.0 ** g.uniform()
        energy = 1e-9 * 200.0 ** g.uniform()
        L = 0.01 * 100.0 ** g.uniform()
        A0 = I.launch_field(N, Nt, dt, "gaussian", fwhm, energy, seed * 1000 + i)
        P0 = float(np.max(np.sum(np.abs(A0) ** 2, axis=0)))
        w = I.grin_mode_width(25e-6, 0.2, 1030e-9)
        gamma = 2.3e-20 * 2 * math.pi / 1030e-9 / (math.pi * w * w)
        znl = 1.0 / (gamma * P0)
        nsub = M * math.ceil(L / (M * znl / 200))
        dz = L / nsub
        if max_substeps and nsub > max_substeps:
            nsub = max_substeps
            L = nsub * dz
        reqs.append(dict(N=N, Nt=Nt, dt=dt, A0=A0, L=L, dz=dz, M=M, units=N * Nt * nsub))
    return reqs


def _serve_pass(B, srv, ctxs, reqs, gaps=None):
    """Submit the requests (all at once, or each after its gap in seconds
    from the previous one) and poll, while submitting, until every one has
    ended: (seconds, {index: (latency s from submission to the poll that saw
    it end, status, field)})."""
    done, pending = {}, {}
    t0 = time.perf_counter()
    due = t0 + (np.cumsum(gaps) if gaps is not None else np.zeros(len(reqs)))
    nxt = 0
    while nxt < len(reqs) or pending:
        now = time.perf_counter()
        while nxt < len(reqs) and due[nxt] <= now:
            r = reqs[nxt]
            t = srv.submit(ctxs[(r["N"], r["Nt"])], r["A0"], r["L"], r["dz"], r["M"], 1e-6)
            pending[t] = (nxt, time.perf_counter())
            nxt += 1
        for t in list(pending):
            i, ts = pending[t]
            r = reqs[i]
            rc, out, st = srv.poll(t, r["N"], r["Nt"])
            if rc != B.PENDING:
                done[i] = (time.perf_counter() - ts, rc, out)
                del pending[t]
        time.sleep(0.0002)
    return time.perf_counter() - t0, done


def run_serving(B, dev, count=512, max_substeps=0, inflight=32, load=0.9, seed=5, compare=64, sample=8):
    """The C5 request mix through gmmnlse_submit / gmmnlse_poll in MIXED_BF16:
    a closed-loop pass (every request submitted at once: capacity), an
    open-loop pass with Poisson arrivals at `load` x that capacity (p50 / p99
    latency from submission to completion), the first `compare` requests
    served with and without same-shape packing, and the first `sample`
    requests served against the plain FP64 MPA run serially (its rate, and
    the served results' relative L2 error against it)."""
    reqs = serving_requests(count, seed=seed, max_substeps=max_substeps)
    ctxs = {}
    for r in reqs:
        key = (r["N"], r["Nt"])
        if key not in ctxs:
            prob = I.grin_problem("serve", N=r["N"], Nt=r["Nt"], dt=r["dt"], kind="gaussian", fwhm=200e-15,
                                  energy=1e-9, L=0.01, dz=1e-3, M=10, tol=1e-6, seed=1, fR=0.18, s_from="gh")
            ctxs[key] = (prob, B.Context.from_problem(prob, precision="bf16", device=dev))
    cx = {k: v[1] for k, v in ctxs.items()}
    budget = 32 << 30
    srv = B.Server(hbm_budget=budget, max_inflight=inflight)
    _serve_pass(B, srv, cx, reqs[:4])  # warm-up (workspaces, graphs)
    cap_s, done = _serve_pass(B, srv, cx, reqs)
    total_units = sum(r["units"] for r in reqs)
    capacity = len(reqs) / cap_s
    status = {}
    for _, rc, _ in done.values():
        status[rc] = status.get(rc, 0) + 1
    bad = sorted((done[i][0], i) for i in done if done[i][1] != B.OK)
    if bad:  # every request was submitted at once: the first to fail ended first
        srv.close()
        for _, c in ctxs.values():
            c.close()
        i = bad[0][1]
        r = reqs[i]
        raise RuntimeError(f"closed loop: {len(bad)} of {len(reqs)} requests failed; the first: request {i} "
                           f"(N {r['N']}, Nt {r['Nt']}, {r['units'] // (r['N'] * r['Nt'])} substeps) ended "
                           f"after {1e3 * bad[0][0]:.0f} ms with "
                           f"{B.load().gmmnlse_strerror(done[i][1]).decode()}")
    closed_lat = np.array([done[i][0] for i in range(len(reqs))]) * 1e3
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / (load * capacity), size=len(reqs))
    open_s, done_open = _serve_pass(B, srv, cx, reqs, gaps)
    lat = np.array([done_open[i][0] for i in range(len(reqs))]) * 1e3
    served = {i: done_open[i][2] for i in range(min(sample, len(reqs)))}
    _, peak = srv.resident_bytes()
    srv.close()
    # the same first requests with and without packing
    sub = reqs[:compare]
    cmp_units = sum(r["units"] for r in sub)
    os.environ["GMMNLSE_PACK_SLOTS"] = "1"
    try:
        srv1 = B.Server(hbm_budget=budget, max_inflight=inflight)
        _serve_pass(B, srv1, cx, sub[:4])
        unpacked_s, _ = _serve_pass(B, srv1, cx, sub)
        srv1.close()
    finally:
        del os.environ["GMMNLSE_PACK_SLOTS"]
    srvp = B.Server(hbm_budget=budget, max_inflight=inflight)
    _serve_pass(B, srvp, cx, sub[:4])
    packed_s, _ = _serve_pass(B, srvp, cx, sub)
    srvp.close()
    # serial plain FP64 MPA on the first requests: its rate, and the served
    # (BF16, packed) results against it
    t64, errs = 0.0, []
    for i, r in enumerate(reqs[:sample]):
        prob = ctxs[(r["N"], r["Nt"])][0]
        c = B.Context.from_problem(prob, precision="fp64", device=dev)
        c.propagate(r["A0"], min(r["L"], 10 * r["M"] * r["dz"]), r["dz"], r["M"], 1e-6, check=False)  # warm-up
        t1 = time.perf_counter()
        ref, _, rc = c.propagate(r["A0"], r["L"], r["dz"], r["M"], 1e-6, check=False)
        t64 += time.perf_counter() - t1
        c.close()
        if rc != B.OK:
            for _, cc in ctxs.values():
                cc.close()
            raise RuntimeError(f"FP64 serial run of request {i} (N {r['N']}, Nt {r['Nt']}): "
                               f"{B.load().gmmnlse_strerror(rc).decode()}")
        errs.append(float(np.linalg.norm(served[i] - ref) / np.linalg.norm(ref)))
    for _, c in ctxs.values():
        c.close()
    fp64_serial = sum(r["units"] for r in reqs[:sample]) / t64
    return {"requests": len(reqs), "precision": "bf16", "max_inflight": inflight,
            "max_substeps_per_request": max_substeps or None,
            "total_units": total_units,
            "closed_loop_units_per_s": total_units / cap_s, "closed_loop_s": cap_s,
            "closed_loop_p50_ms": float(np.percentile(closed_lat, 50)),
            "closed_loop_p99_ms": float(np.percentile(closed_lat, 99)),
            "offered_load": load, "open_loop_units_per_s": total_units / open_s, "open_loop_s": open_s,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "status_counts": {B.load().gmmnlse_strerror(k).decode(): v for k, v in status.items()},
            "packing": {"requests": len(sub), "packed_units_per_s": cmp_units / packed_s,
                        "unpacked_units_per_s": cmp_units / unpacked_s, "speedup": unpacked_s / packed_s},
            "served_rel_l2_vs_fp64": {"requests": len(errs), "max": max(errs), "median": float(np.median(errs))},
            "fp64_serial_units_per_s": fp64_serial, "fp64_serial_requests": sample,
            "served_vs_fp64_serial": (total_units / cap_s) / fp64_serial,
            "resident_peak_bytes": peak, "hbm_budget_bytes": budget,
            "mix": "C5: N in {1,3,6,10,15}, Nt 2^10..2^14, FWHM 100-500 fs, 1-200 nJ, L 1 cm-1 m, dz = z_NL/200"}


# ----------------------------------------------------------------------------
# Timed propagations
# ----------------------------------------------------------------------------
def propagation_runner(B, prob, precision, dev, stream, flush):
    """A context of the problem and one event-timed whole propagation through
    the C ABI with device buffers (the inputs resident in HBM before the
    timed region), L2 flushed before it: (context, step() -> (ms, stats))."""
    import torch
    ctx = B.Context.from_problem(prob, precision=precision, device=dev, stream=stream.cuda_stream, io_device=True)
    a0 = torch.from_numpy(prob.A0).to(f"cuda:{dev}")
    out = torch.empty_like(a0)

    def one_step():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)  # L2 flush (256 MiB write), outside the timed events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st, rc = ctx.propagate(a0, prob.L, prob.dz, prob.M, prob.tol, out=out, check=False)
        e1.record(stream)
        e1.synchronize()
        if rc != B.OK:
            raise B.GmmnlseError(rc, "propagate")
        return e0.elapsed_time(e1), st

    return ctx, one_step


def workload_text(name, L):
    text = WORKLOADS[name]
    return text if L == FULL_LENGTH[name] else text + f" (a {L} m prefix of the fiber per step)"


def prefix_error(B, name, precision, dev):
    """Relative L2 of this precision against the FP64 GPU path on the
    workload's prefix, and the FP64 path's rate there."""
    L, what = ERR_PREFIX[name]
    pre = problem(name, L=L, dev=dev)
    c64 = B.Context.from_problem(pre, precision="fp64", device=dev)
    ref64, st64, _ = c64.propagate(pre.A0, pre.L, pre.dz, pre.M, pre.tol)
    c64.close()
    cx = B.Context.from_problem(pre, precision=precision, device=dev)
    mine, _, _ = cx.propagate(pre.A0, pre.L, pre.dz, pre.M, pre.tol)
    cx.close()
    return float(np.linalg.norm(mine - ref64) / np.linalg.norm(ref64)), units(pre) / (st64["ms"] / 1e3), what


def roofline(prob, prof, coupling_rank, precision, peaks, src, workload):
    """Roofline of the dominant kernel slot of one MPA iteration, from the
    event-timed per-kernel durations of gmmnlse_profile (launches of
    substeps 1..M).  The contraction of N > 8 modes is bound by the tensor
    cores (mixed precisions; the sustained BF16 peak, since it runs inside a
    seconds-long step; TF32 at the nominal TF32 : BF16 ratio) or the FP32
    ALUs; the rest by HBM."""
    dom = max(prof, key=lambda k: prof[k][0])
    ms_dom, bytes_dom = prof[dom]
    mixed = precision in ("bf16", "fp16", "tf32")
    if dom == "contract" and prob.N > 8:
        flops = contraction_flops_per_point(prob, coupling_rank, mixed) * prob.M * prob.Nt
        achieved = flops / (ms_dom * 1e-3) / 1e12
        if mixed:
            scale = TF32_OVER_BF16 if precision == "tf32" else 1.0
            peak = peaks["bf16_tflops_sustained"] * scale
            roof = {"kernel": "contract (GEMM 1 Z = W U and GEMM 2 R = X V' with the l-sum)"
                    if coupling_rank < prob.N * (prob.N + 1) // 2 else "contract (dense GEMM with the l-sum)",
                    "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "frac_of_burst": achieved / (peaks["bf16_tflops"] * scale),
                    "peak_source": f"{src} bf16_tflops_sustained" + (" x 1.1/2.25 (nominal TF32 : BF16)"
                                                                    if precision == "tf32" else ""),
                    "algorithmic_flops": flops}
        else:
            roof = {"kernel": "contract", "bound": "alu", "achieved": achieved, "peak": FP32_ALU_TFLOPS,
                    "unit": "TFLOP/s", "frac": achieved / FP32_ALU_TFLOPS,
                    "peak_source": "148 SMs x 128 FP32 FMA/clk x 2 x 2.032 GHz", "algorithmic_flops": flops}
    else:
        achieved = bytes_dom / (ms_dom * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_source": f"{src} hbm_gbs", "algorithmic_bytes": bytes_dom}
    roof["traffic"] = TRAFFIC.get((workload, precision, dom))
    roof["kernel_ms"] = ms_dom
    roof["all_kernels_ms"] = {k: v[0] for k, v in prof.items()}
    # every kernel slot against its bound (HBM for all but the contraction);
    # each slot is timed over back-to-back launches on the same buffers, so
    # operands that fit the 126 MB L2 are partly served from it (K5 reads
    # the integrand K4 writes: its fraction can exceed 1)
    roof["hbm_frac_by_kernel"] = {k: (v[1] / (v[0] * 1e-3) / 1e9) / peaks["hbm_gbs"] for k, v in prof.items()
                                  if v[0] > 0 and k != "contract"}
    roof["hbm_frac_note"] = ("algorithmic bytes / event time of back-to-back launches on the same buffers "
                             "(warm L2: operands below 126 MB partly hit it)")
    return roof


def extra_line(B, name, precision, length, dev, stream, flush, steps=2, warmup=1):
    """A further workload and precision, event-timed like the headline on a
    prefix of its fiber."""
    prob = problem(name, L=length, dev=dev)
    ctx, one_step = propagation_runner(B, prob, precision, dev, stream, flush)
    for _ in range(warmup):
        one_step()
    runs = [one_step() for _ in range(steps)]
    ctx.close()
    t = sum(r[0] for r in runs) / steps
    st = runs[-1][1]
    return {"workload": workload_text(name, length), "precision": precision, "length_m": length,
            "value": units(prob) / (t / 1e3), "unit": METRIC, "ms_per_step": t, "steps": steps, "warmup": warmup,
            "iters_per_long_step": st["iters_total"] / max(st["long_steps"], 1),
            "coupling_rank": st.get("coupling_rank")}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="C4", choices=["C4", "C3", "C2"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp16", "tf32", "fp32", "fp64"])
    ap.add_argument("--length", type=float, default=None, help="fiber length per step [m] (default: the full fiber)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the further workloads")
    ap.add_argument("--serve-requests", type=int, default=512, help="requests in the serving pass (0: skip)")
    ap.add_argument("--serve-max-substeps", type=int, default=2000,
                    help="serving pass: cut longer requests to this many substeps (0: every request whole, "
                         "lengths up to 1 m; several minutes)")
    ap.add_argument("--serve-only", action="store_true", help="only the serving pass (one JSON line)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--profile-run", action="store_true",
                    help="only the timed propagations (for ncu captures)")
    ap.add_argument("--kernel-profile", action="store_true",
                    help="with --profile-run: also time each kernel of one iteration")
    ap.add_argument("--error-curve", type=int, default=0, metavar="SEGMENTS",
                    help="print the error against the FP64 GPU path at SEGMENTS points along the fiber")
    ap.add_argument("--m-sweep", default="", metavar="M1,M2,...",
                    help="time the workload at each M (and M=1) over --length: MPA speed-up over one substep at a time")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    if args.error_curve:
        if rank == 0:
            run_error_curve(args, local)
        return

    if args.m_sweep:
        if rank == 0:
            run_m_sweep(args, local)
        return

    import torch
    from paper_1708_05324_b300 import binding as B

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = local
    torch.cuda.set_device(dev)
    if args.serve_only:
        if rank == 0:
            print(json.dumps({"serving": run_serving(B, dev, count=args.serve_requests,
                                                     max_substeps=args.serve_max_substeps)}))
        return

    # each rank draws its own replica of the workload (seed + rank)
    prob = problem(args.workload, L=args.length, seed=SEED[args.workload] + rank, dev=dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
    u = units(prob)

    ctx, one_step = propagation_runner(B, prob, args.precision, dev, stream, flush)
    for _ in range(args.warmup):
        one_step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, stats = [], []
    with ClockSampler(dev) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ms, st = one_step()
            step_ms.append(ms)
            stats.append(st)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        wall = time.perf_counter() - t0
    dev_s = max_over_ranks(sum(step_ms) / 1e3, dist, f"cuda:{dev}")
    value = job_rate(u, args.steps, world, dev_s)
    coupling_rank = stats[-1].get("coupling_rank")

    if args.profile_run:
        line = {"profile_run": True, "workload": args.workload, "precision": args.precision, "length_m": prob.L,
                "ms_per_step": 1e3 * dev_s / args.steps, "value": value,
                "iters_total": stats[-1]["iters_total"], "long_steps": stats[-1]["long_steps"],
                "coupling_rank": coupling_rank}
        if args.kernel_profile:
            prof = ctx.profile(prob.M, reps=20)
            line["kernels_ms"] = {k: v[0] for k, v in prof.items()}
            line["kernels_bytes"] = {k: v[1] for k, v in prof.items()}
        if rank == 0:
            print(json.dumps(line))
        ctx.close()
        if dist:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel (CUDA events on the context's stream)
    prof = ctx.profile(prob.M, reps=20)
    ctx.close()

    # end to end through the C ABI with host buffers (copies inside the timed region)
    ctx_h = B.Context.from_problem(prob, precision=args.precision, device=dev, stream=stream.cuda_stream)
    h_in = np.ascontiguousarray(prob.A0)
    h_out = np.empty_like(h_in)
    ctx_h.propagate(h_in, prob.L, prob.dz, prob.M, prob.tol, out=h_out)
    torch.cuda.synchronize()
    e2e_t = []
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    for _ in range(e2e_steps):
        t1 = time.perf_counter()
        ctx_h.propagate(h_in, prob.L, prob.dz, prob.M, prob.tol, out=h_out)
        e2e_t.append(time.perf_counter() - t1)
    ctx_h.close()
    e2e_s = max_over_ranks(sum(e2e_t), dist, f"cuda:{dev}")
    e2e = {"value": job_rate(u, e2e_steps, world, e2e_s), "unit": METRIC, "steps": e2e_steps,
           "h2d_bytes_per_step": int(h_in.nbytes), "d2h_bytes_per_step": int(h_out.nbytes)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    err, fp64_rate, err_prefix = prefix_error(B, args.workload, args.precision, dev)
    peaks, src = measured_peaks()
    roof = roofline(prob, prof, coupling_rank, args.precision, peaks, src, args.workload)
    mixed = args.precision in ("bf16", "fp16", "tf32")
    launches = sum(launches_per_step(st, prob.fR != 0, mixed, args.precision == "fp64", N=prob.N, Nt=prob.Nt,
                                     tf32=args.precision == "tf32") for st in stats)
    workload = workload_text(args.workload, prob.L)
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "bf16": "f32+bf16x3", "fp16": "f32+f16x3",
                  "tf32": "f32+tf32x3"}[args.precision],
        "data": "synthetic",
        "config": {"workload": workload, "name": args.workload,
                   "length_m": prob.L, "precision": args.precision,
                   "l2": "flushed between steps (256 MiB write); working set above L2",
                   "units_per_step": u, "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "long_steps_per_step": stats[-1]["long_steps"],
                   "iters_per_long_step": stats[-1]["iters_total"] / max(stats[-1]["long_steps"], 1),
                   "coupling_rank": coupling_rank,
                   "rel_l2_err_vs_fp64_gpu": err, "err_prefix": err_prefix, "fp64_gpu_value": fp64_rate,
                   "wall_s": wall},
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": roof,
        "clocks": clk.summary(),
    }
    if not args.no_extra:
        extra = {}
        for key, (name, prec, length) in {"C4_fp32": ("C4", "fp32", 0.012), "C3_bf16": ("C3", "bf16", 0.05),
                                          "C2_fp32": ("C2", "fp32", 0.5)}.items():
            if (name, prec) != (args.workload, args.precision):
                extra[key] = extra_line(B, name, prec, length, dev, stream, flush)
        line["extra"] = extra
    if args.serve_requests > 0:
        # the headline above is complete: a failure in the serving block is
        # reported in its place rather than losing the line
        try:
            line["serving"] = run_serving(B, dev, count=args.serve_requests, max_substeps=args.serve_max_substeps)
        except Exception as e:
            line["serving"] = {"error": f"{type(e).__name__}: {e}"}
    if not args.no_cpu_baseline:
        its = line["config"]["iters_per_long_step"] if args.workload == "C4" else C4_ITERS_PER_LONG_STEP
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, its)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
