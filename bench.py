"""Benchmark of the MPA hot path: mode * sample * z-steps per second.

Workload (the GMMNLSE Kerr + Raman propagation the metric is quoted on):
parabolic GRIN fiber (a = 25 um, NA = 0.2, 1030 nm, n2 = 2.3e-20 m^2/W),
N = 6 Hermite-Gauss modes, Nt = 2^13 over 10 ps, f_R = 0.18 (tau1 = 12.2 fs,
tau2 = 32 fs), self-steepening on, 200 fs Gaussian pulse of 50 nJ with seeded
random complex mode weights, L = 0.5 m, dz = 25 um, M = 10, tol = 1e-8.
One bench step = one full propagation over the 0.5 m fiber (20000 substeps,
2000 long steps) through the C ABI.  Synthetic inputs (no dataset).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64]
    python bench.py --impl reference     # the CPU oracle on a bounded sample
"""
from __future__ import annotations

import argparse
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
WORKLOAD = ("GRIN a=25um NA=0.2 1030nm, N=6 HG modes, Nt=2^13 over 10 ps, Kerr+Raman fR=0.18, "
            "self-steepening, 200 fs Gaussian 50 nJ seeded weights, L=0.5 m, dz=25 um, M=10, tol=1e-8")
WORKLOADS = {
    "C2": WORKLOAD,
    "C3": ("GRIN a=25um NA=0.2 1030nm, N=15 HG modes (groups 0-4), Nt=2^14 over 20 ps, Kerr+Raman fR=0.18, "
           "self-steepening, 500 fs Gaussian 200 nJ seeded weights, dz=12.5 um, M=20, tol=1e-6"),
    "C4": ("step-index a=25um NA=0.22 1030nm, N=42 LP modes (both orientations, S from a 200^2 grid), "
           "Nt=2^13 over 10 ps, Kerr+Raman fR=0.18, self-steepening, 100 fs Gaussian 100 nJ seeded weights, "
           "dz=37.5 um, M=16, tol=1e-6"),
}
# DRAM bytes per launch of the dominant kernel from one ncu capture (the
# kernel unchanged since): k_pairs_raman<float, 16, 0> on the 6-mode
# workload, warm L2, profiles/pairs_raman_c2_fp32.md.
TRAFFIC = {("C2", "fp32", "pairs_raman"): 1024 + 256}
FP32_ALU_TFLOPS = 148 * 128 * 2 * 2.032 / 1e3  # SMs x FP32 lanes x 2 (FMA) x max SM clock [GHz]


def problem(seed=2, L=0.5, name="C2"):
    if name == "C2":
        return I.workload("C2", L=L, seed=seed)
    if name == "C3":
        return I.workload(name, L=L, seed=seed + 1, s_from="gh")
    return I.workload(name, L=L, npts=200)  # C4: S on a 200^2 grid for the profile runs


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


def run_error_curve(args, dev):
    """Relative L2 difference between this precision and the FP64 GPU path
    along the fiber.  Both propagate the same input in SEGMENTS pieces of
    whole long steps, each piece continuing from its own previous output
    (the field between long steps is kept in FP64 on both paths, so the
    pieces add only FP64 transforms); the difference is printed at the end
    of each piece.  Over long, strongly nonlinear fibers rounding differences
    grow, so this is the curve that says how far a prefix parity carries."""
    from paper_1708_05324_b300 import binding as B
    prob = problem(L=args.length, name=args.workload)
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
                      "workload": args.workload, "length_m": args.length, "long_steps": nlong,
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
    prob = problem(L=args.length, name=args.workload)
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
                      "length_m": args.length, "dz": prob.dz, "tol": prob.tol, "unit": METRIC,
                      "choose_m": {"M": auto_M, "trial_substeps": 2 * max(Ms),
                                   "us_per_substep": {m: round(1e6 * t, 3) for m, t in auto_sec.items()}},
                      "timing": "CUDA events per propagation, median of --steps, L2 flushed before each"}))


def run_reference(args):
    """The CPU oracle as it stands, on a bounded sample of the workload."""
    import oracle as O
    prob = problem()
    fib = O.Fiber.from_problem(prob)
    sample_L = 2 * prob.M * prob.dz  # two long steps per bench step
    for _ in range(max(args.warmup, 0)):
        O.mpa_propagate(fib, prob.A0, sample_L, prob.dz, prob.M, prob.tol)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.mpa_propagate(fib, prob.A0, sample_L, prob.dz, prob.M, prob.tol)
        times.append(time.perf_counter() - t0)
    u = units(prob, sample_L)
    value = u * len(times) / sum(times)
    cores = _blas_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "fp64-cpu-oracle"},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
                             "sample": "first 2 long steps (20 substeps, 0.5 mm) of the 0.5 m run per step"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        return max([d.get("num_threads", 1) for d in info] or [1])
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(seconds=15.0):
    """Oracle rate on the host cores for as many long steps as fit in ~seconds."""
    import oracle as O
    prob = problem()
    fib = O.Fiber.from_problem(prob)
    psi = O.freq_from_time(prob.A0)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds:
        psi, n, trace, status = O.mpa_long_step(fib, psi, prob.dz, prob.M, prob.tol)
        steps += 1
    dt = time.perf_counter() - t0
    rate = prob.N * prob.Nt * prob.M * steps / dt
    return {"value": rate, "unit": METRIC, "cores": _blas_threads(), "kind": "oracle",
            "sample": f"first {steps} long steps ({steps * prob.M} substeps) of the 0.5 m run, {dt:.1f} s"}


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
    substeps is cut to that many (same dz), so the pass fits in minutes."""
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
        if nsub > max_substeps:
            nsub = max_substeps
            L = nsub * dz
        reqs.append(dict(N=N, Nt=Nt, dt=dt, A0=A0, L=L, dz=dz, M=M, units=N * Nt * nsub))
    return reqs


def run_serving(B, dev, count=32, max_substeps=2000, inflight=8, load=0.9, seed=5):
    reqs = serving_requests(count, seed=seed, max_substeps=max_substeps)
    ctxs = {}
    for r in reqs:
        key = (r["N"], r["Nt"])
        if key not in ctxs:
            prob = I.grin_problem("serve", N=r["N"], Nt=r["Nt"], dt=r["dt"], kind="gaussian", fwhm=200e-15,
                                  energy=1e-9, L=0.01, dz=1e-3, M=10, tol=1e-6, seed=1, fR=0.18, s_from="gh")
            ctxs[key] = B.Context.from_problem(prob, precision="bf16", device=dev)
    srv = B.Server(hbm_budget=32 << 30, max_inflight=inflight)

    def submit(r):
        return srv.submit(ctxs[(r["N"], r["Nt"])], r["A0"], r["L"], r["dz"], r["M"], 1e-6)

    def drain(tickets, t_submit):
        done = {}
        while len(done) < len(tickets):
            for t in tickets:
                if t in done:
                    continue
                rc, out, st = srv.poll(t, *shapes[t])
                if rc != B.PENDING:
                    done[t] = (time.perf_counter() - t_submit[t], rc)
            time.sleep(0.0005)
        return done

    # warm-up (graphs, workspaces)
    shapes = {}
    warm = []
    for r in reqs[:4]:
        t = submit(r)
        shapes[t] = (r["N"], r["Nt"])
        warm.append(t)
    drain(warm, {t: time.perf_counter() for t in warm})
    # capacity: all requests at once
    t0 = time.perf_counter()
    tickets, t_submit = [], {}
    for r in reqs:
        t = submit(r)
        shapes[t] = (r["N"], r["Nt"])
        t_submit[t] = time.perf_counter()
        tickets.append(t)
    done = drain(tickets, t_submit)
    cap_s = time.perf_counter() - t0
    units = sum(r["units"] for r in reqs)
    status = {}
    for _, rc in done.values():
        status[rc] = status.get(rc, 0) + 1
    capacity = len(reqs) / cap_s
    # open loop: Poisson arrivals at load x capacity
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / (load * capacity), size=len(reqs))
    tickets, t_submit = [], {}
    t0 = time.perf_counter()
    next_t = t0
    for r, gap in zip(reqs, gaps):
        next_t += gap
        while time.perf_counter() < next_t:
            time.sleep(0.0002)
        t = submit(r)
        shapes[t] = (r["N"], r["Nt"])
        t_submit[t] = time.perf_counter()
        tickets.append(t)
    done = drain(tickets, t_submit)
    open_s = time.perf_counter() - t0
    lat = np.array([done[t][0] for t in tickets]) * 1e3
    srv.close()
    for c in ctxs.values():
        c.close()
    # serial plain FP64 MPA on the first 8 of the same requests
    sub = reqs[:8]
    t64 = 0.0
    for r in sub:
        prob = I.grin_problem("serve", N=r["N"], Nt=r["Nt"], dt=r["dt"], kind="gaussian", fwhm=200e-15,
                              energy=1e-9, L=0.01, dz=1e-3, M=10, tol=1e-6, seed=1, fR=0.18, s_from="gh")
        c = B.Context.from_problem(prob, precision="fp64", device=dev)
        c.propagate(r["A0"], r["L"], r["dz"], r["M"], 1e-6, check=False)  # warm-up
        t1 = time.perf_counter()
        c.propagate(r["A0"], r["L"], r["dz"], r["M"], 1e-6, check=False)
        t64 += time.perf_counter() - t1
        c.close()
    fp64_serial = sum(r["units"] for r in sub) / t64
    return {"requests": len(reqs), "precision": "bf16", "max_inflight": inflight,
            "max_substeps_per_request": max_substeps,
            "closed_loop_units_per_s": units / cap_s, "closed_loop_s": cap_s,
            "offered_load": load, "open_loop_units_per_s": units / open_s,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "status_counts": {B.load().gmmnlse_strerror(k).decode(): v for k, v in status.items()},
            "fp64_serial_units_per_s": fp64_serial, "fp64_serial_requests": len(sub),
            "mix": "C5: N in {1,3,6,10,15}, Nt 2^10..2^14, FWHM 100-500 fs, 1-200 nJ, L 1 cm-1 m, dz = z_NL/200"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "bf16", "fp16", "tf32"])
    ap.add_argument("--length", type=float, default=0.5, help="fiber length per step [m]")
    ap.add_argument("--workload", default="C2", choices=["C2", "C3", "C4"],
                    help="C3 (N=15, Nt=2^14, M=20) and C4 (N=42, Nt=2^13, M=16) are for --profile-run; the metric is quoted on C2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=32, help="requests in the serving pass (0: skip)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
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

    prob = problem(seed=2 + rank, L=args.length, name=args.workload)
    stream = torch.cuda.Stream(device=dev)
    ctx = B.Context.from_problem(prob, precision=args.precision, device=dev, stream=stream.cuda_stream,
                                 io_device=True)
    a0 = torch.from_numpy(prob.A0).to(f"cuda:{dev}")
    out = torch.empty_like(a0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
    u = units(prob)

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

    for _ in range(args.warmup):
        one_step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = []
    stats = []
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

    if args.profile_run:
        line = {"profile_run": True, "precision": args.precision, "length_m": args.length,
                "ms_per_step": 1e3 * dev_s / args.steps, "value": value,
                "iters_total": stats[-1]["iters_total"], "long_steps": stats[-1]["long_steps"]}
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

    # end to end through the C ABI with host buffers (copies inside the timed region)
    ctx_h = B.Context.from_problem(prob, precision=args.precision, device=dev, stream=stream.cuda_stream)
    h_in = np.ascontiguousarray(prob.A0)
    h_out = np.empty_like(h_in)
    ctx_h.propagate(h_in, prob.L, prob.dz, prob.M, prob.tol, out=h_out)
    torch.cuda.synchronize()
    e2e_t = []
    for _ in range(args.steps):
        t1 = time.perf_counter()
        ctx_h.propagate(h_in, prob.L, prob.dz, prob.M, prob.tol, out=h_out)
        e2e_t.append(time.perf_counter() - t1)
    ctx_h.close()
    e2e_s = max_over_ranks(sum(e2e_t), dist, f"cuda:{dev}")
    e2e = {"value": job_rate(u, args.steps, world, e2e_s), "unit": METRIC,
           "h2d_bytes_per_step": int(h_in.nbytes), "d2h_bytes_per_step": int(h_out.nbytes)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # error of this path against the FP64 GPU path on a prefix: 5 mm (200 long
    # steps) of the 6-mode run, 2 mm (8 long steps) of the 15-mode run, one
    # long step of the 42-mode run
    err, fp64_rate, err_prefix = None, None, None
    if args.workload in ("C2", "C3", "C4"):
        pre = {"C2": lambda: I.workload("C2", L=5e-3),
               "C3": lambda: problem(L=2e-3, name="C3"),
               "C4": lambda: problem(L=16 * 37.5e-6, name="C4")}[args.workload]()
        err_prefix = {"C2": "5 mm", "C3": "2 mm (8 long steps)", "C4": "one long step (0.6 mm)"}[args.workload]
        c64 = B.Context.from_problem(pre, precision="fp64", device=dev)
        ref64, st64, _ = c64.propagate(pre.A0, pre.L, pre.dz, pre.M, pre.tol)
        c64.close()
        cx = B.Context.from_problem(pre, precision=args.precision, device=dev)
        mine, _, _ = cx.propagate(pre.A0, pre.L, pre.dz, pre.M, pre.tol)
        cx.close()
        err = float(np.linalg.norm(mine - ref64) / np.linalg.norm(ref64))
        fp64_rate = units(pre) / (st64["ms"] / 1e3)

    # roofline of the dominant kernel (CUDA events on the context's stream)
    prof = ctx.profile(prob.M, reps=20)
    dom = max(prof, key=lambda k: prof[k][0])
    ms_dom, bytes_dom = prof[dom]
    peaks, src = measured_peaks()
    mixed = args.precision in ("bf16", "fp16", "tf32")
    if dom == "contract" and prob.N > 8:
        # a dense GEMM: 2 P KK flops per point and iteration, or with the
        # low-rank coupling (rank r) the two GEMMs 2 r (K + P); x3 for the
        # hi/lo products on the tensor cores; points = M substeps x Nt
        P = prob.N * (prob.N + 1) // 2
        KK = P if prob.fR == 0 or prob.SR is None or prob.SR is prob.SK else 2 * P
        r = stats[-1].get("coupling_rank", P)
        per_point = 2.0 * r * (P + P) if r < P else 2.0 * P * KK
        flops = per_point * prob.M * prob.Nt * (3 if mixed else 1)
        achieved = flops / (ms_dom * 1e-3) / 1e12
        roof = {"kernel": dom, "bound": "tensor" if mixed else "alu", "achieved": achieved,
                "peak": (peaks["bf16_tflops"] * (1.1 / 2.25 if args.precision == "tf32" else 1.0)) if mixed
                else FP32_ALU_TFLOPS, "unit": "TFLOP/s",
                "algorithmic_flops": flops}
        roof["frac"] = achieved / roof["peak"]
        roof["peak_source"] = ((src + (", x 1.1/2.25 (nominal TF32 : BF16 dense)" if args.precision == "tf32" else ""))
                               if mixed else "148 SMs x 128 FP32 FMA/clk x 2 x 2.032 GHz")
    else:
        achieved = bytes_dom / (ms_dom * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_source": src, "algorithmic_bytes": bytes_dom}
    roof["traffic"] = TRAFFIC.get((args.workload, args.precision, dom))
    roof["kernel_ms"] = ms_dom
    roof["all_kernels_ms"] = {k: v[0] for k, v in prof.items()}
    raman = prob.fR != 0
    launches = sum(launches_per_step(st, raman, mixed, args.precision == "fp64", N=prob.N, Nt=prob.Nt,
                                     tf32=args.precision == "tf32") for st in stats)
    ctx.close()
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "bf16": "f32+bf16x3", "fp16": "f32+f16x3", "tf32": "f32+tf32x3"}[args.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload] if args.length == 0.5 or args.workload != "C2"
                   else WORKLOAD.replace("L=0.5 m", f"L={args.length} m"),
                   "length_m": args.length, "precision": args.precision,
                   "l2": "flushed between steps (256 MiB write)",
                   "units_per_step": u, "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "long_steps_per_step": stats[-1]["long_steps"],
                   "iters_per_long_step": stats[-1]["iters_total"] / max(stats[-1]["long_steps"], 1),
                   "coupling_rank": stats[-1].get("coupling_rank"),
                   "rel_l2_err_vs_fp64_gpu": err, "err_prefix": err_prefix, "fp64_gpu_value": fp64_rate,
                   "wall_s": wall},
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": roof,
        "clocks": clk.summary(),
    }
    if args.serve_requests > 0:
        line["serving"] = run_serving(B, dev, count=args.serve_requests)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
