"""Serving: continuous batching of propagation requests (gmmnlse_submit/poll).

Requests of different mode counts, grids and lengths run concurrently on
their own streams; each result must equal the same request run alone."""
import time

import numpy as np
import pytest

from paper_1708_05324_b300 import binding as B
from paper_1708_05324_b300 import inputs as I

pytestmark = pytest.mark.gpu


def _ctx(N, Nt, precision, seed):
    prob = I.grin_problem(f"s{N}", N=N, Nt=Nt, dt=4e-12 / Nt, kind="gaussian", fwhm=150e-15,
                          energy=15e-9, L=1.5e-3, dz=1e-4, M=5, tol=1e-11, seed=seed, fR=0.18, s_from="gh")
    return prob, B.Context.from_problem(prob, precision=precision)


def _wait(srv, tickets, shapes, timeout=120):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t, (N, Nt) in zip(tickets, shapes):
            if t in out:
                continue
            rc, a, st = srv.poll(t, N, Nt)
            if rc != B.PENDING:
                out[t] = (rc, a, st)
        assert time.time() - t0 < timeout, "requests did not finish"
        time.sleep(0.002)
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16", "fp16", "tf32"])
def test_results_are_the_same_alone_and_in_the_mix(precision):
    """Alone vs in the mix: FP64 to 1e-12, FP32 to 1e-6, the mixed served
    path (tensor-core contraction for the 10-, 12- and 15-mode requests) to
    its stated 1e-3."""
    mixed = precision in ("bf16", "fp16", "tf32")
    specs = ([(10, 256, 1), (15, 512, 2), (3, 256, 3), (12, 128, 4)] if mixed
             else [(1, 256, 1), (3, 1024, 2), (6, 512, 3), (3, 256, 4)])
    ctxs = [_ctx(*s[:2], precision, s[2]) for s in specs]
    alone = []
    for prob, ctx in ctxs:
        lengths = (prob.L, 2 * prob.L)
        alone.append({L: ctx.propagate(prob.A0, L, prob.dz, prob.M, prob.tol)[0] for L in lengths})
    srv = B.Server(hbm_budget=1 << 30, max_inflight=4)
    tickets, shapes, expect = [], [], []
    for rep in range(3):
        for (prob, ctx), ref in zip(ctxs, alone):
            L = prob.L * (1 + (rep % 2))
            tickets.append(srv.submit(ctx, prob.A0, L, prob.dz, prob.M, prob.tol))
            shapes.append((prob.N, prob.Nt))
            expect.append(ref[L])
    res = _wait(srv, tickets, shapes)
    bar = {"fp64": 1e-12, "fp32": 1e-6}.get(precision, 1e-3)
    for t, ref in zip(tickets, expect):
        rc, a, st = res[t]
        assert rc == B.OK
        assert np.linalg.norm(a - ref) / np.linalg.norm(ref) < bar
        assert st["long_steps"] in (3, 6)
    srv.close()
    for _, ctx in ctxs:
        ctx.close()


def test_admission_by_memory_budget_and_ticket_errors():
    prob, ctx = _ctx(3, 1024, "fp64", 5)
    one = ctx.request_bytes(prob.M)
    # room for one request at a time: every request still completes, in order
    srv = B.Server(hbm_budget=int(one * 1.5), max_inflight=4)
    with pytest.raises(B.GmmnlseError) as e:
        srv.submit(ctx, prob.A0, prob.L, prob.dz, 64, prob.tol)  # bigger workspace than the budget
    assert e.value.status == B.E_NOMEM
    tickets = [srv.submit(ctx, prob.A0, prob.L, prob.dz, prob.M, prob.tol) for _ in range(4)]
    res = _wait(srv, tickets, [(3, 1024)] * 4)
    ref = res[tickets[0]][1]
    for t in tickets:
        assert res[t][0] == B.OK
        assert np.array_equal(res[t][1], ref)
    rc, _, _ = srv.poll(tickets[0], 3, 1024)  # already released
    assert rc == B.E_INVALID
    rc, _, _ = srv.poll(987654321, 3, 1024)
    assert rc == B.E_INVALID
    srv.close()
    ctx.close()


def test_shutdown_with_queued_requests_does_not_hang():
    prob, ctx = _ctx(6, 512, "fp32", 6)
    srv = B.Server(hbm_budget=1 << 30, max_inflight=1)
    for _ in range(6):
        srv.submit(ctx, prob.A0, 10 * prob.L, prob.dz, prob.M, prob.tol)
    t0 = time.time()
    srv.close()  # waits for the running one, cancels the queued ones
    assert time.time() - t0 < 60
    ctx.close()


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-12), ("fp32", 1e-6), ("bf16", 1e-3)])
def test_packed_requests_equal_single_propagations(precision, bar):
    """Requests on one context with the same M share a packed workspace (one
    launch advances every slot by a long step); each has its own dz, length,
    tolerance and field, joins and leaves at long-step boundaries, and must
    give what gmmnlse_propagate gives alone.  A request whose length is not a
    whole number of long steps runs unpacked beside them."""
    N, Nt = (10, 256) if precision == "bf16" else (3, 512)
    prob, ctx = _ctx(N, Nt, precision, 7)
    rng = np.random.default_rng(3)
    reqs = []
    for k in range(7):
        dz = prob.dz * (1.0 + 0.5 * k / 7)
        nlong = 2 + (k % 4)
        L = nlong * prob.M * dz if k != 5 else (nlong * prob.M + 2) * dz  # k = 5: a remainder long step
        A0 = prob.A0 * (1.0 + 0.1 * rng.standard_normal())
        tol = prob.tol if precision == "fp64" else 1e-9 * (1 + k)
        reqs.append((A0, L, dz, tol))
    alone = [ctx.propagate(A0, L, dz, prob.M, tol)[0] for (A0, L, dz, tol) in reqs]
    srv = B.Server(hbm_budget=4 << 30, max_inflight=4)
    tickets = [srv.submit(ctx, A0, L, dz, prob.M, tol) for (A0, L, dz, tol) in reqs]
    res = _wait(srv, tickets, [(N, Nt)] * len(reqs))
    for t, ref, (A0, L, dz, tol) in zip(tickets, alone, reqs):
        rc, a, st = res[t]
        assert rc == B.OK
        assert np.linalg.norm(a - ref) / np.linalg.norm(ref) < bar
        assert st["z"] == pytest.approx(L, rel=1e-9)
    srv.close()
    ctx.close()


def test_resident_bytes_never_exceed_the_budget():
    """Four shapes whose packed workspaces do not all fit: the server frees
    idle ones to admit the next shape, every request completes, and the bytes
    its workspaces hold never exceed the budget."""
    specs = [(3, 256, 11), (6, 512, 12), (3, 1024, 13), (1, 512, 14)]
    ctxs = [_ctx(s[0], s[1], "fp32", s[2]) for s in specs]
    packed = max(c.request_bytes(p.M) for p, c in ctxs) * 4
    budget = int(packed * 2.5)  # about two packed workspaces at a time
    srv = B.Server(hbm_budget=budget, max_inflight=4)
    tickets, shapes = [], []
    for rep in range(3):
        for prob, ctx in ctxs:
            tickets.append(srv.submit(ctx, prob.A0, prob.L * (1 + rep), prob.dz, prob.M, 1e-8))
            shapes.append((prob.N, prob.Nt))
    res = _wait(srv, tickets, shapes, timeout=300)
    assert all(r[0] == B.OK for r in res.values())
    now, peak = srv.resident_bytes()
    assert 0 < peak <= budget
    srv.close()
    for _, ctx in ctxs:
        ctx.close()


def test_cancel_a_queued_request():
    prob, ctx = _ctx(6, 512, "fp32", 15)
    srv = B.Server(hbm_budget=1 << 30, max_inflight=1)
    tickets = [srv.submit(ctx, prob.A0, 20 * prob.L, prob.dz, prob.M, prob.tol) for _ in range(3)]
    assert srv.cancel(tickets[2]) == B.OK
    res = _wait(srv, tickets[:1], [(6, 512)], timeout=300)
    assert res[tickets[0]][0] == B.OK
    rc, _, _ = srv.poll(tickets[2], 6, 512)
    assert rc == B.E_CANCELLED
    srv.close()
    ctx.close()


@pytest.mark.parametrize("slots", ["16", "1"])
def test_many_tensor_core_requests_in_flight(slots, monkeypatch):
    """Forty requests, 32 in flight, on two contexts whose contraction runs on
    the tensor cores (10 and 15 modes, MIXED_BF16) and two that run it on the
    CUDA cores (3 and 6 modes), packed and unpacked: every request ends
    within the deadline (tensor-core work never shares the device with other
    work of the library) and a sample equals the same request run alone."""
    monkeypatch.setenv("GMMNLSE_PACK_SLOTS", slots)
    specs = [(10, 1024, 21), (15, 1024, 22), (3, 2048, 23), (6, 1024, 24)]
    ctxs = [_ctx(N, Nt, "bf16", seed) for N, Nt, seed in specs]
    rng = np.random.default_rng(9)
    reqs = []
    for k in range(40):
        prob, ctx = ctxs[k % 4]
        dz = prob.dz * (1.0 + 0.3 * rng.uniform())
        steps = prob.M * int(rng.integers(2, 9)) + (3 if k % 7 == 0 else 0)  # a few with a remainder
        reqs.append((prob, ctx, prob.A0 * (1.0 + 0.2 * rng.standard_normal()), steps * dz, dz))
    srv = B.Server(hbm_budget=8 << 30, max_inflight=32)
    tickets = [srv.submit(ctx, A0, L, dz, prob.M, 1e-9) for prob, ctx, A0, L, dz in reqs]
    res = _wait(srv, tickets, [(p.N, p.Nt) for p, *_ in reqs], timeout=240)
    srv.close()
    assert all(res[t][0] == B.OK for t in tickets)
    for t, (prob, ctx, A0, L, dz) in list(zip(tickets, reqs))[::5]:
        ref = ctx.propagate(A0, L, dz, prob.M, 1e-9)[0]
        a = res[t][1]
        assert np.linalg.norm(a - ref) / np.linalg.norm(ref) < 1e-3
    for _, ctx in ctxs:
        ctx.close()
