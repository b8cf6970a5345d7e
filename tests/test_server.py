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
