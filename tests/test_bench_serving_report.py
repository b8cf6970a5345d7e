"""The bench's serving block reports a request that fails instead of
averaging over it: a request whose field holds a NaN ends with
GMMNLSE_E_INVALID (the input check at admission, on the host's side of the
run), and the closed-loop pass then raises with that request's index, shape
and status, which the bench prints in the block's place."""
import numpy as np
import pytest

import bench
from paper_1708_05324_b300 import binding as B

pytestmark = pytest.mark.gpu


def test_a_failed_request_is_reported_with_its_shape(monkeypatch):
    orig = bench.serving_requests

    def poisoned(count, seed=5, max_substeps=2000, M=10):
        reqs = orig(count, seed=seed, max_substeps=max_substeps, M=M)
        reqs[1]["A0"] = reqs[1]["A0"].copy()
        reqs[1]["A0"][0, 0] = np.nan
        return reqs

    monkeypatch.setattr(bench, "serving_requests", poisoned)
    with pytest.raises(RuntimeError) as e:
        bench.run_serving(B, 0, count=6, max_substeps=20, compare=4, sample=2)
    r = orig(6, seed=5, max_substeps=20)[1]
    msg = str(e.value)
    assert "closed loop: 1 of 6 requests failed" in msg
    assert f"request 1 (N {r['N']}, Nt {r['Nt']}, 20 substeps)" in msg
    assert B.load().gmmnlse_strerror(B.E_INVALID).decode() in msg
