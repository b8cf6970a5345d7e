"""The seeded request mix of the serving workload (C5): N in {1, 3, 6, 10,
15}, Nt in 2^10..2^14, Gaussian pulses of 100-500 fs FWHM and 1-200 nJ,
fibers of 1 cm to 1 m, M = 10 and dz the largest whole-long-step division of
L at or below z_NL / 200 (the short-step condition of Sec. III.D, dz well
below the nonlinear length).  Checked on the CPU: the ranges, the step rule,
the units counted per request, the cap on substeps, and the seeding."""
import math

import numpy as np
import pytest

import bench
from paper_1708_05324_b300 import inputs as I

DT = 4.8828125e-15


@pytest.fixture(scope="module")
def mix():
    return bench.serving_requests(512, seed=5, max_substeps=0)


def z_nl(r):
    # the nonlinear length of the request's launched peak power on the GRIN
    # fiber's fundamental mode (gamma = n2 omega0 / (c pi w^2))
    P0 = float(np.max(np.sum(np.abs(r["A0"]) ** 2, axis=0)))
    w = I.grin_mode_width(25e-6, 0.2, 1030e-9)
    gamma = 2.3e-20 * 2 * math.pi / 1030e-9 / (math.pi * w * w)
    return 1.0 / (gamma * P0)


def test_every_shape_of_the_mix_occurs(mix):
    assert len(mix) == 512
    assert {r["N"] for r in mix} == {1, 3, 6, 10, 15}
    assert {r["Nt"] for r in mix} == {1024, 2048, 4096, 8192, 16384}
    for r in mix:
        assert r["A0"].shape == (r["N"], r["Nt"])
        assert r["dt"] == DT and r["M"] == 10


def test_lengths_energies_and_widths_in_range(mix):
    for r in mix:
        assert 0.01 <= r["L"] <= 1.0 * (1 + 1e-12)
        energy = DT * float(np.sum(np.abs(r["A0"]) ** 2))
        assert 1e-9 * (1 - 1e-12) <= energy <= 200e-9 * (1 + 1e-12)
        p = np.sum(np.abs(r["A0"]) ** 2, axis=0)
        above = np.nonzero(p >= p.max() / 2)[0]
        fwhm = (above[-1] - above[0] + 1) * DT
        assert 100e-15 - 2 * DT <= fwhm <= 500e-15 + 2 * DT


def test_whole_long_steps_below_the_nonlinear_length(mix):
    for r in mix:
        nsub = r["units"] // (r["N"] * r["Nt"])
        assert r["units"] == r["N"] * r["Nt"] * nsub
        assert nsub % r["M"] == 0  # whole long steps
        assert r["dz"] * nsub == pytest.approx(r["L"], rel=1e-12)
        # dz <= z_NL / 200, and one long step fewer would break it
        zl = z_nl(r)
        assert r["dz"] <= zl / 200 * (1 + 1e-12)
        assert r["L"] / (nsub - r["M"]) > zl / 200 if nsub > r["M"] else True


def test_cap_keeps_dz_and_cuts_the_length(mix):
    capped = bench.serving_requests(512, seed=5, max_substeps=2000)
    cut = 0
    for a, b in zip(mix, capped):
        assert b["dz"] == a["dz"]
        np.testing.assert_array_equal(a["A0"], b["A0"])
        na = a["units"] // (a["N"] * a["Nt"])
        nb = b["units"] // (b["N"] * b["Nt"])
        assert nb == min(na, 2000)
        assert b["L"] == pytest.approx(nb * b["dz"], rel=1e-12)
        cut += na > 2000
    assert cut > 0  # the cap is exercised by this mix


def test_seeded():
    a = bench.serving_requests(16, seed=5, max_substeps=0)
    b = bench.serving_requests(16, seed=5, max_substeps=0)
    c = bench.serving_requests(16, seed=6, max_substeps=0)
    for x, y in zip(a, b):
        assert (x["N"], x["Nt"], x["L"], x["dz"]) == (y["N"], y["Nt"], y["L"], y["dz"])
        np.testing.assert_array_equal(x["A0"], y["A0"])
    assert [(x["N"], x["Nt"], x["L"]) for x in a] != [(x["N"], x["Nt"], x["L"]) for x in c]
