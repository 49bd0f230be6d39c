"""The accuracy figures of the bench line come from bench.py's own helpers
(Mie traces and field of the penetrable sphere, the P1 mass norm): checked
here against the Mie series the oracle's solve tests use and against exact
cases.  No GPU."""
import numpy as np
import pytest

import bench
from paper_2104_04609_gb300.inputs import icosphere
from test_oracle_solve import mie_field, mie_traces


@pytest.mark.parametrize("k0,k1,rho", [(20.0, 26.0, 1.5), (2.0, 3.0, 1.5), (15.0, 36.0, 1.9)])
def test_bench_mie_traces_match_the_tests_series(k0, k1, rho):
    cth = np.linspace(-1.0, 1.0, 41)
    phi_b, psi_b = bench.mie_traces(k0, k1, rho, 1.0, cth)
    phi_t, psi_t = mie_traces(k0, k1, rho, 1.0, cth)
    assert np.abs(phi_b - phi_t).max() <= 1e-12 * np.abs(phi_t).max()
    assert np.abs(psi_b - psi_t).max() <= 1e-12 * np.abs(psi_t).max()


def test_bench_mie_field_matches_the_tests_series():
    g = np.random.default_rng(5)
    pts = g.uniform(-3.0, 3.0, size=(60, 3))
    pts[:5] *= 0.2  # a few points inside the sphere
    ub = bench.mie_total_field(2.0, 3.0, 1.5, 1.0, pts)
    ut = mie_field(2.0, 3.0, 1.5, 1.0, pts)
    assert np.abs(ub - ut).max() <= 1e-10 * np.abs(ut).max()


def test_bench_p1_mass_and_solution_error():
    v, t = icosphere(2)
    M = bench.p1_mass(v, t)
    p0, p1, p2 = (v[t[:, i]] for i in range(3))
    area = 0.5 * np.linalg.norm(np.cross(p1 - p0, p2 - p0), axis=1).sum()
    assert abs(M.sum() - area) < 1e-12 * area              # sum of the P1 mass matrix = area
    assert np.abs((M - M.T).toarray()).max() == 0.0
    W = {"verts": v, "tris": t, "k_ext": 2.0, "k_int": 3.0, "rho_ratio": 1.5}
    d = np.array([0.0, 0.0, 1.0])
    phi, psi = mie_traces(2.0, 3.0, 1.5, 1.0, v[:, 2] / np.linalg.norm(v, axis=1))
    x = np.concatenate([psi, phi])
    e = bench.solution_error_vs_mie(W, x, d)
    assert e["psi"] < 1e-12 and e["phi"] < 1e-12 and e["both"] < 1e-12
    e = bench.solution_error_vs_mie(W, 1.01 * x, d)       # a 1 % scaling is a 1 % error
    assert abs(e["psi"] - 0.01) < 1e-12 and abs(e["phi"] - 0.01) < 1e-12 and abs(e["both"] - 0.01) < 1e-12
    # the direction enters through cos(angle to d): rotating both leaves the error unchanged
    R = np.array([[0.0, 0.0, 1.0], [0.0, 1.0, 0.0], [-1.0, 0.0, 0.0]])
    W2 = dict(W, verts=v @ R.T)
    e2 = bench.solution_error_vs_mie(W2, 1.01 * x, R @ d)
    assert abs(e2["both"] - 0.01) < 1e-12


def test_clock_record_parsing():
    """The clocks object of the bench line: median / max SM clock of the
    sampled GPU and the throttle reasons seen while the timed region ran."""
    lines = [
        "0, 2070, 2070, 1100.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "0, 2055, 2070, 1380.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
        "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
        "1, 900, 2070, 300.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active\n",  # other GPU
        "0, [N/A], 2070, 1000, 0x0, Not Active, Not Active, Not Active, Not Active\n",            # no clock
        "garbage line\n",
    ]
    r = bench.ClockSampler.parse(lines, [0])
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]
    r = bench.ClockSampler.parse(lines, [0, 1])
    assert r["reasons"] == ["hw_slowdown", "sw_power_cap"] and r["samples"] == 4
    r = bench.ClockSampler.parse([], [0])
    assert r["sm_mhz"] is None and r["reasons"] == [] and r["samples"] == 0
