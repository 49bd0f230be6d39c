"""Pins of the oracle's field evaluation (representation formulas, Sec. 2.2):
the region test is Gauss's solid-angle identity; the potentials reproduce an
entire plane wave inside and vanish outside (and the reverse for a field
radiating from a point inside), converging O(h^2) under refinement; the field
of the oracle's solve matches the Mie series of the penetrable sphere."""
import numpy as np
import pytest

import oracle as O
from paper_2104_04609_gb300.inputs import ellipsoid, icosphere
from test_oracle_solve import mie_field


def _pts(rng, n, rmin, rmax):
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    return d * rng.uniform(rmin, rmax, n)[:, None]


def test_region_by_solid_angle():
    rng = np.random.default_rng(0)
    for v, t in (icosphere(2), ellipsoid(400)):
        ax = np.abs(v).max(axis=0)
        inner = _pts(rng, 40, 0.0, 0.8) * ax
        outer = _pts(rng, 40, 1.2, 3.0) * ax
        assert O.inside(v, t, inner).all()
        assert not O.inside(v, t, outer).any()


def _reproduction_errors(lev, k=2.0):
    """SLP(dn v) - DLP(v) for the entire field v = exp(i k d.x): v inside, 0
    outside; and for w = G(x, x0) radiating from x0 inside: DLP(w) - SLP(dn w)
    = w outside, 0 inside."""
    v, t = icosphere(lev)
    n = v / np.linalg.norm(v, axis=1)[:, None]
    rng = np.random.default_rng(1)
    pin, pout = _pts(rng, 30, 0.0, 0.6), _pts(rng, 30, 1.6, 3.0)
    d = np.array([0.0, 0.6, 0.8])
    u = np.exp(1j * k * v @ d)
    du = 1j * k * (n @ d) * u
    S, D = O.potentials(v, t, k, du, u, np.vstack([pin, pout]))
    ein = np.abs((S - D)[:30] - np.exp(1j * k * pin @ d)).max()
    eout = np.abs((S - D)[30:]).max()
    x0 = np.array([0.1, -0.2, 0.15])
    R = v - x0
    r = np.linalg.norm(R, axis=1)
    w = np.exp(1j * k * r) / (4 * np.pi * r)
    dw = w * (1j * k * r - 1.0) / r ** 2 * np.sum(R * n, axis=1)
    S, D = O.potentials(v, t, k, dw, w, np.vstack([pin, pout]))
    ro = np.linalg.norm(pout - x0, axis=1)
    wout = np.exp(1j * k * ro) / (4 * np.pi * ro)
    e2out = np.abs((D - S)[30:] - wout).max() / np.abs(wout).max()
    e2in = np.abs((D - S)[:30]).max() / np.abs(wout).max()
    return ein, eout, e2out, e2in


def test_potentials_reproduce_entire_and_radiating_fields():
    e2 = _reproduction_errors(2)
    e3 = _reproduction_errors(3)
    assert max(e3) < 2e-2, e3
    for a, b in zip(e2, e3):
        assert b < a / 2.5, (e2, e3)  # O(h^2): h halves from level 2 to 3


def test_field_of_solution_matches_mie():
    v, t = icosphere(3)
    k0, k1, rho = 2.0, 3.0, 1.5
    P = O.Problem(v, t, k0, k1, rho, nss=4)
    x = P.solve_direct(P.rhs())
    g = np.linspace(-3.0, 3.0, 25)
    X, Y = np.meshgrid(g, g)
    pts = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    r = np.linalg.norm(pts, axis=1)
    pts = pts[(r < 0.75) | (r > 1.3)]
    u, ins = O.field(v, t, k0, k1, rho, x, pts)
    assert (ins == (np.linalg.norm(pts, axis=1) < 1.0)).all()
    ue = mie_field(k0, k1, rho, 1.0, pts)
    err = np.linalg.norm(u - ue) / np.linalg.norm(ue)
    assert err < 5e-3, err
