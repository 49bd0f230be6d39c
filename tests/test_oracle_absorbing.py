"""Pins of the oracle with an attenuating interior (complex wavenumber
k_int = 2 pi f / c + i alpha, Sec. 3.1): the solution converges O(h^2) to
the Mie series of the absorbing sphere (spherical Bessel functions of
complex argument), OSRC-preconditioned GMRES equals the direct solve, and
the field inside and outside matches the Mie field."""
import numpy as np

import oracle as O
from paper_2104_04609_gb300.inputs import icosphere
from test_oracle_solve import mie_field, mie_traces

K0, K1, RHO = 2.0, 3.0 + 0.4j, 1.5


def _merr(M, a, e):
    d = a - e
    return np.sqrt(abs(np.vdot(d, M @ d)) / abs(np.vdot(e, M @ e)))


def test_absorbing_sphere_converges_to_mie():
    errs = []
    for lev in (2, 3):
        v, t = icosphere(lev)
        nv = len(v)
        P = O.Problem(v, t, K0, K1, RHO, nss=4)
        b = P.rhs()
        x = P.solve_direct(b)
        phi, psi = mie_traces(K0, K1, RHO, 1.0, v[:, 2])
        errs.append(max(_merr(P.M, x[nv:], phi), _merr(P.M, x[:nv], psi)))
        xg, it, hist = P.solve_gmres(b, tol=1e-9, maxit=300)
        assert np.linalg.norm(xg - x) / np.linalg.norm(x) < 1e-7
    assert errs[1] < 0.01 and errs[1] < errs[0] / 3, errs


def test_absorbing_sphere_field():
    v, t = icosphere(3)
    P = O.Problem(v, t, K0, K1, RHO, nss=4)
    x = P.solve_direct(P.rhs())
    g = np.linspace(-2.5, 2.5, 15)
    X, Y = np.meshgrid(g, g)
    pts = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    r = np.linalg.norm(pts, axis=1)
    pts = pts[(r < 0.75) | (r > 1.3)]
    u, _ = O.field(v, t, K0, K1, RHO, x, pts)
    ue = mie_field(K0, K1, RHO, 1.0, pts)
    assert np.linalg.norm(u - ue) / np.linalg.norm(ue) < 5e-3
