"""Pins of the oracle for disjoint objects with their own materials (Sec.
2.2, multiple scattering): one object reduces to the single-object system
exactly; the objects decouple as they move apart, the coupling falling off
like the scattered field (1/d); a mirror-symmetric pair has a mirror-
symmetric solution; the block-diagonal OSRC solve equals the direct solve;
the field of one object equals the single-object field."""
import numpy as np
import pytest

import oracle as O
from paper_2104_04609_gb300.inputs import icosphere

K0 = 2.0
MATS = ([3.0, 1.5], [1.5, 0.8])  # (k_int, rho_ratio) of the two objects


def _pair(d, lev=2):
    v, t = icosphere(lev)
    return (np.vstack([v + [-d / 2, 0, 0], v + [d / 2, 0, 0]]),
            np.vstack([t, t + len(v)]), v, t)


def test_components_numbered_by_first_triangle():
    v, t = icosphere(1)
    n = len(v)
    T = np.vstack([t + n, t, t + 2 * n])
    tc, vc = O.components(T)
    assert (tc[:len(t)] == 0).all() and (tc[len(t):2 * len(t)] == 1).all()
    assert (tc[2 * len(t):] == 2).all()
    assert (vc[:n] == 1).all() and (vc[n:2 * n] == 0).all() and (vc[2 * n:] == 2).all()


def test_single_object_equals_single_system():
    v, t = icosphere(2)
    a = O.pmchwt_matrix(v, t, K0, 3.0, 1.5, nss=4)
    b = O.pmchwt_matrix_objects(v, t, K0, [3.0], [1.5], nss=4)
    assert np.array_equal(a, b)


def test_objects_decouple_like_one_over_distance():
    errs = []
    for d in (6.0, 12.0, 24.0):
        V, T, v, t = _pair(d)
        nv = len(v)
        P = O.Problem(V, T, K0, None, None, nss=4, objects=MATS)
        x = P.solve_direct(P.rhs())
        xs = []
        for m, sh in enumerate((-d / 2, d / 2)):
            Pm = O.Problem(v + [sh, 0, 0], t, K0, MATS[0][m], MATS[1][m], nss=4)
            xs.append(Pm.solve_direct(Pm.rhs()))
        xu = np.concatenate([xs[0][:nv], xs[1][:nv], xs[0][nv:], xs[1][nv:]])
        errs.append(np.linalg.norm(x - xu) / np.linalg.norm(x))
    assert errs[0] > 1e-2
    for a, b in zip(errs, errs[1:]):
        assert 0.4 < b / a < 0.6, errs


def test_mirror_symmetric_pair():
    V, T, v, t = _pair(4.0)
    nv = len(v)
    P = O.Problem(V, T, K0, None, None, nss=4, objects=([3.0, 3.0], [1.5, 1.5]))
    x = P.solve_direct(P.rhs())
    vm = v * [-1.0, 1.0, 1.0]
    idx = np.array([np.argmin(np.linalg.norm(v - p, axis=1)) for p in vm])
    # object 1 is object 0 mirrored in x = 0; the plane wave along +z is even
    for half in (0, 2 * nv):
        a, b = x[half:half + nv], x[half + nv:half + 2 * nv][idx]
        assert np.abs(a - b).max() < 1e-5 * np.abs(x).max()


def test_block_osrc_gmres_equals_direct():
    V, T, _, _ = _pair(4.0)
    P = O.Problem(V, T, K0, None, None, nss=4, objects=MATS)
    b = P.rhs()
    x = P.solve_direct(b)
    xg, it, hist = P.solve_gmres(b, tol=1e-10, maxit=300)
    assert hist[-1] <= 1e-10 and it < 60
    assert np.linalg.norm(xg - x) / np.linalg.norm(x) < 1e-8


def test_field_of_objects():
    v, t = icosphere(2)
    P = O.Problem(v, t, K0, 3.0, 1.5, nss=4)
    x = P.solve_direct(P.rhs())
    rng = np.random.default_rng(0)
    d = rng.standard_normal((40, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    pts = d * np.concatenate([rng.uniform(0, 0.6, 20), rng.uniform(1.5, 3, 20)])[:, None]
    u1, ins = O.field(v, t, K0, 3.0, 1.5, x, pts)
    u2, reg = O.field_objects(v, t, K0, [3.0], [1.5], x, pts)
    assert (reg == ins.astype(int)).all()
    assert np.abs(u1 - u2).max() < 1e-13 * np.abs(u1).max()
