"""Pins of the Mueller formulation (Sec. 2.2: the difference of the exterior
and interior Calderon equations plus the identity): it solves the same
transmission problem as PMCHWT (its solution converges to the Mie series at
the same O(h^2) rate), and without density contrast it is of the second
kind (the spectrum of the strong form stays bounded and bounded away from 0
under refinement)."""
import numpy as np

import oracle as O
from paper_2104_04609_gb300.inputs import icosphere
from test_oracle_solve import mie_traces


def _merr(M, a, e):
    d = a - e
    return np.sqrt(abs(np.vdot(d, M @ d)) / abs(np.vdot(e, M @ e)))


def test_muller_solution_converges_to_mie():
    errs = []
    for lev in (2, 3):
        v, t = icosphere(lev)
        nv = len(v)
        P = O.Problem(v, t, 2.0, 3.0, 1.5, nss=4, formulation="muller", precond="mass")
        x = P.solve_direct(P.rhs())
        phi, psi = mie_traces(2.0, 3.0, 1.5, 1.0, v[:, 2])
        errs.append(max(_merr(P.M, x[nv:], phi), _merr(P.M, x[:nv], psi)))
        xg, it, hist = P.solve_gmres(P.rhs(), tol=1e-10, maxit=300)
        assert np.linalg.norm(xg - x) / np.linalg.norm(x) < 1e-8
    assert errs[1] < 0.012 and errs[1] < errs[0] / 3, errs


def test_muller_second_kind_without_contrast():
    rng = []
    for lev in (2, 3):
        v, t = icosphere(lev)
        B = O.pmchwt_matrix(v, t, 2.0, 3.0, 1.0, nss=4, formulation="muller")
        Mi = np.linalg.inv(O.mass_stiffness(v, t)[0].toarray())
        Z = np.zeros_like(Mi)
        ev = np.abs(np.linalg.eigvals(np.block([[Mi, Z], [Z, Mi]]) @ B))
        rng.append((ev.min(), ev.max()))
    (a2, b2), (a3, b3) = rng
    assert a3 > 0.3 and b3 < 3.5 and abs(b3 / b2 - 1) < 0.1 and abs(a3 / a2 - 1) < 0.1, rng


def test_muller_objects_reduce_to_single():
    v, t = icosphere(2)
    a = O.pmchwt_matrix(v, t, 2.0, 3.0, 1.5, nss=4, formulation="muller")
    b = O.pmchwt_matrix_objects(v, t, 2.0, [3.0], [1.5], nss=4, formulation="muller")
    assert np.abs(a - b).max() < 1e-14 * np.abs(a).max()
