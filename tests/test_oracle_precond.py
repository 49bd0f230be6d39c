"""Pins of the alternative preconditioners the paper compares OSRC with
(Sec. 2.4 mass preconditioning, Sec. 2.5 Calderon preconditioning): the
Calderon identity puts the spectrum of the Calderon-preconditioned PMCHWT
operator of a scatterer without contrast (k_int = k_ext, rho = 1) next to
+1 and -1 at every mesh size; with contrast it stays clustered; every
preconditioner leaves the solution unchanged."""
import numpy as np

import oracle as O
from paper_2104_04609_gb300.inputs import icosphere


def _calderon_spectrum(lev, k0, k1, rho):
    v, t = icosphere(lev)
    P = O.Problem(v, t, k0, k1, rho, nss=4, precond="calderon")
    n = 2 * v.shape[0]
    C = np.stack([P.apply_preconditioned(e) for e in np.eye(n)], axis=1)
    return np.linalg.eigvals(C)


def test_calderon_identity_without_contrast():
    """Without contrast the PMCHWT operator is twice a Calderon projector,
    whose square is a quarter of the identity: every eigenvalue of the
    preconditioned operator lies near +1 or -1, at every mesh size."""
    for lev in (2, 3):
        ev = _calderon_spectrum(lev, 2.0, 2.0, 1.0)
        assert np.abs(np.abs(ev) - 1.0).max() < 0.1, lev
        assert np.abs(ev.imag).max() < 0.05, lev


def test_calderon_spectrum_clustered_with_contrast():
    ev = _calderon_spectrum(2, 2.0, 3.0, 1.5)
    assert np.abs(ev).min() > 0.5 and np.abs(ev).max() < 2.0


def test_preconditioners_keep_the_solution():
    v, t = icosphere(2)
    ref = None
    for kind in ("osrc", "mass", "calderon"):
        P = O.Problem(v, t, 2.0, 3.0, 1.5, nss=4, precond=kind)
        b = P.rhs()
        if ref is None:
            ref = P.solve_direct(b)
        x, it, hist = P.solve_gmres(b, tol=1e-10, maxit=400)
        assert hist[-1] <= 1e-10
        assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-8, kind
