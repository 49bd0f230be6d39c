"""The Mueller formulation (Sec. 2.2) on the GPU against the oracle: operator
parts (the identity blocks ride in the touching-pair CSR), the solve with
mass preconditioning (solution and iteration count), the FP64 dense path,
disjoint objects, and the level-3 sphere against the Mie series.
Tolerances as for PMCHWT."""
import numpy as np
import pytest

import oracle as O
from paper_2104_04609_gb300.inputs import fibonacci_hull, icosphere
from test_oracle_solve import mie_traces

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K0, K1, RHO = 2.0, 3.0, 1.5


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


@pytest.fixture(scope="module")
def B():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2104_04609_gb300 import binding

    return binding


def _apply(S, x, part):
    return S.apply(torch.tensor(x[None, :], device="cuda"), part=part).cpu().numpy().ravel()


@pytest.mark.parametrize("part,tol", [(1, 1e-5), (2, 1e-10), (3, 1e-5)])
def test_muller_operator(B, part, tol):
    v, t = fibonacci_hull(150)
    S = B.Solver(v, t, K0, K1, RHO, formulation=B.OSRC_MULLER)
    try:
        ref = O.pmchwt_matrix(v, t, K0, K1, RHO, nss=S.params.n_ss, part=part, formulation="muller")
        x = _rand(2 * len(v), 21)
        assert _rel(_apply(S, x, part), ref @ x) < tol
    finally:
        S.close()


def test_muller_solve(B):
    v, t = fibonacci_hull(150)
    S = B.Solver(v, t, K0, K1, RHO, formulation=B.OSRC_MULLER, precond=B.OSRC_PRECOND_MASS)
    try:
        P = O.Problem(v, t, K0, K1, RHO, nss=S.params.n_ss, formulation="muller", precond="mass")
        b = S.rhs_planewave([[0.0, 0.0, 1.0]])
        x, info = S.solve(b, tol=1e-8, maxit=300)
        assert _rel(x.cpu().numpy().ravel(), P.solve_direct(P.rhs())) < 1e-5
        _, it_ref, _ = P.solve_gmres(P.rhs(), tol=1e-6, maxit=300)
        _, info6 = S.solve(b, tol=1e-6, maxit=300)
        assert abs(info6.iterations - it_ref) <= 2, (info6.iterations, it_ref)
    finally:
        S.close()


def test_muller_dense_and_objects(B):
    v, t = fibonacci_hull(150)
    S = B.Solver(v, t, K0, K1, RHO, formulation=B.OSRC_MULLER, precision=B.OSRC_FP64_DENSE)
    try:
        ref = O.pmchwt_matrix(v, t, K0, K1, RHO, nss=S.params.n_ss, formulation="muller")
        x = _rand(2 * len(v), 22)
        assert _rel(_apply(S, x, 3), ref @ x) < 1e-12
    finally:
        S.close()
    V = np.vstack([v + [-2.0, 0, 0], v + [2.0, 0, 0]])
    T = np.vstack([t, t + len(v)])
    mats = ([3.0, 1.5], [1.5, 0.8])
    S = B.Solver(V, T, K0, None, None, objects=mats, formulation=B.OSRC_MULLER)
    try:
        ref = O.pmchwt_matrix_objects(V, T, K0, *mats, nss=S.params.n_ss, formulation="muller")
        x = _rand(2 * len(V), 23)
        assert _rel(_apply(S, x, 3), ref @ x) < 1e-5
    finally:
        S.close()


def test_muller_sphere642_vs_mie(B):
    v, t = icosphere(3)
    S = B.Solver(v, t, K0, K1, RHO, formulation=B.OSRC_MULLER, precond=B.OSRC_PRECOND_MASS)
    try:
        b = S.rhs_planewave([[0.0, 0.0, 1.0]])
        x, info = S.solve(b, tol=1e-8, maxit=300)
        x = x.cpu().numpy().ravel()
        nv = len(v)
        phi, psi = mie_traces(K0, K1, RHO, 1.0, v[:, 2])
        assert _rel(x[nv:], phi) < 0.02 and _rel(x[:nv], psi) < 0.02
    finally:
        S.close()
