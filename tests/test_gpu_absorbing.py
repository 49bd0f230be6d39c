"""An attenuating interior (complex wavenumber k_int + i k_int_im, Sec. 3.1)
on the GPU against the oracle: operator parts, the OSRC preconditioner with
its complex wavenumber, the solve, the field, the FP64 dense and batched
paths, disjoint objects, the large-ka far kernel, and the level-3 sphere
against the Mie series of the absorbing sphere.  Tolerances as without
attenuation."""
import numpy as np
import pytest

import oracle as O
from paper_2104_04609_gb300.inputs import fibonacci_hull, icosphere
from test_oracle_solve import mie_traces

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K0, K1R, K1I, RHO = 2.0, 3.0, 0.4, 1.5
K1 = K1R + 1j * K1I


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


@pytest.fixture(scope="module")
def sph(B):
    v, t = fibonacci_hull(150)
    S = B.Solver(v, t, K0, K1R, RHO, k_int_im=K1I)
    P = O.Problem(v, t, K0, K1, RHO, nss=S.params.n_ss)
    yield v, t, S, P
    S.close()


def _apply(S, x, part):
    return S.apply(torch.tensor(x[None, :], device="cuda"), part=part).cpu().numpy().ravel()


@pytest.mark.parametrize("part,tol", [(1, 1e-5), (2, 1e-10), (3, 1e-5)])
def test_operator_parts(B, sph, part, tol):
    v, t, S, P = sph
    ref = O.pmchwt_matrix(v, t, K0, K1, RHO, nss=S.params.n_ss, part=part)
    x = _rand(2 * len(v), 31)
    assert _rel(_apply(S, x, part), ref @ x) < tol


def test_osrc_and_solve(B, sph):
    v, t, S, P = sph
    x = _rand(2 * len(v), 32)
    y = S.precond(torch.tensor(x[None, :], device="cuda")).cpu().numpy().ravel()
    assert _rel(y, P.precond(x)) < 1e-7
    b = S.rhs_planewave([[0.0, 0.0, 1.0]])
    xs, info = S.solve(b, tol=1e-8, maxit=300)
    assert _rel(xs.cpu().numpy().ravel(), P.solve_direct(P.rhs())) < 1e-5
    _, it_ref, _ = P.solve_gmres(P.rhs(), tol=1e-6, maxit=300)
    _, info6 = S.solve(b, tol=1e-6, maxit=300)
    assert abs(info6.iterations - it_ref) <= 2, (info6.iterations, it_ref)


def test_field(B, sph):
    v, t, S, P = sph
    x = _rand(2 * len(v), 33)
    rng = np.random.default_rng(6)
    d = rng.standard_normal((80, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    pts = d * np.concatenate([rng.uniform(0, 0.7, 40), rng.uniform(1.4, 3, 40)])[:, None]
    u, reg = S.field(torch.tensor(x, device="cuda"), torch.tensor(pts, device="cuda"),
                     B.OSRC_INC_PLANEWAVE, [0.0, 0.0, 1.0])
    ref, ins = O.field(v, t, K0, K1, RHO, x, pts)
    assert (reg.cpu().numpy() == ins).all()
    assert _rel(u.cpu().numpy(), ref) < 1e-10


def test_dense_batched_and_objects(B):
    v, t = fibonacci_hull(150)
    S = B.Solver(v, t, K0, K1R, RHO, k_int_im=K1I, precision=B.OSRC_FP64_DENSE)
    try:
        Bm = O.pmchwt_matrix(v, t, K0, K1, RHO, nss=S.params.n_ss)
        x = _rand(2 * len(v), 34)
        assert _rel(_apply(S, x, 3), Bm @ x) < 1e-12
        b = S.rhs_planewave([[0.0, 0.0, 1.0], [0.6, 0.0, 0.8]])
        xs = torch.zeros_like(b)
        info = B.osrc_dense_batched_solve(S.pb, b, xs, tol=1e-10, max_refine=12, inner_tol=1e-3,
                                          inner_maxit=200)
        assert info["residual"] <= 1e-10
        ref = np.linalg.solve(Bm, b.cpu().numpy().T).T
        assert np.abs(xs.cpu().numpy() - ref).max() < 1e-8 * np.abs(ref).max()
    finally:
        S.close()
    V = np.vstack([v + [-2.0, 0, 0], v + [2.0, 0, 0]])
    T = np.vstack([t, t + len(v)])
    S = B.Solver(V, T, K0, None, None, objects=([3.0, 1.5], [1.5, 0.8]), k_int_im=K1I)
    try:
        ref = O.pmchwt_matrix_objects(V, T, K0, [3.0 + 1j * K1I, 1.5 + 1j * K1I], [1.5, 0.8],
                                      nss=S.params.n_ss)
        x = _rand(2 * len(V), 35)
        assert _rel(_apply(S, x, 3), ref @ x) < 1e-5
    finally:
        S.close()


def test_large_ka_far_kernel(B):
    v, t = fibonacci_hull(150)
    S = B.Solver(v, t, 40.0, 70.0, RHO, k_int_im=2.0)
    try:
        ref = O.pmchwt_matrix(v, t, 40.0, 70.0 + 2.0j, RHO, nss=S.params.n_ss, part=1)
        x = _rand(2 * len(v), 36)
        assert _rel(_apply(S, x, 1), ref @ x) < 1e-5
    finally:
        S.close()


def test_absorbing_sphere642_vs_mie(B):
    v, t = icosphere(3)
    S = B.Solver(v, t, K0, K1R, RHO, k_int_im=K1I)
    try:
        b = S.rhs_planewave([[0.0, 0.0, 1.0]])
        x, info = S.solve(b, tol=1e-8, maxit=300)
        x = x.cpu().numpy().ravel()
        nv = len(v)
        phi, psi = mie_traces(K0, K1, RHO, 1.0, v[:, 2])
        assert _rel(x[nv:], phi) < 0.02 and _rel(x[:nv], psi) < 0.02
    finally:
        S.close()
