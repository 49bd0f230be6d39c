"""Disjoint objects with their own materials (Sec. 2.2, multiple scattering)
on the GPU against the oracle: operator parts, the block-diagonal OSRC
preconditioner, the GMRES solve, the field, the FP64 dense and batched
paths, and the large-ka far kernel.

Mesh: two 150-vertex Fibonacci spheres centred at (-2, 0, 0) and (2, 0, 0)
(592 triangles, 3552 rule points: ragged blocks and tiles, tiles straddling
the two objects).  Tolerances as for one object."""
import numpy as np
import pytest

import oracle as O
from paper_2104_04609_gb300.inputs import fibonacci_hull

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K0 = 2.0
MATS = ([3.0, 1.5], [1.5, 0.8])


def _pair():
    v, t = fibonacci_hull(150)
    return (np.vstack([v + [-2.0, 0, 0], v + [2.0, 0, 0]]), np.vstack([t, t + len(v)]))


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
def pair(B):
    V, T = _pair()
    S = B.Solver(V, T, K0, None, None, objects=MATS)
    P = O.Problem(V, T, K0, None, None, nss=S.params.n_ss, objects=MATS)
    yield V, T, S, P
    S.close()


def _apply(B, S, x, part):
    xt = torch.tensor(x[None, :], device="cuda")
    return S.apply(xt, part=part).cpu().numpy().ravel()


def test_objects_numbered_like_the_oracle(B, pair):
    V, T, S, P = pair
    assert B.osrc_mesh_objects(S.mesh) == 2
    tc, _ = O.components(T)
    assert tc[0] == 0 and tc[-1] == 1


@pytest.mark.parametrize("part,tol", [(1, 1e-5), (2, 1e-10), (3, 1e-5)])
def test_operator_parts(B, pair, part, tol):
    V, T, S, P = pair
    ref = O.pmchwt_matrix_objects(V, T, K0, *MATS, nss=S.params.n_ss, part=part)
    x = _rand(2 * len(V), 11)
    assert _rel(_apply(B, S, x, part), ref @ x) < tol


def test_block_osrc_preconditioner(B, pair):
    V, T, S, P = pair
    x = _rand(2 * len(V), 12)
    y = S.precond(torch.tensor(x[None, :], device="cuda")).cpu().numpy().ravel()
    assert _rel(y, P.precond(x)) < 1e-7


def test_solve_matches_direct_and_oracle_iterations(B, pair):
    V, T, S, P = pair
    b = S.rhs_planewave([[0.0, 0.0, 1.0]])
    x, info = S.solve(b, tol=1e-8, maxit=300)
    ref = P.solve_direct(P.rhs())
    assert _rel(x.cpu().numpy().ravel(), ref) < 1e-5
    _, it_ref, _ = P.solve_gmres(P.rhs(), tol=1e-6, maxit=300)
    _, info6 = S.solve(b, tol=1e-6, maxit=300)
    assert abs(info6.iterations - it_ref) <= 2, (info6.iterations, it_ref)


def test_field_of_objects(B, pair):
    V, T, S, P = pair
    x = _rand(2 * len(V), 13)
    rng = np.random.default_rng(5)
    d = rng.standard_normal((90, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    r = np.concatenate([rng.uniform(0, 0.6, 60), rng.uniform(1.5, 3, 30)])
    c = np.where(np.arange(90)[:, None] % 2 == 0, [-2.0, 0, 0], [2.0, 0, 0])
    pts = d * r[:, None] + np.where(np.arange(90)[:, None] < 60, c, 0.0)
    pts[60:] *= 2.5  # outside both
    u, reg = S.field(torch.tensor(x, device="cuda"), torch.tensor(pts, device="cuda"),
                     B.OSRC_INC_PLANEWAVE, [0.0, 0.0, 1.0])
    ref, rr = O.field_objects(V, T, K0, *MATS, x, pts)
    assert (reg.cpu().numpy() == rr).all() and set(rr[:60]) == {1, 2}
    assert _rel(u.cpu().numpy(), ref) < 1e-10


def test_dense_and_batched_paths(B):
    V, T = _pair()
    S = B.Solver(V, T, K0, None, None, objects=MATS, precision=B.OSRC_FP64_DENSE)
    try:
        Bm = O.pmchwt_matrix_objects(V, T, K0, *MATS, nss=S.params.n_ss)
        x = _rand(2 * len(V), 14)
        assert _rel(_apply(B, S, x, 3), Bm @ x) < 1e-12
        b = S.rhs_planewave([[0.0, 0.0, 1.0], [0.6, 0.0, 0.8]])
        xs = torch.zeros_like(b)
        info = B.osrc_dense_batched_solve(S.pb, b, xs, tol=1e-10, max_refine=12, inner_tol=1e-3,
                                          inner_maxit=200)
        assert info["residual"] <= 1e-10
        ref = np.linalg.solve(Bm, b.cpu().numpy().T).T
        assert np.abs(xs.cpu().numpy() - ref).max() < 1e-8 * np.abs(ref).max()
    finally:
        S.close()


def test_large_ka_far_kernel(B):
    """k_int up to 40 over a mesh 6 wide: the centred far kernel, per object."""
    V, T = _pair()
    mats = ([40.0, 25.0], [1.5, 0.8])
    S = B.Solver(V, T, 10.0, None, None, objects=mats)
    try:
        ref = O.pmchwt_matrix_objects(V, T, 10.0, *mats, nss=S.params.n_ss, part=1)
        x = _rand(2 * len(V), 15)
        assert _rel(_apply(B, S, x, 1), ref @ x) < 1e-5
    finally:
        S.close()
