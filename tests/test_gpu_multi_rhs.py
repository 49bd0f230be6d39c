"""Several right-hand sides per far-field launch, and GMRES advanced in
lockstep over them, against the FP64 oracle and against the one-right-hand-
side path (through the C ABI).

The far field of R vectors is one launch of up to 8 right-hand sides
(larger counts run as chunks of 8, 4, 2 and a single vector), sharing each
point pair's geometry and sine / cosine values.  Sizes: the 150-vertex
Fibonacci sphere (296 triangles: ragged 64-triangle blocks and 16-triangle
source tiles), R = 2, 3, 8, 13 (8 + 4 + 1), 16 (8 + 8); the centred variant
for large k r; sampled rows of the 10242-vertex sphere at R = 8 (the bench's
launch configuration).  Tolerance: 1e-5 relative, as the one-vector FP32
apply."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2104_04609_gb300.inputs import fibonacci_hull, icosphere, plane_wave_dirs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K0, K1, RHO = 2.0, 3.0, 1.5


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.fixture(scope="module")
def B():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2104_04609_gb300 import binding

    assert torch.cuda.is_available()
    return binding


@pytest.fixture(scope="module")
def small(B):
    v, t = fibonacci_hull(150)
    S = B.Solver(v, t, K0, K1, RHO)
    far = O.pmchwt_matrix(v, t, K0, K1, RHO, nss=S.params.n_ss, part=1)
    near = O.pmchwt_matrix(v, t, K0, K1, RHO, nss=S.params.n_ss, part=2)
    yield v, t, S, far, near
    S.close()


def _apply(B, S, X, part):
    xt = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    y = torch.empty_like(xt)
    B.osrc_pmchwt_apply(S.pb, xt, y, X.shape[0], B.OSRC_WEAK, part)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def _check(Y, REF, tol=1e-5):
    for y, ref in zip(Y, REF):
        assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < tol
        assert np.abs(y - ref).max() < tol * np.abs(ref).max()


@pytest.mark.parametrize("R", [2, 3, 8, 13, 16])
def test_multi_far_apply_vs_oracle(B, small, R):
    v, t, S, far, near = small
    X = _rand((R, 2 * v.shape[0]), 100 + R)
    _check(_apply(B, S, X, B.OSRC_PART_FAR), (far @ X.T).T)
    _check(_apply(B, S, X, B.OSRC_PART_ALL), ((far + near) @ X.T).T)
    Yn = _apply(B, S, X, B.OSRC_PART_NEAR)
    _check(Yn, (near @ X.T).T, 1e-10)


def test_multi_equals_single(B, small):
    """Each right-hand side of a multi launch equals the one-vector kernel's
    result to FP32 rounding (the sums run in another order)."""
    v, t, S, _, _ = small
    X = _rand((8, 2 * v.shape[0]), 5)
    Y = _apply(B, S, X, B.OSRC_PART_ALL)
    for r in range(8):
        y1 = _apply(B, S, X[r:r + 1], B.OSRC_PART_ALL)[0]
        assert np.linalg.norm(Y[r] - y1) / np.linalg.norm(y1) < 2e-6


def test_multi_far_apply_centred(B, small):
    """k_max x diagonal above the plain kernel's range: the centred variant
    (float-float centroid phases) of the several-right-hand-side kernel."""
    v, t, _, _, _ = small
    k0, k1 = 40.0, 70.0
    S = B.Solver(v, t, k0, k1, RHO)
    try:
        far = O.pmchwt_matrix(v, t, k0, k1, RHO, nss=S.params.n_ss, part=1)
        X = _rand((5, 2 * v.shape[0]), 31)   # 4 + 1
        _check(_apply(B, S, X, B.OSRC_PART_FAR), (far @ X.T).T)
    finally:
        S.close()


def test_multi_apply_objects_falls_back(B):
    """Two objects (per-object far kernel): the several-right-hand-side apply
    runs vector by vector and still matches the oracle."""
    v1, t1 = fibonacci_hull(80)
    v = np.vstack([v1 + [-2.0, 0, 0], v1 + [2.0, 0, 0]])
    t = np.vstack([t1, t1 + v1.shape[0]]).astype(np.int32)
    S = B.Solver(v, t, K0, 0.0, 0.0, objects=([3.0, 4.0], [1.5, 2.0]))
    try:
        A = O.pmchwt_matrix_objects(v, t, K0, [3.0, 4.0], [1.5, 2.0], nss=S.params.n_ss)
        X = _rand((3, 2 * v.shape[0]), 41)
        _check(_apply(B, S, X, B.OSRC_PART_ALL), (A @ X.T).T)
    finally:
        S.close()


def test_lockstep_gmres_matches_single_and_direct(B, small):
    v, t, S, far, near = small
    dirs = plane_wave_dirs(5, seed=9)
    b = S.rhs_planewave(dirs)
    xb, info = S.solve(b, tol=1e-8, maxit=300)
    A = far + near
    bn = b.cpu().numpy()
    for r in range(5):
        xs, inf1 = S.solve(b[r:r + 1].contiguous(), tol=1e-8, maxit=300)
        d = np.linalg.norm(xb[r].cpu().numpy() - xs[0].cpu().numpy()) / np.linalg.norm(xs[0].cpu().numpy())
        assert d < 1e-5, d
        xd = np.linalg.solve(A, bn[r])
        e = np.linalg.norm(xb[r].cpu().numpy() - xd) / np.linalg.norm(xd)
        assert e < 1e-5, e
    assert info.converged == 1 and info.total_iterations > 0


def test_lockstep_gmres_host_buffers_and_zero_rhs(B, small):
    """Host buffers (copies inside the call) and a zero right-hand side in the
    batch (its solution is zero, the others are unaffected)."""
    v, t, S, _, _ = small
    b = S.rhs_planewave(plane_wave_dirs(3, seed=4))
    b[1].zero_()
    hb = b.cpu().numpy().copy()
    hx = np.zeros_like(hb)
    B.osrc_gmres_solve(S.pb, hb, hx, 3, 1e-8, 300, host_buffers=True)
    xd, _ = S.solve(b, tol=1e-8, maxit=300)
    assert np.abs(hx[1]).max() == 0.0
    assert np.linalg.norm(hx - xd.cpu().numpy()) / np.linalg.norm(hx) < 1e-12


def test_multi_sampled_rows_sphere10242(B):
    """R = 8 at the bench's size and launch configuration: 16 sampled rows of
    both block rows against the oracle, for all 8 right-hand sides."""
    from paper_2104_04609_gb300.inputs import workload

    W = workload("sphere10242")
    v, t = W["verts"], W["tris"]
    S = B.Solver(v, t, W["k_ext"], W["k_int"], W["rho_ratio"])
    try:
        nv = v.shape[0]
        X = _rand((8, 2 * nv), 77)
        Y = _apply(B, S, X, B.OSRC_PART_ALL)
        rows = np.random.default_rng(3).choice(nv, 16, replace=False)
        R1, R2 = O.pmchwt_rows(v, t, W["k_ext"], W["k_int"], W["rho_ratio"], rows, nss=S.params.n_ss)
        for r in range(8):
            ref = np.concatenate([R1 @ X[r], R2 @ X[r]])
            got = np.concatenate([Y[r][rows], Y[r][nv + rows]])
            assert np.abs(got - ref).max() < 1e-5 * np.abs(ref).max()
        y1 = _apply(B, S, X[:1], B.OSRC_PART_ALL)[0]
        assert np.linalg.norm(Y[0] - y1) / np.linalg.norm(y1) < 2e-6
    finally:
        S.close()


def test_lockstep_more_than_sixteen_and_not_converged(B, small):
    """19 right-hand sides (two groups: 16 + 3) equal one-at-a-time solves;
    with an iteration cap below what some need, the call reports
    OSRC_NOT_CONVERGED and every run stopped at the cap."""
    v, t, S, _, _ = small
    b = S.rhs_planewave(plane_wave_dirs(19, seed=12))
    x, info = S.solve(b, tol=1e-8, maxit=300)
    assert info.converged == 1
    for r in (0, 15, 16, 18):
        xs, _ = S.solve(b[r:r + 1].contiguous(), tol=1e-8, maxit=300)
        d = np.linalg.norm(x[r].cpu().numpy() - xs[0].cpu().numpy()) / np.linalg.norm(xs[0].cpu().numpy())
        assert d < 1e-5, (r, d)
    x2, info2 = S.solve(b[:4].contiguous(), tol=1e-12, maxit=5, raise_on_nonconvergence=False)
    assert info2.converged == 0 and info2.total_iterations == 4 * 5
    assert np.isfinite(x2.cpu().numpy()).all()


def test_lockstep_calderon_falls_back(B, small):
    """The Calderon preconditioner applies the operator inside the
    preconditioner: several right-hand sides are then solved one at a time,
    with the same results as single solves."""
    v, t, _, far, near = small
    S = B.Solver(v, t, K0, K1, RHO, precond=B.OSRC_PRECOND_CALDERON)
    try:
        b = S.rhs_planewave(plane_wave_dirs(2, seed=8))
        x, _ = S.solve(b, tol=1e-8, maxit=300)
        xd = np.linalg.solve(far + near, b.cpu().numpy().T).T
        assert np.linalg.norm(x.cpu().numpy() - xd) / np.linalg.norm(xd) < 1e-5
    finally:
        S.close()
