"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Sizes: a Fibonacci-hull sphere with 150 vertices / 296 triangles (1776 rule
points: several 128-thread blocks and 64-triangle tiles, each with a ragged
tail), a level-3 icosphere, and sampled rows at the full 10242-vertex
icosphere.  Tolerances: FP32 far field 1e-5 relative (operator apply),
FP64 near field / right-hand sides 1e-10, inner Krylov solves 1e-7
(COCG/CG stopped at 1e-10 relative residual), solutions 1e-5 after GMRES
to 1e-8 (FP32 operator) and 1e-8 for the FP64 dense path."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2104_04609_gb300.inputs import fibonacci_hull, icosphere

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K0, K1, RHO = 2.0, 3.0, 1.5


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


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
    yield v, t, S
    S.close()


@pytest.fixture(scope="module")
def small_ref(small):
    v, t, S = small
    nss = S.params.n_ss
    far = O.pmchwt_matrix(v, t, K0, K1, RHO, nss=nss, part=1)
    near = O.pmchwt_matrix(v, t, K0, K1, RHO, nss=nss, part=2)
    M, Sm = O.mass_stiffness(v, t)
    return far, near, M, Sm


def _apply(B, S, x, form=0, part=3):
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda().reshape(1, -1)
    y = torch.empty_like(xt)
    B.osrc_pmchwt_apply(S.pb, xt, y, 1, form, part)
    torch.cuda.synchronize()
    return y.cpu().numpy().ravel()


def test_far_field_parity(B, small, small_ref):
    v, t, S = small
    far, _, _, _ = small_ref
    for seed in range(3):
        x = _rand(2 * v.shape[0], seed)
        y = _apply(B, S, x, part=B.OSRC_PART_FAR)
        ref = far @ x
        assert _rel(y, ref) < 1e-5
        assert np.abs(y - ref).max() < 1e-5 * np.abs(ref).max()


def test_far_field_parity_large_phase(B, small):
    """k r up to ~250 rad: the kernel switches to its centred variant (phase
    of the centroid distance in float-float arithmetic, offsets in FP32)."""
    v, t, S0 = small
    k0, k1 = 40.0, 70.0
    S = B.Solver(v, t, k0, k1, RHO)
    try:
        far = O.pmchwt_matrix(v, t, k0, k1, RHO, nss=S.params.n_ss, part=1)
        x = _rand(2 * v.shape[0], 17)
        y = _apply(B, S, x, part=B.OSRC_PART_FAR)
        assert _rel(y, far @ x) < 1e-5
    finally:
        S.close()


@pytest.mark.parametrize("phase_pi", [31.0, 33.0])
def test_far_field_parity_top_of_plain_phase_range(B, small, phase_pi):
    """The plain far kernel feeds k r straight to the FP32 sine / cosine until
    k_max x (bounding-box diagonal) exceeds 32 pi, then switches to the centred
    variant.  31 pi: just below the switch, where the plain variant's FP32
    phase error is largest (phases up to about k_max x diameter = 56 rad on
    this sphere); 33 pi: the centred variant just above it."""
    v, t, _ = small
    diag = float(np.linalg.norm(v.max(axis=0) - v.min(axis=0)))
    k1 = phase_pi * math.pi / diag
    k0 = 0.7 * k1
    S = B.Solver(v, t, k0, k1, RHO)
    try:
        far = O.pmchwt_matrix(v, t, k0, k1, RHO, nss=S.params.n_ss, part=1)
        for seed in (23, 24):
            x = _rand(2 * v.shape[0], seed)
            y = _apply(B, S, x, part=B.OSRC_PART_FAR)
            ref = far @ x
            assert _rel(y, ref) < 1e-5
            assert np.abs(y - ref).max() < 1e-5 * np.abs(ref).max()
    finally:
        S.close()


def test_near_field_parity(B, small, small_ref):
    v, t, S = small
    _, near, _, _ = small_ref
    x = _rand(2 * v.shape[0], 7)
    y = _apply(B, S, x, part=B.OSRC_PART_NEAR)
    ref = near @ x
    assert np.abs(y - ref).max() < 1e-10 * np.abs(ref).max()


def test_full_apply_weak_and_strong(B, small, small_ref):
    v, t, S = small
    far, near, M, _ = small_ref
    nv = v.shape[0]
    x = _rand(2 * nv, 11)
    ref = (far + near) @ x
    y = _apply(B, S, x)
    assert _rel(y, ref) < 1e-5
    ys = _apply(B, S, x, form=B.OSRC_STRONG)
    Md = M.toarray()
    ref_s = np.concatenate([np.linalg.solve(Md, ref[:nv]), np.linalg.solve(Md, ref[nv:])])
    assert _rel(ys, ref_s) < 1e-5


def test_mass_and_osrc_preconditioner(B, small, small_ref):
    v, t, S = small
    _, _, M, Sm = small_ref
    nv = v.shape[0]
    x = _rand(2 * nv, 3)
    xt = torch.from_numpy(x).cuda().reshape(1, -1)
    y = torch.empty_like(xt)
    B.osrc_mass_solve(S.pb, xt, y)
    Md = M.toarray()
    ref = np.concatenate([np.linalg.solve(Md, x[:nv]), np.linalg.solve(Md, x[nv:])])
    assert _rel(y.cpu().numpy().ravel(), ref) < 1e-8
    B.osrc_precond_apply(S.pb, xt, y)
    k = K1  # interior wavenumber (default side)
    R = O.mean_edge_length(v, t)
    ke = O.damped_wavenumber(k, R)
    z1, z2 = O.osrc_apply(M, Sm, x[:nv], x[nv:], k, ke, 4, math.pi / 3)
    assert _rel(y.cpu().numpy().ravel(), np.concatenate([z1, z2])) < 1e-7


def test_rhs_parity(B, small):
    v, t, S = small
    d = np.array([[0.6, 0.0, 0.8]])
    b = S.rhs_planewave(d).cpu().numpy().ravel()
    assert _rel(b, O.rhs(v, t, K0, "planewave", d[0])) < 1e-12
    src = np.array([[2.5, 0.3, -0.4]])
    b = S.rhs_pointsource(src).cpu().numpy().ravel()
    assert _rel(b, O.rhs(v, t, K0, "point", src[0])) < 1e-12


def test_gmres_solve_matches_direct(B, small, small_ref):
    v, t, S = small
    far, near, _, _ = small_ref
    b = S.rhs_planewave([[0.0, 0.0, 1.0]])
    x, info = S.solve(b, tol=1e-8, maxit=300)
    ref = np.linalg.solve(far + near, b.cpu().numpy().ravel())
    assert info.converged == 1 and info.precond_residual <= 1e-8
    assert _rel(x.cpu().numpy().ravel(), ref) < 1e-5
    assert info.true_residual < 1e-5


def test_oracle_gmres_iterations_agree(B, small):
    v, t, S = small
    P = O.Problem(v, t, K0, K1, RHO, nss=S.params.n_ss)
    b = P.rhs()
    _, it_ref, _ = P.solve_gmres(b, tol=1e-6, maxit=300)
    bt = S.rhs_planewave([[0.0, 0.0, 1.0]])
    _, info = S.solve(bt, tol=1e-6, maxit=300)
    assert abs(info.iterations - it_ref) <= 2


@pytest.mark.parametrize("kind", ["mass", "calderon"])
def test_other_preconditioners(B, small, small_ref, kind):
    """Mass-only and Calderon preconditioning (Sec. 2.4, 2.5): the solution is
    the direct solve's and the iteration count the oracle's (+-2)."""
    v, t, S0 = small
    far, near, _, _ = small_ref
    code = {"mass": B.OSRC_PRECOND_MASS, "calderon": B.OSRC_PRECOND_CALDERON}[kind]
    S = B.Solver(v, t, K0, K1, RHO, precond=code)
    try:
        b = S.rhs_planewave([[0.0, 0.0, 1.0]])
        x, info = S.solve(b, tol=1e-8, maxit=400)
        ref = np.linalg.solve(far + near, b.cpu().numpy().ravel())
        assert info.converged == 1 and _rel(x.cpu().numpy().ravel(), ref) < 1e-5
        P = O.Problem(v, t, K0, K1, RHO, nss=S.params.n_ss, precond=kind)
        _, it_ref, _ = P.solve_gmres(P.rhs(), tol=1e-6, maxit=400)
        _, info6 = S.solve(b, tol=1e-6, maxit=400)
        assert abs(info6.iterations - it_ref) <= 2, (info6.iterations, it_ref)
    finally:
        S.close()


def test_dense_fp64_path(B):
    v, t = icosphere(2)
    S = B.Solver(v, t, K0, K1, RHO, precision=B.OSRC_FP64_DENSE)
    try:
        Bm = O.pmchwt_matrix(v, t, K0, K1, RHO, nss=S.params.n_ss)
        x = _rand(2 * v.shape[0], 5)
        y = _apply(B, S, x)
        assert _rel(y, Bm @ x) < 1e-12
        b = S.rhs_planewave([[0.0, 0.0, 1.0]])
        xs, info = S.solve(b, tol=1e-10, maxit=300)
        ref = np.linalg.solve(Bm, b.cpu().numpy().ravel())
        assert _rel(xs.cpu().numpy().ravel(), ref) < 1e-8
    finally:
        S.close()


def test_sphere642_solution_vs_oracle_and_mie(B):
    from test_oracle_solve import mie_traces

    v, t = icosphere(3)
    S = B.Solver(v, t, K0, K1, RHO)
    try:
        b = S.rhs_planewave([[0.0, 0.0, 1.0]])
        x, info = S.solve(b, tol=1e-8, maxit=300)
        x = x.cpu().numpy().ravel()
        P = O.Problem(v, t, K0, K1, RHO, nss=S.params.n_ss)
        ref = P.solve_direct(P.rhs())
        assert _rel(x, ref) < 1e-5
        nv = v.shape[0]
        phi_ex, psi_ex = mie_traces(K0, K1, RHO, 1.0, v[:, 2])
        assert _rel(x[nv:], phi_ex) < 0.02 and _rel(x[:nv], psi_ex) < 0.02
    finally:
        S.close()


def test_sphere10242_sampled_rows(B):
    """Full-size 10242-vertex icosphere at k = 20 / 26: the apply, as the
    bench runs it, against oracle rows computed one by one."""
    v, t = icosphere(5)
    k0, k1, rho = 20.0, 26.0, 1.5
    S = B.Solver(v, t, k0, k1, rho)
    try:
        nv = v.shape[0]
        x = _rand(2 * nv, 21)
        y = _apply(B, S, x)
        rows = np.random.default_rng(4).choice(nv, 24, replace=False)
        R1, R2 = O.pmchwt_rows(v, t, k0, k1, rho, rows, nss=S.params.n_ss)
        ref1, ref2 = R1 @ x, R2 @ x
        scale1, scale2 = np.abs(ref1).max(), np.abs(ref2).max()
        assert np.abs(y[rows] - ref1).max() < 1e-5 * scale1
        assert np.abs(y[nv + rows] - ref2).max() < 1e-5 * scale2
    finally:
        S.close()


def test_bumpy80000_point_source_sampled_rows(B):
    """Large workload: bumpy (2, 1, 1) ellipsoid, 80000 vertices / 159996
    triangles, k_ext 60, k_int 144 (phases up to ~650 rad, centred far
    kernel), point-source right-hand side; the apply against oracle rows."""
    from paper_2104_04609_gb300.inputs import workload

    W = workload("bumpy80000")
    v, t = W["verts"], W["tris"]
    S = B.Solver(v, t, W["k_ext"], W["k_int"], W["rho_ratio"])
    try:
        nv = v.shape[0]
        b = S.rhs_pointsource(W["src"]).cpu().numpy().ravel()
        assert _rel(b, O.rhs(v, t, W["k_ext"], "point", W["src"][0])) < 1e-12
        x = _rand(2 * nv, 33)
        y = _apply(B, S, x)
        rows = np.random.default_rng(5).choice(nv, 16, replace=False)
        R1, R2 = O.pmchwt_rows(v, t, W["k_ext"], W["k_int"], W["rho_ratio"], rows,
                               nss=S.params.n_ss)
        ref1, ref2 = R1 @ x, R2 @ x
        assert np.abs(y[rows] - ref1).max() < 1e-5 * np.abs(ref1).max()
        assert np.abs(y[nv + rows] - ref2).max() < 1e-5 * np.abs(ref2).max()
    finally:
        S.close()


def test_low_frequency(B, small):
    """k r far below 1 everywhere (k_ext 0.05, k_int 0.08 on the unit
    sphere): the apply and the OSRC-preconditioned solve still match."""
    v, t, _ = small
    k0, k1 = 0.05, 0.08
    S = B.Solver(v, t, k0, k1, RHO)
    try:
        ref = O.pmchwt_matrix(v, t, k0, k1, RHO, nss=S.params.n_ss)
        x = _rand(2 * v.shape[0], 19)
        y = _apply(B, S, x)
        assert _rel(y, ref @ x) < 1e-5
        b = S.rhs_planewave([[0.0, 0.0, 1.0]])
        xs, info = S.solve(b, tol=1e-8, maxit=300)
        assert _rel(xs.cpu().numpy().ravel(), np.linalg.solve(ref, b.cpu().numpy().ravel())) < 1e-5
    finally:
        S.close()


@pytest.mark.parametrize("k0,k1", [(1e-12, 3.0), (3.0, 1e-12)])
def test_extreme_wavenumber_ratio(B, small, k0, k1):
    """One wavenumber 1e-12 against 3: the far kernel writes its D normal term
    k0^2 G0 + (k1^2/rho) G1 as s (G0 + ratio G1) with s >= 1e-20 (k1^2/rho),
    so neither the scale underflows nor the ratio overflows in FP32."""
    v, t, _ = small
    S = B.Solver(v, t, k0, k1, RHO)
    try:
        far = O.pmchwt_matrix(v, t, k0, k1, RHO, nss=S.params.n_ss, part=1)
        x = _rand(2 * v.shape[0], 23)
        y = _apply(B, S, x, part=B.OSRC_PART_FAR)
        assert _rel(y, far @ x) < 1e-5
    finally:
        S.close()


def test_invalid_arguments_rejected(B, small):
    v, t, S = small
    x = torch.zeros((1, 2 * v.shape[0]), dtype=torch.complex128, device="cuda")
    with pytest.raises(B.OsrcError):
        B.osrc_pmchwt_apply(S.pb, x, x)          # aliasing input and output
    with pytest.raises(B.OsrcError):
        B.osrc_rhs_planewave(S.pb, np.array([[0.0, 0.0, 2.0]]), x)   # not a unit direction
    with pytest.raises(B.OsrcError):
        B.Solver(v, t, -1.0, K1, RHO)


def test_zero_rhs_gives_zero_solution(B, small):
    v, t, S = small
    b = torch.zeros((1, 2 * v.shape[0]), dtype=torch.complex128, device="cuda")
    x, info = S.solve(b, tol=1e-8)
    assert info.iterations == 0 and float(x.abs().max()) == 0.0


def test_launches_counted(B, small):
    v, t, S = small
    n0 = S.launches()
    _apply(B, S, _rand(2 * v.shape[0], 1))
    assert S.launches() >= n0 + 3
