"""The float-float dense assembly (OSRC_ASSEMBLE_FF) against the oracle and
against the FP64 assembly: operator applies of the assembled system, two
objects, the Mueller formulation, the batched solve, large phases, and the
FP64 fallback for attenuating interiors.

Tolerances: 1e-12 relative against the FP64 oracle at phases k r < 10
(float-float keeps about 48 bits; the FP64 assembly meets the same bound);
2e-12 against the FP64 assembly at phases up to about 90 rad (the phase
itself carries a float-float rounding of about 2^-48 k r); the batched solve
as for the FP64 assembly (true residual 1e-10, solution 1e-8)."""
import numpy as np
import pytest

import oracle as O
from paper_2104_04609_gb300.inputs import fibonacci_hull, icosphere

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


def _apply(S, x):
    return S.apply(torch.tensor(x[None, :], device="cuda")).cpu().numpy().ravel()


def _solver(B, v, t, k0, k1, rho, **kw):
    return B.Solver(v, t, k0, k1, rho, precision=B.OSRC_FP64_DENSE, dense_assembly=B.OSRC_ASSEMBLE_FF, **kw)


def test_ff_apply_matches_oracle(B):
    v, t = fibonacci_hull(150)
    S = _solver(B, v, t, K0, K1, RHO)
    try:
        ref = O.pmchwt_matrix(v, t, K0, K1, RHO, nss=S.params.n_ss)
        for seed in range(2):
            x = _rand(2 * len(v), 60 + seed)
            assert _rel(_apply(S, x), ref @ x) < 1e-12
    finally:
        S.close()


@pytest.mark.parametrize("formulation", ["pmchwt", "muller"])
def test_ff_objects_and_muller(B, formulation):
    v, t = fibonacci_hull(150)
    V = np.vstack([v + [-2.0, 0, 0], v + [2.0, 0, 0]])
    T = np.vstack([t, t + len(v)])
    mats = ([3.0, 1.5], [1.5, 0.8])
    form = B.OSRC_MULLER if formulation == "muller" else B.OSRC_PMCHWT
    S = _solver(B, V, T, K0, None, None, objects=mats, formulation=form)
    try:
        ref = O.pmchwt_matrix_objects(V, T, K0, *mats, nss=S.params.n_ss, formulation=formulation)
        x = _rand(2 * len(V), 62)
        assert _rel(_apply(S, x), ref @ x) < 1e-12
    finally:
        S.close()


def test_ff_large_phase_vs_fp64_assembly(B):
    """icosphere(4) at k 20 / 36: phases k r up to about 72 rad."""
    v, t = icosphere(4)
    S = _solver(B, v, t, 20.0, 36.0, 1.9)
    D = B.Solver(v, t, 20.0, 36.0, 1.9, precision=B.OSRC_FP64_DENSE)
    try:
        for seed in range(2):
            x = _rand(2 * len(v), 64 + seed)
            assert _rel(_apply(S, x), _apply(D, x)) < 2e-12
    finally:
        S.close()
        D.close()


def test_ff_batched_solve(B):
    v, t = fibonacci_hull(150)
    S = _solver(B, v, t, K0, K1, RHO)
    try:
        Bm = O.pmchwt_matrix(v, t, K0, K1, RHO, nss=S.params.n_ss)
        b = S.rhs_planewave([[0.0, 0.0, 1.0], [0.6, 0.0, 0.8], [0.0, 1.0, 0.0]])
        xs = torch.zeros_like(b)
        info = B.osrc_dense_batched_solve(S.pb, b, xs, tol=1e-10, max_refine=12, inner_tol=1e-3,
                                          inner_maxit=200)
        assert info["residual"] <= 1e-10
        ref = np.linalg.solve(Bm, b.cpu().numpy().T).T
        assert np.abs(xs.cpu().numpy() - ref).max() < 1e-8 * np.abs(ref).max()
    finally:
        S.close()


def test_ff_request_with_attenuation_keeps_fp64(B):
    v, t = fibonacci_hull(150)
    S = _solver(B, v, t, K0, K1, RHO, k_int_im=0.4)
    try:
        ref = O.pmchwt_matrix(v, t, K0, K1 + 0.4j, RHO, nss=S.params.n_ss)
        x = _rand(2 * len(v), 66)
        assert _rel(_apply(S, x), ref @ x) < 1e-12
    finally:
        S.close()
