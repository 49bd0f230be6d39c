"""A non-smooth domain (Sec. 3.4): the level-1 Menger sponge (right-angled
edges and corners, concave tunnels) on the GPU against the oracle: operator
parts, the OSRC preconditioner and the solve."""
import numpy as np
import pytest

import oracle as O
from paper_2104_04609_gb300.inputs import menger_sponge

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K0, RHO = 5.0, 1.9
K1 = K0 * 1500.0 / 3600.0  # bone-like interior


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def B():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2104_04609_gb300 import binding

    return binding


def test_sponge_operator_and_solve(B):
    v, t = menger_sponge(1, 2, edge=2.0)
    S = B.Solver(v, t, K0, K1, RHO)
    try:
        rng = np.random.default_rng(41)
        x = rng.standard_normal(2 * len(v)) + 1j * rng.standard_normal(2 * len(v))
        xt = torch.tensor(x[None, :], device="cuda")
        for part, tol in ((1, 1e-5), (2, 1e-10), (3, 1e-5)):
            ref = O.pmchwt_matrix(v, t, K0, K1, RHO, nss=S.params.n_ss, part=part)
            y = S.apply(xt, part=part).cpu().numpy().ravel()
            assert _rel(y, ref @ x) < tol, part
        P = O.Problem(v, t, K0, K1, RHO, nss=S.params.n_ss)
        z = S.precond(xt).cpu().numpy().ravel()
        assert _rel(z, P.precond(x)) < 1e-7
        b = S.rhs_planewave([[1.0, 0.0, 0.0]])
        xs, info = S.solve(b, tol=1e-8, maxit=400)
        assert _rel(xs.cpu().numpy().ravel(), P.solve_direct(P.rhs(src=(1.0, 0.0, 0.0)))) < 1e-5
    finally:
        S.close()
