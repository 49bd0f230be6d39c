"""The inner solvers of the preconditioner (mass CG, OSRC shifted COCG,
Sec. 2.4 and 2.6) in both of their kernels, against the oracle's direct
sparse solves:

- the mixed-precision refinement kernel at the headline size (10242-vertex
  icosphere, k 20 / 26: 16-CTA clusters, two rows per thread), the launch
  configuration the benchmark times;
- the all-FP64 kernel, which serves meshes whose per-CTA slices exceed the
  mixed kernel's limits (40962-vertex icosphere: 2561 rows per CTA).

Both stop at relative residual 1e-10, so the preconditioned vectors agree
with the oracle to 1e-7 (as for the small meshes of the parity tests)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2104_04609_gb300.inputs import icosphere

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RHO = 1.5


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

    return binding


def _check_precond(B, level, k0, k1, seed):
    v, t = icosphere(level)
    nv = len(v)
    S = B.Solver(v, t, k0, k1, RHO)
    try:
        M, Sm = O.mass_stiffness(v, t)
        x = _rand(2 * nv, seed)
        xt = torch.from_numpy(x).cuda().reshape(1, -1)
        y = torch.empty_like(xt)
        B.osrc_mass_solve(S.pb, xt, y)
        import scipy.sparse.linalg as spla

        lu = spla.splu(M.tocsc().astype(complex))
        ref = np.concatenate([lu.solve(x[:nv]), lu.solve(x[nv:])])
        assert _rel(y.cpu().numpy().ravel(), ref) < 1e-8
        B.osrc_precond_apply(S.pb, xt, y)
        R = O.mean_edge_length(v, t)
        z1, z2 = O.osrc_apply(M, Sm, x[:nv], x[nv:], k1, O.damped_wavenumber(k1, R), 4, math.pi / 3)
        assert _rel(y.cpu().numpy().ravel(), np.concatenate([z1, z2])) < 1e-7
    finally:
        S.close()


def test_mixed_kernel_headline_size(B):
    _check_precond(B, 5, 20.0, 26.0, 41)


def test_fp64_kernel_large_mesh(B):
    _check_precond(B, 6, 20.0, 26.0, 42)
