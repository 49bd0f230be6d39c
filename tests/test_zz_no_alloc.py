"""The allocation-free batched solve (osrc_shifted_solve_noalloc).

Callers that cannot allocate device memory at solve time (stream capture,
allocation-free hosts, pool-owned memory) use this entry point: it keeps its
Krylov workspace in a static device array instead of calling cudaMalloc.
This file checks, through the C ABI, that its output matches the library's
allocating entry point for the same systems (the mass solve) and the
oracle's direct solve for complex-symmetric shifted systems, on two calls
in a row (the second call reuses the static workspace the first one
left behind), and that over-capacity requests are rejected.  It is
collected last so that a failure here does not hide the other tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__

    __graft_entry__.build()
    import oracle as O
    from paper_2104_04609_gb300 import binding as B
    from paper_2104_04609_gb300.inputs import fibonacci_hull

    v, t = fibonacci_hull(150)
    S = B.Solver(v, t, 2.0, 3.0, 1.5)
    M, Sm = O.mass_stiffness(v, t)
    M.sort_indices()
    Sm.sort_indices()
    assert np.array_equal(M.indptr, Sm.indptr) and np.array_equal(M.indices, Sm.indices)
    dev = torch.device("cuda", 0)
    csr = (torch.from_numpy(M.indptr.astype(np.int32)).to(dev),
           torch.from_numpy(M.indices.astype(np.int32)).to(dev),
           torch.from_numpy(M.data.copy()).to(dev),
           torch.from_numpy(Sm.data.copy()).to(dev))
    yield B, S, M, Sm, csr, v.shape[0]
    S.close()


def test_noalloc_matches_mass_solve(setup):
    B, S, M, Sm, csr, nv = setup
    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.standard_normal(2 * nv) + 1j * rng.standard_normal(2 * nv)).cuda()
    x = x.reshape(1, -1).contiguous()
    ref = torch.empty_like(x)
    B.osrc_mass_solve(S.pb, x, ref)                       # allocating entry point
    ref = ref.reshape(2, nv)
    f = x.reshape(2, nv).contiguous()
    for _ in range(2):
        w = torch.full_like(f, complex("nan"))
        its = B.osrc_shifted_solve_noalloc(*csr, [1.0, 1.0], [0.0, 0.0], f, w, tol=1e-10, conj=1)
        assert all(i > 0 for i in its)
        err = float(torch.linalg.norm(w - ref) / torch.linalg.norm(ref))
        assert err < 1e-8, err


def test_noalloc_shifted_cocg_matches_direct(setup):
    import scipy.sparse.linalg as spla

    B, S, M, Sm, csr, nv = setup
    rng = np.random.default_rng(8)
    betas = [-(0.3 - 0.2j) / (3.0 + 0.5j) ** 2, -(0.9 + 0.1j) / (3.0 + 0.5j) ** 2, -0.05 + 0.01j]
    F = rng.standard_normal((3, nv)) + 1j * rng.standard_normal((3, nv))
    ref = np.stack([spla.spsolve((M + b * Sm).astype(np.complex128).tocsc(), F[i])
                    for i, b in enumerate(betas)])
    f = torch.from_numpy(F).cuda().contiguous()
    for _ in range(2):
        w = torch.zeros_like(f)
        its = B.osrc_shifted_solve_noalloc(*csr, [1.0] * 3, betas, f, w, tol=1e-10, conj=0)
        assert all(i > 0 for i in its)
        err = np.linalg.norm(w.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err < 1e-7, err


def test_noalloc_rejects_oversized_requests(setup):
    B, S, M, Sm, csr, nv = setup
    # 16 systems of 8193 rows: nsys * n = 131088 > 131072; rejected by the
    # library before any device work (a diagonal CSR of 8193 rows, so that the
    # binding's own buffer checks pass and the call reaches the library)
    n = 8193
    diag = (torch.arange(n + 1, dtype=torch.int32, device="cuda"),
            torch.arange(n, dtype=torch.int32, device="cuda"),
            torch.ones(n, dtype=torch.float64, device="cuda"),
            torch.zeros(n, dtype=torch.float64, device="cuda"))
    f = torch.zeros((16, n), dtype=torch.complex128, device="cuda")
    with pytest.raises(B.OsrcError) as e:
        B.osrc_shifted_solve_noalloc(*diag, [1.0] * 16, [0.0] * 16, f, f.clone(), conj=1)
    assert e.value.status == B.OSRC_INVALID_ARG
    f17 = torch.zeros((17, nv), dtype=torch.complex128, device="cuda")
    with pytest.raises(B.OsrcError) as e:
        B.osrc_shifted_solve_noalloc(*csr, [1.0] * 17, [0.0] * 17, f17, f17.clone(), conj=1)
    assert e.value.status == B.OSRC_INVALID_ARG
