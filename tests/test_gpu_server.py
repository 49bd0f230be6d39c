"""The serving loop (osrc_server_*): continuous batching of solve requests
with resident state and admission by device memory.  Each result must equal
the solve of the same request alone (and the synchronous GMRES entry point),
whatever else is running."""
import numpy as np
import pytest

from paper_2104_04609_gb300.inputs import fibonacci_hull, icosphere

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2104_04609_gb300 import binding

    return binding


def _params(B, k0, k1, rho):
    return B.osrc_params_default(k_ext=k0, k_int=k1, rho_ratio=rho)


def _serve(B, jobs, max_active, budget=0):
    """jobs: list of (verts, tris, (k0, k1, rho), dirs); returns results and stats."""
    ctx = B.osrc_create(0, budget)
    sv = B.osrc_server_create(ctx, max_active)
    try:
        ids = [B.osrc_server_submit(sv, v, t, _params(B, *k), d, tol=1e-8, maxit=300)
               for v, t, k, d in jobs]
        out = []
        for rid, (v, t, k, d) in zip(ids, jobs):
            assert B.osrc_server_wait(sv, rid, 300.0) == B.OSRC_OK
            done, st, lat, info = B.osrc_server_poll(sv, rid)
            assert done and st == B.OSRC_OK and lat > 0
            s, x = B.osrc_server_result(sv, rid, len(d), v.shape[0])
            assert s == B.OSRC_OK
            out.append((x, info))
        stats = B.osrc_server_get_stats(sv)
    finally:
        B.osrc_server_destroy(sv)
        B.osrc_destroy(ctx)
    return out, stats


def test_server_alone_equals_mix_and_direct(B):
    va, ta = fibonacci_hull(150)
    vb, tb = icosphere(2)
    vc, tc = fibonacci_hull(300)
    da = np.array([[0.0, 0.0, 1.0], [0.6, 0.0, 0.8]])
    job_a = (va, ta, (2.0, 3.0, 1.5), da)
    alone, _ = _serve(B, [job_a], max_active=1)
    mix = [(vb, tb, (3.0, 4.0, 1.2), np.array([[1.0, 0.0, 0.0]])),
           job_a,
           (vc, tc, (2.5, 5.0, 1.9), np.array([[0.0, 1.0, 0.0], [0.0, 0.0, -1.0], [0.8, 0.6, 0.0]])),
           job_a]
    mixed, stats = _serve(B, mix, max_active=4)
    xa = alone[0][0]
    assert np.array_equal(mixed[1][0], xa)      # bit-identical in the mix
    assert np.array_equal(mixed[3][0], xa)
    assert stats["cache_hits"] >= 1              # the repeated request reused resident state
    assert stats["active_peak"] >= 2             # jobs overlapped
    # requests with several right-hand sides ran as one lockstep block each
    assert stats["batched_jobs"] == 3
    # the synchronous entry point on its own problem gives the same solution
    S = B.Solver(va, ta, 2.0, 3.0, 1.5)
    try:
        b = S.rhs_planewave(da)
        x, info = S.solve(b, tol=1e-8, maxit=300)
        assert np.abs(x.cpu().numpy() - xa).max() <= 1e-12 * np.abs(xa).max()
    finally:
        S.close()


def test_server_admission_by_memory(B):
    """A budget that holds about one problem at a time: requests still finish,
    one after the other, with evictions of the resident state."""
    meshes = [fibonacci_hull(n) for n in (400, 500, 600)]
    jobs = [(v, t, (2.0, 3.0, 1.5), np.array([[0.0, 0.0, 1.0]])) for v, t in meshes]
    _, free_stats = _serve(B, jobs[2:], max_active=1)   # the largest alone
    one = free_stats["mem_peak"]
    out, stats = _serve(B, jobs, max_active=3, budget=int(1.6 * one))
    assert len(out) == 3
    assert stats["evictions"] >= 1
    assert stats["mem_peak"] <= int(1.6 * one)


def test_server_rejects_what_never_fits(B):
    v, t = fibonacci_hull(400)
    ctx = B.osrc_create(0, 1 << 20)      # 1 MiB: no problem fits
    sv = B.osrc_server_create(ctx, 2)
    try:
        rid = B.osrc_server_submit(sv, v, t, _params(B, 2.0, 3.0, 1.5), [[0.0, 0.0, 1.0]])
        st = B.osrc_server_wait(sv, rid, 60.0)
        assert st == B.OSRC_OUT_OF_MEMORY
    finally:
        B.osrc_server_destroy(sv)
        B.osrc_destroy(ctx)


def test_server_batches_dense_requests(B):
    """A request with precision OSRC_FP64_DENSE is solved as one block of
    right-hand sides by the batched mixed-precision solve on the resident
    problem: the result equals the direct batched solve of the same block,
    alone and in a mix with matrix-free requests, within the dense path's
    solution tolerance (1e-8), and matches the oracle's FP64 direct solve."""
    import oracle as O

    va, ta = fibonacci_hull(150)
    dirs = np.array([[0.0, 0.0, 1.0], [0.6, 0.0, 0.8], [0.0, -0.8, 0.6]])
    k = (2.0, 3.0, 1.5)

    def serve(jobs, max_active):
        ctx = B.osrc_create(0, 0)
        sv = B.osrc_server_create(ctx, max_active)
        try:
            ids = []
            for v, t, kk, d, prec in jobs:
                p = _params(B, *kk)
                p.precision = prec
                ids.append(B.osrc_server_submit(sv, v, t, p, d, tol=1e-10, maxit=300))
            out = []
            for rid, (v, t, kk, d, prec) in zip(ids, jobs):
                assert B.osrc_server_wait(sv, rid, 300.0) == B.OSRC_OK
                done, st, lat, info = B.osrc_server_poll(sv, rid)
                assert done and st == B.OSRC_OK
                s, x = B.osrc_server_result(sv, rid, len(d), v.shape[0])
                out.append(x)
            return out, B.osrc_server_get_stats(sv)
        finally:
            B.osrc_server_destroy(sv)
            B.osrc_destroy(ctx)

    dense_job = (va, ta, k, dirs, B.OSRC_FP64_DENSE)
    alone, st1 = serve([dense_job], 1)
    assert st1["batched_jobs"] == 1
    vb, tb = icosphere(2)
    mix = [(vb, tb, (3.0, 4.0, 1.2), np.array([[1.0, 0.0, 0.0]]), B.OSRC_FP32_MATFREE), dense_job,
           (vb, tb, (3.0, 4.0, 1.2), np.array([[0.0, 1.0, 0.0]]), B.OSRC_FP32_MATFREE), dense_job]
    mixed, st2 = serve(mix, 3)
    assert st2["batched_jobs"] == 2 and st2["cache_hits"] >= 1
    xa = alone[0]
    # the dense assembly adds in a fixed order (no atomics), so a batched
    # request gives the same bytes alone and in the mix
    for x in (mixed[1], mixed[3]):
        assert np.array_equal(x, xa)
    S = B.Solver(va, ta, *k, precision=B.OSRC_FP64_DENSE)
    try:
        b = S.rhs_planewave(dirs)
        x = torch.zeros_like(b)
        B.osrc_dense_precond_build(S.pb, tol=1e-3, maxit=500)  # as the server does
        B.osrc_dense_batched_solve(S.pb, b, x, tol=1e-10, max_refine=10, inner_tol=1e-3,
                                   inner_maxit=400)
        assert np.abs(x.cpu().numpy() - xa).max() <= 1e-8 * np.abs(xa).max()
        Bm = O.pmchwt_matrix(va, ta, *k, nss=S.params.n_ss)
        ref = np.linalg.solve(Bm, b.cpu().numpy().T).T
        assert np.abs(xa - ref).max() <= 1e-8 * np.abs(ref).max()
    finally:
        S.close()


def test_server_batched_requests_overlap(B):
    """Batched requests on different meshes run concurrently (each on its own
    host thread and stream); every result equals the same request served
    alone, within the dense path's solution tolerance."""
    meshes = [fibonacci_hull(n) for n in (150, 200, 250)]
    dirs = np.array([[0.0, 0.0, 1.0], [0.6, 0.0, 0.8]])

    def serve(jobs, max_active):
        ctx = B.osrc_create(0, 0)
        sv = B.osrc_server_create(ctx, max_active)
        try:
            ids = []
            for v, t in jobs:
                p = _params(B, 2.0, 3.0, 1.5)
                p.precision = B.OSRC_FP64_DENSE
                ids.append(B.osrc_server_submit(sv, v, t, p, dirs, tol=1e-10, maxit=300))
            out = []
            for rid, (v, t) in zip(ids, jobs):
                assert B.osrc_server_wait(sv, rid, 300.0) == B.OSRC_OK
                done, st, lat, info = B.osrc_server_poll(sv, rid)
                assert done and st == B.OSRC_OK
                out.append(B.osrc_server_result(sv, rid, len(dirs), v.shape[0])[1])
            return out, B.osrc_server_get_stats(sv)
        finally:
            B.osrc_server_destroy(sv)
            B.osrc_destroy(ctx)

    alone = [serve([m], 1)[0][0] for m in meshes]
    mixed, stats = serve(meshes, 3)
    assert stats["batched_jobs"] == 3 and stats["active_peak"] >= 2
    for a, x in zip(alone, mixed):
        assert np.array_equal(x, a)
