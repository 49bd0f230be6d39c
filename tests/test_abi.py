"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every symbol that include/osrc_pmchwt.h declares, and rejects invalid meshes
on the host (osrc_mesh_validate does no device work)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_04609_gb300 import build as libbuild
    from paper_2104_04609_gb300 import binding

    libbuild.build()
    return binding.lib()


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "osrc_pmchwt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(osrc_[a-z_0-9]+)\s*\(", src)))


def test_header_symbols_exported(lib):
    from paper_2104_04609_gb300 import binding

    names = _declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
        assert n in binding.SIGNATURES, f"binding misses {n}"


def test_status_strings(lib):
    from paper_2104_04609_gb300 import binding as B

    assert B.osrc_status_string(0) == "OSRC_OK"
    assert B.osrc_status_string(4) == "OSRC_NOT_CONVERGED"
    assert B.osrc_status_string(99) == "OSRC_UNKNOWN_STATUS"


def test_params_default(lib):
    from paper_2104_04609_gb300 import binding as B

    p = B.osrc_params_default()
    assert p.n_pade == 4 and abs(p.theta - np.pi / 3) < 1e-15 and p.osrc_side == 1
    assert p.inner_tol <= 1e-8


def test_mesh_validation(lib):
    from paper_2104_04609_gb300 import binding as B
    from paper_2104_04609_gb300.inputs import icosphere

    v, t = icosphere(1)
    assert B.osrc_mesh_validate(v, t) == B.OSRC_OK
    bad = t.copy(); bad[0, 0] = v.shape[0]            # index out of range
    assert B.osrc_mesh_validate(v, bad) == B.OSRC_INVALID_ARG
    bad = t.copy(); bad[0, 1] = bad[0, 0]             # repeated vertex
    assert B.osrc_mesh_validate(v, bad) == B.OSRC_INVALID_ARG
    bad = t.copy(); bad[3] = bad[3][[0, 2, 1]]        # flipped orientation
    assert B.osrc_mesh_validate(v, bad) == B.OSRC_INVALID_ARG
    assert B.osrc_mesh_validate(v, t[:-1]) == B.OSRC_INVALID_ARG   # open surface
    vv = v.copy(); vv[5] = np.nan
    assert B.osrc_mesh_validate(vv, t) == B.OSRC_INVALID_ARG
    vv = v.copy(); a, b, c = t[0]; vv[c] = vv[a] * 0.5 + vv[b] * 0.5   # zero area
    assert B.osrc_mesh_validate(vv, t) == B.OSRC_INVALID_ARG
    assert B.osrc_mesh_validate(np.zeros((0, 3)), np.zeros((0, 3), np.int32)) == B.OSRC_INVALID_ARG
    vx = np.vstack([v, [[5.0, 5.0, 5.0]]])            # unreferenced vertex
    assert B.osrc_mesh_validate(vx, t) == B.OSRC_INVALID_ARG


def test_input_meshes_valid(lib):
    from paper_2104_04609_gb300 import binding as B
    from paper_2104_04609_gb300.inputs import ellipsoid, icosphere, bumpy_ellipsoid

    for v, t in (icosphere(3), ellipsoid(500), bumpy_ellipsoid(800)):
        assert B.osrc_mesh_validate(v, t) == B.OSRC_OK
        assert t.shape[0] == 2 * v.shape[0] - 4


def test_struct_layouts_match_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    of the C structure in include/osrc_pmchwt.h (compiled with gcc)."""
    import ctypes
    import shutil
    import subprocess

    from paper_2104_04609_gb300 import binding as B

    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = [B.osrc_params, B.osrc_solve_info, B.osrc_batched_info, B.osrc_request, B.osrc_server_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "osrc_pmchwt.h"', "int main(void) {"]
    for S in structs:
        lines.append(f'    printf("{S.__name__} sizeof %zu\\n", sizeof({S.__name__}));')
        for name, _ in S._fields_:
            lines.append(f'    printf("{S.__name__} {name} %zu\\n", offsetof({S.__name__}, {name}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for S in structs:
        assert got[(S.__name__, "sizeof")] == ctypes.sizeof(S), S.__name__
        for name, _ in S._fields_:
            assert got[(S.__name__, name)] == getattr(S, name).offset, (S.__name__, name)


def test_unknown_params_rejected(lib):
    """A misspelt parameter raises instead of becoming a stray Python
    attribute of the ctypes structure (checked before any device call)."""
    from paper_2104_04609_gb300 import binding as B
    from paper_2104_04609_gb300.inputs import icosphere

    p = B.osrc_params_default(dense_assembly=B.OSRC_ASSEMBLE_FF, k_int_im=0.1)
    assert p.dense_assembly == B.OSRC_ASSEMBLE_FF and p.k_int_im == 0.1
    with pytest.raises(TypeError):
        B.osrc_params_default(dense_asembly=1)
    pytest.importorskip("torch")
    v, t = icosphere(1)
    with pytest.raises(TypeError):
        B.Solver(v, t, 2.0, 3.0, 1.5, precision=B.OSRC_FP64_DENSE, dense_asembly=1)


def test_short_buffers_rejected_on_the_host():
    """The binding's size check (the C ABI takes bare pointers) raises for a
    buffer shorter than the call needs, for tensors and numpy arrays."""
    from paper_2104_04609_gb300 import binding as B

    B._need(np.zeros(8), 8, "x")
    with pytest.raises(ValueError):
        B._need(np.zeros(7), 8, "x")
    torch = pytest.importorskip("torch")
    B._need(torch.zeros(2, 4, dtype=torch.complex128), 8, "x")
    with pytest.raises(ValueError):
        B._need(torch.zeros(2, 3, dtype=torch.complex128), 8, "x")


def test_gemm_shapes_rejected_on_the_host():
    """The tensor-core GEMM takes M, K, N and bare pointers: B must have A's
    K columns and C at least M x N, checked before any device call."""
    from paper_2104_04609_gb300 import binding as B

    torch = pytest.importorskip("torch")
    A = torch.zeros(256, 128, dtype=torch.bfloat16)
    Bm = torch.zeros(32, 128, dtype=torch.bfloat16)
    C = torch.zeros(256, 32)
    err = torch.zeros(1, dtype=torch.int32)
    assert B._gemm_shapes(A, Bm, C, err) == (256, 128, 32)
    assert B._gemm_shapes(A, Bm, torch.zeros(256, 48), err) == (256, 128, 32)  # ldc > N
    for bad in [(A, torch.zeros(32, 64, dtype=torch.bfloat16), C, err),   # K mismatch
                (A, Bm, torch.zeros(128, 32), err),                        # C too short
                (A, Bm, torch.zeros(256, 16), err),                        # C too narrow
                (A, Bm, C, torch.zeros(0, dtype=torch.int32)),             # no error word
                (A.reshape(-1), Bm, C, err)]:                              # not a matrix
        with pytest.raises(ValueError):
            B._gemm_shapes(*bad)


def test_noalloc_shapes_rejected_on_the_host():
    """The allocation-free shifted solve takes bare pointers too: every
    buffer is checked against n and nsys before any device call."""
    from paper_2104_04609_gb300 import binding as B

    torch = pytest.importorskip("torch")
    n, nsys, nnz = 10, 3, 28
    rp = torch.zeros(n + 1, dtype=torch.int32)
    ci = torch.zeros(nnz, dtype=torch.int32)
    mv = torch.zeros(nnz, dtype=torch.float64)
    sv = torch.zeros(nnz, dtype=torch.float64)
    f = torch.zeros(nsys, n, dtype=torch.complex128)
    w = torch.zeros(nsys, n, dtype=torch.complex128)
    al, be = [1.0] * nsys, [0.5] * nsys
    assert B._noalloc_shapes(rp, ci, mv, sv, al, be, f, w) == (nsys, n)
    bad = [
        (rp, ci, mv, sv, al, be, f.reshape(-1), w),                      # f not 2-D
        (rp, ci, mv, sv, al, be, f, w[:, :-1]),                          # w short
        (rp[:-1], ci, mv, sv, al, be, f, w),                             # row_ptr short
        (rp, ci, mv[:-1], sv, al, be, f, w),                             # values differ
        (rp, ci, mv, sv[:-2], al, be, f, w),
        (rp, ci, mv, sv, al[:-1], be, f, w),                             # alpha short
        (rp, ci, mv, sv, al, be + [1.0], f, w),                          # beta long
    ]
    for args in bad:
        with pytest.raises(ValueError):
            B._noalloc_shapes(*args)
        # the public wrapper checks shapes before it looks at devices
        with pytest.raises(ValueError):
            B.osrc_shifted_solve_noalloc(*args)


def test_server_destroy_forgets_request_shapes():
    """Request shapes kept for sizing results are dropped with their server,
    so a later server at the same address starts clean."""
    import ctypes

    from paper_2104_04609_gb300 import binding as B

    class _NoLib:
        def osrc_server_destroy(self, sv):
            return None

    sv = ctypes.c_void_p(0x5678)
    B._REQ_SHAPE[(sv.value, 1)] = (2, 100)
    B._REQ_SHAPE[(0x9999, 1)] = (1, 50)
    saved = B._LIB
    B._LIB = _NoLib()
    try:
        B.osrc_server_destroy(sv)
    finally:
        B._LIB = saved
    assert (sv.value, 1) not in B._REQ_SHAPE and (0x9999, 1) in B._REQ_SHAPE
    del B._REQ_SHAPE[(0x9999, 1)]


def test_server_result_needs_a_submitted_request():
    """The host copy of a server result is sized from the submitted request;
    an id that was never submitted raises before the library is called."""
    import ctypes

    from paper_2104_04609_gb300 import binding as B

    with pytest.raises(ValueError):
        B.osrc_server_result(ctypes.c_void_p(0x1234), 7)
