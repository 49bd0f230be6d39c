"""Thin ctypes binding of the C ABI in include/osrc_pmchwt.h.

Argument marshalling only: every function has the name of the C entry point
it calls, takes numpy arrays for host data and torch CUDA tensors (complex128,
contiguous) for device data, and raises ``OsrcError`` on a non-zero status.
All computation happens in the CUDA library; if the library is missing the
import fails loudly (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libosrc_pmchwt.so")

OSRC_OK = 0
OSRC_INVALID_ARG = 1
OSRC_OUT_OF_MEMORY = 2
OSRC_CUDA_ERROR = 3
OSRC_NOT_CONVERGED = 4
OSRC_BREAKDOWN = 5
OSRC_TIMEOUT = 6
OSRC_UNSUPPORTED = 7

OSRC_FP32_MATFREE = 0
OSRC_FP64_DENSE = 1
OSRC_ASSEMBLE_FP64 = 0
OSRC_ASSEMBLE_FF = 1
OSRC_WEAK = 0
OSRC_STRONG = 1
OSRC_PART_FAR = 1
OSRC_PART_NEAR = 2
OSRC_PART_ALL = 3
OSRC_HOST_BUFFERS = 1
OSRC_PMCHWT = 0
OSRC_MULLER = 1
OSRC_PRECOND_OSRC = 0
OSRC_PRECOND_MASS = 1
OSRC_PRECOND_CALDERON = 2
OSRC_INC_NONE = 0
OSRC_INC_PLANEWAVE = 1
OSRC_INC_POINTSOURCE = 2


class OsrcError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {osrc_status_string(status)} ({status})")


class osrc_params(ctypes.Structure):
    _fields_ = [
        ("k_ext", ctypes.c_double), ("k_int", ctypes.c_double),
        ("rho_ratio", ctypes.c_double), ("n_pade", ctypes.c_int),
        ("theta", ctypes.c_double), ("damping_R", ctypes.c_double),
        ("osrc_side", ctypes.c_int), ("n_ss", ctypes.c_int),
        ("precision", ctypes.c_int), ("inner_tol", ctypes.c_double),
        ("inner_maxit", ctypes.c_int), ("precond", ctypes.c_int),
        ("formulation", ctypes.c_int), ("k_int_im", ctypes.c_double),
        ("dense_assembly", ctypes.c_int),
    ]


class osrc_solve_info(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int), ("converged", ctypes.c_int),
        ("precond_residual", ctypes.c_double), ("true_residual", ctypes.c_double),
        ("ms_total", ctypes.c_double), ("ms_matvec", ctypes.c_double),
        ("ms_precond", ctypes.c_double), ("ms_arnoldi", ctypes.c_double),
        ("inner_iterations_max", ctypes.c_int), ("total_iterations", ctypes.c_int),
        ("ms_queued", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class osrc_batched_info(ctypes.Structure):
    _fields_ = [("refinements", ctypes.c_int), ("inner_iterations", ctypes.c_int),
                ("residual", ctypes.c_double), ("ms_total", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class osrc_request(ctypes.Structure):
    _fields_ = [
        ("verts", ctypes.c_void_p), ("nv", ctypes.c_int32),
        ("tris", ctypes.c_void_p), ("nt", ctypes.c_int32),
        ("params", osrc_params), ("rhs_kind", ctypes.c_int),
        ("src", ctypes.c_void_p), ("nrhs", ctypes.c_int),
        ("tol", ctypes.c_double), ("maxit", ctypes.c_int),
    ]


class osrc_server_stats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
        ("failed", ctypes.c_longlong), ("jobs_started", ctypes.c_longlong),
        ("cache_hits", ctypes.c_longlong), ("cache_misses", ctypes.c_longlong),
        ("evictions", ctypes.c_longlong), ("active_peak", ctypes.c_longlong),
        ("mem_peak", ctypes.c_size_t), ("mem_used", ctypes.c_size_t),
        ("batched_jobs", ctypes.c_longlong),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int32)

# name -> (restype, argtypes)
SIGNATURES = {
    "osrc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "osrc_params_default": (None, [ctypes.POINTER(osrc_params)]),
    "osrc_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_size_t]),
    "osrc_destroy": (None, [_VP]),
    "osrc_mem_used": (ctypes.c_size_t, [_VP]),
    "osrc_mesh_validate": (ctypes.c_int, [_DP, ctypes.c_int32, _IP, ctypes.c_int32]),
    "osrc_mesh_create": (ctypes.c_int, [_VP, _DP, ctypes.c_int32, _IP, ctypes.c_int32,
                                        ctypes.POINTER(_VP)]),
    "osrc_mesh_destroy": (None, [_VP]),
    "osrc_mesh_mean_edge": (ctypes.c_double, [_VP]),
    "osrc_problem_create": (ctypes.c_int, [_VP, ctypes.POINTER(osrc_params),
                                           ctypes.POINTER(_VP), _VP]),
    "osrc_problem_create_objects": (ctypes.c_int, [_VP, ctypes.POINTER(osrc_params), ctypes.c_int,
                                                   _DP, _DP, ctypes.POINTER(_VP), _VP]),
    "osrc_mesh_objects": (ctypes.c_int, [_VP]),
    "osrc_problem_destroy": (None, [_VP]),
    "osrc_problem_nv": (ctypes.c_int, [_VP]),
    "osrc_rhs_planewave": (ctypes.c_int, [_VP, _DP, ctypes.c_int, _VP, _VP]),
    "osrc_rhs_pointsource": (ctypes.c_int, [_VP, _DP, ctypes.c_int, _VP, _VP]),
    "osrc_pmchwt_apply": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, _VP]),
    "osrc_mass_solve": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP]),
    "osrc_precond_apply": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP]),
    "osrc_gmres_solve": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(osrc_solve_info), _VP]),
    "osrc_shifted_solve_noalloc": (ctypes.c_int, [ctypes.c_int, _VP, _VP, _VP, _VP, ctypes.c_int,
                                                  _DP, _DP, _VP, _VP, ctypes.c_double,
                                                  ctypes.c_int, ctypes.c_int,
                                                  ctypes.POINTER(ctypes.c_int), _VP]),
    "osrc_server_create": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(_VP)]),
    "osrc_server_submit": (ctypes.c_int, [_VP, ctypes.POINTER(osrc_request),
                                          ctypes.POINTER(ctypes.c_longlong)]),
    "osrc_server_poll": (ctypes.c_int, [_VP, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(osrc_solve_info)]),
    "osrc_server_wait": (ctypes.c_int, [_VP, ctypes.c_longlong, ctypes.c_double]),
    "osrc_server_result": (ctypes.c_int, [_VP, ctypes.c_longlong, _VP]),
    "osrc_server_get_stats": (ctypes.c_int, [_VP, ctypes.POINTER(osrc_server_stats)]),
    "osrc_server_destroy": (None, [_VP]),
    "osrc_gemm_bf16": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int, _VP,
                                      ctypes.c_int, _VP, ctypes.c_size_t, _VP, _VP]),
    "osrc_gemm_bf16_ws_bytes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_size_t)]),
    "osrc_dense_batched_solve": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_double,
                                                ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                                ctypes.c_double, ctypes.POINTER(osrc_batched_info),
                                                _VP]),
    "osrc_dense_batched_apply": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, _VP]),
    "osrc_dense_batched_apply_ex": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_double, ctypes.c_int,
                                                   ctypes.POINTER(ctypes.c_int), _VP]),
    "osrc_dense_precond_build": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int, _VP]),
    "osrc_dense_precond_drop": (ctypes.c_int, [_VP]),
    "osrc_field_eval": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, _DP, _VP, _VP,
                                       _VP]),
    "osrc_launch_count": (ctypes.c_longlong, [_VP]),
    "osrc_profile_enable": (ctypes.c_int, [_VP, ctypes.c_int]),
    "osrc_far_kernel_stats": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_longlong),
                                             ctypes.POINTER(ctypes.c_double)]),
    "osrc_far_pairs": (ctypes.c_longlong, [_VP]),
    "osrc_near_pairs": (ctypes.c_longlong, [_VP]),
    "osrc_near_nnz": (ctypes.c_longlong, [_VP]),
    "osrc_fp32_peak": (ctypes.c_int, [ctypes.c_int, _DP, _DP, _VP]),
    "osrc_far_kernel_rhs": (ctypes.c_longlong, [_VP]),
}

_LIB = None


def lib():
    """Load the in-tree CUDA library (built by paper_2104_04609_gb300.build)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA library not built: {LIB_PATH} is missing; run "
                "`python -c 'import __graft_entry__ as g; g.build()'` first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(status, where):
    if status != OSRC_OK:
        raise OsrcError(status, where)


def _host_f64(a, shape_last=3):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_DP)


def _host_i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_IP)


def _dev(t):
    """Device pointer of a contiguous complex128 CUDA tensor."""
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128
            and t.is_contiguous()):
        raise TypeError("expected a contiguous complex128 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _need(t, n, what):
    """Raises unless the buffer t (torch tensor or numpy array) holds at least
    n elements: the C ABI takes bare pointers, so a short buffer would be
    read or written past its end on the device."""
    have = int(t.numel()) if hasattr(t, "numel") else int(np.size(t))
    if have < n:
        raise ValueError(f"{what}: buffer holds {have} elements, {n} needed")


def _nv2(pb):
    return 2 * int(lib().osrc_problem_nv(pb))


def _stream(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------
def osrc_status_string(status):
    return lib().osrc_status_string(int(status)).decode()


def osrc_params_default(**overrides):
    p = osrc_params()
    lib().osrc_params_default(ctypes.byref(p))
    names = {f[0] for f in osrc_params._fields_}
    for k, v in overrides.items():
        if k not in names:  # ctypes would accept any attribute name silently
            raise TypeError(f"unknown osrc_params field {k!r}")
        setattr(p, k, v)
    return p


def osrc_create(device=0, mem_budget_bytes=0):
    h = _VP()
    _check(lib().osrc_create(ctypes.byref(h), int(device), int(mem_budget_bytes)), "osrc_create")
    return h


def osrc_destroy(ctx):
    lib().osrc_destroy(ctx)


def osrc_mem_used(ctx):
    return lib().osrc_mem_used(ctx)


def osrc_mesh_validate(verts, tris):
    v, vp = _host_f64(verts)
    t, tp = _host_i32(tris)
    return lib().osrc_mesh_validate(vp, v.shape[0] if v.ndim == 2 else 0, tp,
                                    t.shape[0] if t.ndim == 2 else 0)


def osrc_mesh_create(ctx, verts, tris):
    v, vp = _host_f64(verts)
    t, tp = _host_i32(tris)
    h = _VP()
    _check(lib().osrc_mesh_create(ctx, vp, v.shape[0], tp, t.shape[0], ctypes.byref(h)),
           "osrc_mesh_create")
    return h


def osrc_mesh_destroy(mesh):
    lib().osrc_mesh_destroy(mesh)


def osrc_mesh_mean_edge(mesh):
    return lib().osrc_mesh_mean_edge(mesh)


def osrc_problem_create(mesh, params, stream=None):
    h = _VP()
    _check(lib().osrc_problem_create(mesh, ctypes.byref(params), ctypes.byref(h), _stream(stream)),
           "osrc_problem_create")
    return h


def osrc_problem_create_objects(mesh, params, k_int, rho_ratio, stream=None):
    """Problem on a mesh of disjoint objects, object m with k_int[m], rho_ratio[m]."""
    k = np.ascontiguousarray(k_int, dtype=np.float64)
    r = np.ascontiguousarray(rho_ratio, dtype=np.float64)
    h = _VP()
    _check(lib().osrc_problem_create_objects(mesh, ctypes.byref(params), len(k), k.ctypes.data_as(_DP),
                                             r.ctypes.data_as(_DP), ctypes.byref(h), _stream(stream)),
           "osrc_problem_create_objects")
    return h


def osrc_mesh_objects(mesh):
    return lib().osrc_mesh_objects(mesh)


def osrc_problem_destroy(pb):
    lib().osrc_problem_destroy(pb)


def osrc_problem_nv(pb):
    return lib().osrc_problem_nv(pb)


def osrc_rhs_planewave(pb, dirs, b, stream=None):
    d, dp = _host_f64(np.atleast_2d(dirs))
    _need(b, d.shape[0] * _nv2(pb), "osrc_rhs_planewave b")
    _check(lib().osrc_rhs_planewave(pb, dp, d.shape[0], _dev(b), _stream(stream)),
           "osrc_rhs_planewave")


def osrc_rhs_pointsource(pb, srcs, b, stream=None):
    d, dp = _host_f64(np.atleast_2d(srcs))
    _need(b, d.shape[0] * _nv2(pb), "osrc_rhs_pointsource b")
    _check(lib().osrc_rhs_pointsource(pb, dp, d.shape[0], _dev(b), _stream(stream)),
           "osrc_rhs_pointsource")


def osrc_pmchwt_apply(pb, x, y, nrhs=1, form=OSRC_WEAK, part=OSRC_PART_ALL, stream=None):
    _need(x, int(nrhs) * _nv2(pb), "osrc_pmchwt_apply x")
    _need(y, int(nrhs) * _nv2(pb), "osrc_pmchwt_apply y")
    _check(lib().osrc_pmchwt_apply(pb, _dev(x), _dev(y), int(nrhs), int(form), int(part),
                                   _stream(stream)), "osrc_pmchwt_apply")


def osrc_mass_solve(pb, x, y, nrhs=1, stream=None):
    _need(x, int(nrhs) * _nv2(pb), "osrc_mass_solve x")
    _need(y, int(nrhs) * _nv2(pb), "osrc_mass_solve y")
    _check(lib().osrc_mass_solve(pb, _dev(x), _dev(y), int(nrhs), _stream(stream)),
           "osrc_mass_solve")


def osrc_precond_apply(pb, x, y, nrhs=1, stream=None):
    _need(x, int(nrhs) * _nv2(pb), "osrc_precond_apply x")
    _need(y, int(nrhs) * _nv2(pb), "osrc_precond_apply y")
    _check(lib().osrc_precond_apply(pb, _dev(x), _dev(y), int(nrhs), _stream(stream)),
           "osrc_precond_apply")


def osrc_gmres_solve(pb, b, x, nrhs=1, tol=1e-5, maxit=500, host_buffers=False,
                     stream=None, raise_on_nonconvergence=True):
    """Returns the osrc_solve_info record.  With host_buffers, b and x are
    numpy complex128 arrays (C-contiguous), else CUDA tensors."""
    info = osrc_solve_info()
    _need(b, int(nrhs) * _nv2(pb), "osrc_gmres_solve b")
    _need(x, int(nrhs) * _nv2(pb), "osrc_gmres_solve x")
    if host_buffers:
        if not (isinstance(b, np.ndarray) and isinstance(x, np.ndarray)
                and b.dtype == np.complex128 and x.dtype == np.complex128
                and b.flags.c_contiguous and x.flags.c_contiguous):
            raise TypeError("host buffers must be C-contiguous complex128 numpy arrays")
        bp, xp = ctypes.c_void_p(b.ctypes.data), ctypes.c_void_p(x.ctypes.data)
        flags = OSRC_HOST_BUFFERS
    else:
        bp, xp = _dev(b), _dev(x)
        flags = 0
    s = lib().osrc_gmres_solve(pb, bp, xp, int(nrhs), float(tol), int(maxit), flags,
                               ctypes.byref(info), _stream(stream))
    if s != OSRC_OK and (s != OSRC_NOT_CONVERGED or raise_on_nonconvergence):
        raise OsrcError(s, "osrc_gmres_solve")
    return info


def _noalloc_shapes(row_ptr, col_idx, M_vals, S_vals, alpha, beta, f, w):
    """Shape checks of osrc_shifted_solve_noalloc, before any device call:
    the C side takes bare pointers, so every buffer must hold what the n rows
    and nsys systems imply (else ValueError).  Returns (nsys, n)."""
    if len(getattr(f, "shape", ())) != 2:
        raise ValueError("f must be a 2-D (nsys, n) array")
    nsys, n = int(f.shape[0]), int(f.shape[1])
    if tuple(getattr(w, "shape", ())) != (nsys, n):
        raise ValueError(f"w must have the shape of f, ({nsys}, {n})")
    _need(row_ptr, n + 1, "osrc_shifted_solve_noalloc row_ptr")
    nnz = [int(t.numel()) if hasattr(t, "numel") else int(np.size(t)) for t in (col_idx, M_vals, S_vals)]
    if len(set(nnz)) != 1:
        raise ValueError(f"col_idx, M_vals and S_vals must have one length, got {nnz}")
    if len(np.atleast_1d(alpha)) != nsys or len(np.atleast_1d(beta)) != nsys:
        raise ValueError(f"alpha and beta must hold nsys = {nsys} values each")
    return nsys, n


def osrc_shifted_solve_noalloc(row_ptr, col_idx, M_vals, S_vals, alpha, beta, f, w,
                               tol=1e-10, maxit=2000, conj=0, stream=None):
    """Allocation-free batched solve of (alpha_s M + beta_s S) w_s = f_s.

    For callers that cannot allocate device memory at solve time (stream
    capture, allocation-free hosts, pool-owned memory): the library uses a
    static 10 MiB device workspace instead of cudaMalloc.  row_ptr, col_idx
    (int32) and M_vals, S_vals (float64) are CUDA tensors of one CSR pattern;
    f, w are (nsys, n) complex128 CUDA tensors; alpha, beta are sequences of
    nsys complex numbers.  Returns the per-system iteration counts."""
    import torch

    nsys, n = _noalloc_shapes(row_ptr, col_idx, M_vals, S_vals, alpha, beta, f, w)
    for t, dt in ((row_ptr, torch.int32), (col_idx, torch.int32), (M_vals, torch.float64),
                  (S_vals, torch.float64)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise TypeError("CSR arrays must be contiguous CUDA tensors (int32 / float64)")
    a = np.ascontiguousarray(np.asarray(alpha, dtype=np.complex128).reshape(-1).view(np.float64))
    b = np.ascontiguousarray(np.asarray(beta, dtype=np.complex128).reshape(-1).view(np.float64))
    it = (ctypes.c_int * nsys)()
    s = lib().osrc_shifted_solve_noalloc(
        n, ctypes.c_void_p(row_ptr.data_ptr()), ctypes.c_void_p(col_idx.data_ptr()),
        ctypes.c_void_p(M_vals.data_ptr()), ctypes.c_void_p(S_vals.data_ptr()), nsys,
        a.ctypes.data_as(_DP), b.ctypes.data_as(_DP), _dev(f), _dev(w), float(tol),
        int(maxit), int(conj), it, _stream(stream))
    _check(s, "osrc_shifted_solve_noalloc")
    return list(it)


def osrc_server_create(ctx, max_active=4):
    h = _VP()
    _check(lib().osrc_server_create(ctx, int(max_active), ctypes.byref(h)), "osrc_server_create")
    return h


def osrc_server_submit(sv, verts, tris, params, src, rhs_kind=0, tol=1e-5, maxit=500):
    """Queues a request; returns its id.  verts (nv, 3), tris (nt, 3), src
    (nrhs, 3) host arrays; params an osrc_params."""
    v, _ = _host_f64(verts)
    t, _ = _host_i32(tris)
    s = np.ascontiguousarray(np.atleast_2d(src), dtype=np.float64)
    rq = osrc_request(v.ctypes.data, v.shape[0], t.ctypes.data, t.shape[0], params,
                      int(rhs_kind), s.ctypes.data, s.shape[0], float(tol), int(maxit))
    rid = ctypes.c_longlong()
    _check(lib().osrc_server_submit(sv, ctypes.byref(rq), ctypes.byref(rid)), "osrc_server_submit")
    _REQ_SHAPE[(sv.value, rid.value)] = (s.shape[0], v.shape[0])
    return rid.value


# (server, request id) -> (right-hand sides, vertices) of each submitted
# request, so that osrc_server_result sizes the host copy from the request
_REQ_SHAPE = {}


def osrc_server_poll(sv, rid):
    """Returns (done, status, latency_ms, info dict or None)."""
    done = ctypes.c_int()
    lat = ctypes.c_double()
    info = osrc_solve_info()
    s = lib().osrc_server_poll(sv, int(rid), ctypes.byref(done), ctypes.byref(lat), ctypes.byref(info))
    if done.value:
        return True, s, lat.value, info.as_dict()
    if s != OSRC_OK:
        raise OsrcError(s, "osrc_server_poll")
    return False, s, None, None


def osrc_server_wait(sv, rid, timeout_s=600.0):
    return lib().osrc_server_wait(sv, int(rid), float(timeout_s))


def osrc_server_result(sv, rid, nrhs=None, nv=None):
    """(status, solution (nrhs, 2nv)); the sizes come from the submitted
    request (nrhs, nv, when given, must match it)."""
    key = (sv.value, int(rid))
    shape = _REQ_SHAPE.get(key)
    if shape is None:
        raise ValueError(f"request {rid} was not submitted through this binding")
    if (nrhs is not None and int(nrhs) != shape[0]) or (nv is not None and int(nv) != shape[1]):
        raise ValueError(f"request {rid} has {shape[0]} right-hand sides on {shape[1]} vertices")
    x = np.zeros((shape[0], 2 * shape[1]), dtype=np.complex128)
    s = lib().osrc_server_result(sv, int(rid), ctypes.c_void_p(x.ctypes.data))
    if s != OSRC_TIMEOUT:  # the library released the request
        _REQ_SHAPE.pop(key, None)
    return s, x


def osrc_server_get_stats(sv):
    st = osrc_server_stats()
    _check(lib().osrc_server_get_stats(sv, ctypes.byref(st)), "osrc_server_get_stats")
    return st.as_dict()


def osrc_server_destroy(sv):
    lib().osrc_server_destroy(sv)
    for key in [k for k in _REQ_SHAPE if k[0] == sv.value]:
        del _REQ_SHAPE[key]


def osrc_gemm_bf16_ws_bytes(M, N, K):
    """Workspace bytes the tensor-core GEMM needs for this shape on the current device."""
    out = ctypes.c_size_t(0)
    _check(lib().osrc_gemm_bf16_ws_bytes(int(M), int(N), int(K), ctypes.byref(out)), "osrc_gemm_bf16_ws_bytes")
    return int(out.value)


def _gemm_shapes(A, B, C, err):
    """(M, K, N) of C = A B^T, checked before any device call: the C ABI
    takes bare pointers and sizes, so B must have A's K columns, C must have
    M rows and at least N columns, and err one element."""
    if A.dim() != 2 or B.dim() != 2 or C.dim() != 2:
        raise ValueError("osrc_gemm_bf16: A, B and C must be matrices")
    M, K = (int(v) for v in A.shape)
    N = int(B.shape[0])
    if int(B.shape[1]) != K:
        raise ValueError(f"osrc_gemm_bf16: B has {int(B.shape[1])} columns, A has {K}")
    if int(C.shape[0]) != M or int(C.shape[1]) < N:
        raise ValueError(f"osrc_gemm_bf16: C is {tuple(C.shape)}, ({M}, >= {N}) needed")
    _need(err, 1, "osrc_gemm_bf16 err")
    return M, K, N


def osrc_gemm_bf16(A, B, C, err, ws=None, stream=None):
    """C = A B^T on the tensor cores; A (M, K), B (N, K) bfloat16 CUDA tensors,
    C (M, ldc) float32, err a one-element int32 CUDA tensor (set to 1 if the
    kernel's bounded waits gave up).  ws: CUDA tensor of at least
    osrc_gemm_bf16_ws_bytes(M, N, K) bytes for the pieces of split tiles (one
    is allocated per call when None)."""
    import torch

    M, K, N = _gemm_shapes(A, B, C, err)
    assert A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16 and C.dtype == torch.float32
    assert A.is_cuda and B.is_cuda and C.is_cuda and err.is_cuda and err.dtype == torch.int32
    assert A.is_contiguous() and B.is_contiguous() and C.is_contiguous()
    if ws is None:
        nb = osrc_gemm_bf16_ws_bytes(M, N, K) if M % 128 == 0 and K % 64 == 0 and 16 <= N <= 256 \
            and N % 16 == 0 else 0
        ws = torch.empty(max(nb, 16), dtype=torch.uint8, device=A.device)
    assert ws.is_cuda and ws.is_contiguous()
    _check(lib().osrc_gemm_bf16(ctypes.c_void_p(A.data_ptr()), M, K, ctypes.c_void_p(B.data_ptr()), N,
                                ctypes.c_void_p(C.data_ptr()), C.shape[1],
                                ctypes.c_void_p(ws.data_ptr()), ws.numel() * ws.element_size(),
                                ctypes.c_void_p(err.data_ptr()), _stream(stream)), "osrc_gemm_bf16")


def osrc_dense_batched_solve(pb, b, x, tol=1e-6, max_refine=8, inner_tol=1e-3, inner_maxit=200,
                             precond_tol=0.0, stream=None, raise_on_nonconvergence=True):
    """Batched mixed-precision solve; b, x (nrhs, 2nv) complex128 CUDA tensors.
    Returns the osrc_batched_info record as a dict."""
    info = osrc_batched_info()
    _need(b, int(b.shape[0]) * _nv2(pb), "osrc_dense_batched_solve b")
    _need(x, int(b.shape[0]) * _nv2(pb), "osrc_dense_batched_solve x")
    s = lib().osrc_dense_batched_solve(pb, _dev(b), _dev(x), int(b.shape[0]), float(tol),
                                       int(max_refine), float(inner_tol), int(inner_maxit),
                                       float(precond_tol), ctypes.byref(info), _stream(stream))
    if s != OSRC_OK and (s != OSRC_NOT_CONVERGED or raise_on_nonconvergence):
        raise OsrcError(s, "osrc_dense_batched_solve")
    return info.as_dict()


def osrc_dense_batched_apply(pb, x, y, what, stream=None):
    _need(x, int(x.shape[0]) * _nv2(pb), "osrc_dense_batched_apply x")
    _need(y, int(x.shape[0]) * _nv2(pb), "osrc_dense_batched_apply y")
    _check(lib().osrc_dense_batched_apply(pb, _dev(x), _dev(y), int(x.shape[0]), int(what),
                                          _stream(stream)), "osrc_dense_batched_apply")


def osrc_dense_batched_apply_ex(pb, x, y, what, ptol, pmaxit, stream=None):
    """As osrc_dense_batched_apply with the preconditioner's inner tolerance and
    cap given; returns the largest inner iteration count."""
    k = ctypes.c_int(0)
    _need(x, int(x.shape[0]) * _nv2(pb), "osrc_dense_batched_apply_ex x")
    _need(y, int(x.shape[0]) * _nv2(pb), "osrc_dense_batched_apply_ex y")
    _check(lib().osrc_dense_batched_apply_ex(pb, _dev(x), _dev(y), int(x.shape[0]), int(what),
                                             float(ptol), int(pmaxit), ctypes.byref(k),
                                             _stream(stream)), "osrc_dense_batched_apply_ex")
    return k.value


def osrc_dense_precond_build(pb, tol=1e-3, maxit=500, stream=None):
    """Store P M^-1 as an explicit BF16 matrix for the batched dense solve."""
    _check(lib().osrc_dense_precond_build(pb, float(tol), int(maxit), _stream(stream)),
           "osrc_dense_precond_build")


def osrc_dense_precond_drop(pb):
    _check(lib().osrc_dense_precond_drop(pb), "osrc_dense_precond_drop")


def osrc_field_eval(pb, x, pts, u, inc_kind=OSRC_INC_NONE, inc_param=None, region=None,
                    stream=None):
    """Total field at points off the surface; x (2nv,) complex128, pts (n, 3)
    float64, u (n,) complex128, region (n,) int32 or None: CUDA tensors."""
    import torch

    if not (pts.dtype == torch.float64 and pts.is_cuda and pts.is_contiguous() and pts.dim() == 2
            and pts.shape[1] == 3):
        raise TypeError("pts: expected a contiguous (n, 3) float64 CUDA tensor")
    n = int(pts.shape[0])
    _need(x, _nv2(pb), "osrc_field_eval x")
    _need(u, n, "osrc_field_eval u")
    if region is not None:
        if not (region.dtype == torch.int32 and region.is_cuda and region.is_contiguous()):
            raise TypeError("region: expected a contiguous int32 CUDA tensor")
        _need(region, n, "osrc_field_eval region")
    par = None
    if inc_kind != OSRC_INC_NONE:
        par = np.ascontiguousarray(inc_param, dtype=np.float64).reshape(3)
    _check(lib().osrc_field_eval(pb, _dev(x), ctypes.c_void_p(pts.data_ptr()), n, int(inc_kind),
                                 None if par is None else par.ctypes.data_as(_DP), _dev(u),
                                 None if region is None else ctypes.c_void_p(region.data_ptr()),
                                 _stream(stream)), "osrc_field_eval")


def osrc_launch_count(pb):
    return lib().osrc_launch_count(pb)


def osrc_profile_enable(pb, on=True):
    _check(lib().osrc_profile_enable(pb, 1 if on else 0), "osrc_profile_enable")


def osrc_far_kernel_stats(pb):
    n = ctypes.c_longlong()
    ms = ctypes.c_double()
    _check(lib().osrc_far_kernel_stats(pb, ctypes.byref(n), ctypes.byref(ms)),
           "osrc_far_kernel_stats")
    return n.value, ms.value


def osrc_far_kernel_rhs(pb):
    return lib().osrc_far_kernel_rhs(pb)


def osrc_far_pairs(pb):
    return lib().osrc_far_pairs(pb)


def osrc_near_pairs(pb):
    return lib().osrc_near_pairs(pb)


def osrc_near_nnz(pb):
    return lib().osrc_near_nnz(pb)


def osrc_fp32_peak(reps=5, stream=None):
    """Measured FP32 throughput of the current GPU: (scalar FFMA TFLOP/s,
    packed FP32x2 FMA TFLOP/s)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().osrc_fp32_peak(int(reps), ctypes.byref(a), ctypes.byref(b), _stream(stream)),
           "osrc_fp32_peak")
    return a.value, b.value


# ---------------------------------------------------------------------------
# convenience owner of the three handles
# ---------------------------------------------------------------------------
class Solver:
    """Context + mesh + problem for one transmission problem, with device
    tensors in and out.  Parameters are those of ``osrc_params``."""

    def __init__(self, verts, tris, k_ext, k_int, rho_ratio, device=0, mem_budget_bytes=0,
                 objects=None, **params):
        """objects = (k_int list, rho_ratio list): one material per object
        (connected component) of the mesh; k_int and rho_ratio are then unused."""
        import torch

        kk = float(k_int) if objects is None else float(objects[0][0])
        rr = float(rho_ratio) if objects is None else float(objects[1][0])
        p = osrc_params_default(k_ext=float(k_ext), k_int=kk, rho_ratio=rr, **params)
        self.params = p
        self.device = torch.device("cuda", device)
        self.ctx = osrc_create(device, mem_budget_bytes)
        self.mesh = None
        self.pb = None
        try:
            self.mesh = osrc_mesh_create(self.ctx, verts, tris)
            if objects is None:
                self.pb = osrc_problem_create(self.mesh, p)
            else:
                self.pb = osrc_problem_create_objects(self.mesh, p, objects[0], objects[1])
        except Exception:
            self.close()
            raise
        self.nv = osrc_problem_nv(self.pb)

    def zeros(self, nrhs=1):
        import torch

        return torch.zeros((nrhs, 2 * self.nv), dtype=torch.complex128, device=self.device)

    def rhs_planewave(self, dirs):
        dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
        b = self.zeros(dirs.shape[0])
        osrc_rhs_planewave(self.pb, dirs, b)
        return b

    def rhs_pointsource(self, srcs):
        srcs = np.atleast_2d(np.asarray(srcs, dtype=np.float64))
        b = self.zeros(srcs.shape[0])
        osrc_rhs_pointsource(self.pb, srcs, b)
        return b

    def apply(self, x, form=OSRC_WEAK, part=OSRC_PART_ALL):
        x = x.contiguous()
        y = torch_empty_like(x)
        osrc_pmchwt_apply(self.pb, x, y, x.shape[0] if x.ndim == 2 else 1, form, part)
        return y

    def mass_solve(self, x):
        x = x.contiguous()
        y = torch_empty_like(x)
        osrc_mass_solve(self.pb, x, y, x.shape[0] if x.ndim == 2 else 1)
        return y

    def precond(self, x):
        x = x.contiguous()
        y = torch_empty_like(x)
        osrc_precond_apply(self.pb, x, y, x.shape[0] if x.ndim == 2 else 1)
        return y

    def solve(self, b, tol=1e-5, maxit=500, raise_on_nonconvergence=True):
        b = b.contiguous()
        x = torch_empty_like(b)
        info = osrc_gmres_solve(self.pb, b, x, b.shape[0] if b.ndim == 2 else 1, tol, maxit,
                                raise_on_nonconvergence=raise_on_nonconvergence)
        return x, info

    def field(self, x, pts, inc_kind=OSRC_INC_NONE, inc_param=None):
        """(u, region) at points pts ((n, 3) float64 CUDA tensor) for one
        solution x ((2nv,) or (1, 2nv) complex128 CUDA tensor)."""
        import torch

        x = x.reshape(-1).contiguous()
        pts = pts.contiguous()
        u = torch.empty(pts.shape[0], dtype=torch.complex128, device=pts.device)
        reg = torch.empty(pts.shape[0], dtype=torch.int32, device=pts.device)
        osrc_field_eval(self.pb, x, pts, u, inc_kind, inc_param, reg)
        return u, reg

    def launches(self):
        return osrc_launch_count(self.pb)

    def close(self):
        if self.pb is not None:
            osrc_problem_destroy(self.pb)
            self.pb = None
        if self.mesh is not None:
            osrc_mesh_destroy(self.mesh)
            self.mesh = None
        if self.ctx is not None:
            osrc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def torch_empty_like(x):
    import torch

    return torch.empty_like(x)
