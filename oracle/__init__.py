"""Plain FP64 CPU oracle for the OSRC-preconditioned PMCHWT hot path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.  It
shares no code with the CUDA library: the boundary integrals are evaluated by
the C file ``oracle.c`` (compiled with gcc), the linear algebra here uses
numpy/scipy library primitives (dense solve, sparse LU) as single steps.

Paper: van 't Wout et al., "Frequency-robust preconditioning of boundary
integral equations for acoustic transmission", JCP 2022 (arXiv 2104.04609).

Functions and the passages they follow:
  assemble()          Galerkin V, K, T, D at one wavenumber (Sec. 2.2, 2.3)
  pmchwt_matrix()     permuted PMCHWT block system (Sec. 2.7)
  mass_stiffness()    P1 mass M and Laplace-Beltrami stiffness S (Sec. 2.6)
  rhs()               [<gamma_D u_inc, phi_i>; <gamma_N u_inc, phi_i>] (Sec. 2.7)
  pade()              rotated-branch Pade coefficients of sqrt(1+z) (Sec. 2.6)
  damped_wavenumber() k_eps = k (1 + 0.4 i (k R)^(-2/3)) (Sec. 2.6)
  osrc_apply()        strong-form OSRC DtN / NtD maps (Sec. 2.6, 2.7)
  gmres()             GMRES without restart, x0 = 0, preconditioned residual
                      (Sec. 3.1)
  potentials()        single- and double-layer potentials off the surface
                      (Sec. 2.2, representation formulas)
  field()             total field outside / inside from a PMCHWT solution
                      (Sec. 2.2, with the transmission conditions of Sec. 2.1)
  pmchwt_matrix_objects(), field_objects()
                      the same for disjoint objects with their own materials
                      (Sec. 2.2, multiple scattering)

Readings where the paper is silent or ambiguous:
quadrature orders (6-point rule for separated pairs, Sauter-Schwab with n
Gauss points per dimension for touching ones); the Pade coefficients and the
NtD form; the damping length R; the strong form of the preconditioned system.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

__all__ = [
    "lib", "quad6", "gauss_legendre", "ss_rule", "pair_matrices", "assemble",
    "assemble_rows", "pmchwt_matrix", "pmchwt_rows", "mass_stiffness", "rhs",
    "pade", "pade_eval", "ntd_partial_fractions", "damped_wavenumber",
    "mean_edge_length", "osrc_apply", "strong_apply", "gmres", "Problem", "potentials", "field",
    "components", "pmchwt_matrix_objects", "field_objects",
]

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.orc_quad6.argtypes = [dp, dp]
        L.orc_gauss_legendre.argtypes = [ctypes.c_int, dp, dp]
        L.orc_ss_rule.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int]
        L.orc_pair_matrices.argtypes = [dp, ip, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, dp]
        L.orc_assemble.argtypes = [dp, ctypes.c_int, ip, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int, ctypes.c_int, dp]
        L.orc_assemble_rows.argtypes = [dp, ctypes.c_int, ip, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int, ip,
                                        ctypes.c_int, dp]
        L.orc_mass_stiffness_coo.argtypes = [dp, ip, ctypes.c_int, ip, ip, dp, dp]
        L.orc_rhs.argtypes = [dp, ctypes.c_int, ip, ctypes.c_int, ctypes.c_double,
                              ctypes.c_double, ctypes.c_int, dp, dp]
        L.orc_potentials.argtypes = [dp, ctypes.c_int, ip, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, dp, dp, dp, ctypes.c_int, dp, dp]
        L.orc_num_threads.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _mesh(verts, tris):
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    return v, t


# --------------------------------------------------------------------------
# quadrature (exposed for the tests that pin it)
# --------------------------------------------------------------------------
def quad6():
    """6-point degree-4 rule: barycentric points (6, 3), weights summing to 1."""
    b = np.zeros(18)
    w = np.zeros(6)
    lib().orc_quad6(_dp(b), _dp(w))
    return b.reshape(6, 3), w


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().orc_gauss_legendre(n, _dp(x), _dp(w))
    return x, w


def ss_rule(kase, n):
    """Sauter-Schwab point set on That x That, That = {0 <= x2 <= x1 <= 1}:
    returns (pts (N, 4) = (x1, x2, y1, y2), weights (N,)).  kase 3 identical,
    2 common edge (x2 = y2 = 0), 1 common vertex (origin)."""
    cap = 6 * n ** 4
    out = np.zeros(4 * cap)
    w = np.zeros(cap)
    N = lib().orc_ss_rule(kase, n, _dp(out), _dp(w), cap)
    if N < 0:
        raise ValueError("bad Sauter-Schwab request")
    return out[: 4 * N].reshape(N, 4), w[:N]


def pair_matrices(verts, tris, t, s, k, nss=6):
    """Local 3x3 Galerkin matrices (V, K, T, D) of triangle pair (t, s)."""
    v, tr = _mesh(verts, tris)
    out = np.zeros(2 * 36)
    kase = lib().orc_pair_matrices(_dp(v), _ip(tr), int(t), int(s),
                                   float(np.real(k)), float(np.imag(k)), nss, _dp(out))
    m = out.view(np.complex128).reshape(4, 3, 3)
    return kase, m[0], m[1], m[2], m[3]


# --------------------------------------------------------------------------
# boundary operators (Sec. 2.2) on P1 x P1 (Sec. 2.3)
# --------------------------------------------------------------------------
def assemble(verts, tris, k, nss=6, part=3):
    """Dense Galerkin matrices V, K, T, D at wavenumber k.  part: 1 = pairs
    sharing no vertex (6x6 rule), 2 = touching pairs (Sauter-Schwab), 3 = all."""
    v, t = _mesh(verts, tris)
    nv = v.shape[0]
    out = np.zeros(2 * 4 * nv * nv)
    rc = lib().orc_assemble(_dp(v), nv, _ip(t), t.shape[0], float(np.real(k)),
                            float(np.imag(k)), nss, part, _dp(out))
    if rc != 0:
        raise RuntimeError(f"orc_assemble failed: {rc}")
    m = out.view(np.complex128).reshape(4, nv, nv)
    return m[0], m[1], m[2], m[3]


def assemble_rows(verts, tris, k, rows, nss=6, part=3):
    """Rows ``rows`` of V, K, T, D: arrays (len(rows), n_v) each."""
    v, t = _mesh(verts, tris)
    nv = v.shape[0]
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    out = np.zeros(2 * 4 * nv * len(rows))
    rc = lib().orc_assemble_rows(_dp(v), nv, _ip(t), t.shape[0], float(np.real(k)),
                                 float(np.imag(k)), nss, part, _ip(rows), len(rows),
                                 _dp(out))
    if rc != 0:
        raise RuntimeError(f"orc_assemble_rows failed: {rc}")
    m = out.view(np.complex128).reshape(len(rows), 4, nv)
    return m[:, 0], m[:, 1], m[:, 2], m[:, 3]


def pmchwt_matrix(verts, tris, k_ext, k_int, rho_ratio, nss=6, part=3, formulation="pmchwt"):
    """Permuted PMCHWT matrix of Sec. 2.7 acting on [psi; phi]:
        [[V0 + rho V1, -K0 - K1], [T0 + T1, D0 + D1 / rho]],  rho = rho_int/rho_ext.
    formulation "muller": the difference of the exterior and interior
    Calderon equations plus the identity (Sec. 2.2, Mueller), in the same
    ordering:  [[V0 - rho V1, -K0 + K1 + M], [T0 - T1 + M, D0 - D1 / rho]]
    (M the P1 mass matrix; part 2 carries it, as the touching pairs do)."""
    V0, K0, T0, D0 = assemble(verts, tris, k_ext, nss, part)
    V1, K1, T1, D1 = assemble(verts, tris, k_int, nss, part)
    if formulation == "muller":
        Md = mass_stiffness(verts, tris)[0].toarray() if part & 2 else 0.0
        return np.block([[V0 - rho_ratio * V1, -K0 + K1 + Md],
                         [T0 - T1 + Md, D0 - D1 / rho_ratio]])
    return np.block([[V0 + rho_ratio * V1, -K0 - K1],
                     [T0 + T1, D0 + D1 / rho_ratio]])


def components(tris):
    """Objects of a mesh of disjoint closed surfaces: the connected components
    of the triangle-adjacency graph (triangles sharing a vertex), numbered in
    the order of their first triangle.  Returns (per-triangle ids,
    per-vertex ids)."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    t = np.asarray(tris, dtype=np.int64)
    nv = int(t.max()) + 1
    rows = np.repeat(t[:, 0], 2)
    cols = t[:, 1:].ravel()
    G = sp.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(nv, nv))
    _, lab = connected_components(G, directed=False)
    # renumber by first triangle
    order, seen = {}, []
    for c in lab[t[:, 0]]:
        if c not in order:
            order[c] = len(order)
    vcomp = np.array([order[c] for c in lab])
    return vcomp[t[:, 0]], vcomp


def pmchwt_matrix_objects(verts, tris, k_ext, k_int, rho_ratio, nss=6, part=3, formulation="pmchwt"):
    """Permuted PMCHWT matrix of disjoint objects (Sec. 2.2, multiple
    scattering): object m has its own k_int[m] and rho_ratio[m]; the interior
    operators act within each object only (diagonal blocks A_0,mm + A^_m),
    the exterior ones between all surfaces (cross blocks A_0,mn):
        [[V0 + sum_m rho_m V_m|mm, -K0 - sum_m K_m|mm],
         [T0 + sum_m T_m|mm,        D0 + sum_m D_m|mm / rho_m]]."""
    _, vc = components(tris)
    sg = -1.0 if formulation == "muller" else 1.0
    V, K, T, D = (a.copy() for a in assemble(verts, tris, k_ext, nss, part))
    for m in range(vc.max() + 1):
        sel = np.outer(vc == m, vc == m)
        Vm, Km, Tm, Dm = assemble(verts, tris, k_int[m], nss, part)
        V = V + sg * rho_ratio[m] * np.where(sel, Vm, 0)
        K = K + sg * np.where(sel, Km, 0)
        T = T + sg * np.where(sel, Tm, 0)
        D = D + sg * np.where(sel, Dm, 0) / rho_ratio[m]
    if formulation == "muller" and part & 2:
        Md = mass_stiffness(verts, tris)[0].toarray()
        return np.block([[V, -K + Md], [T + Md, D]])
    return np.block([[V, -K], [T, D]])


def pmchwt_rows(verts, tris, k_ext, k_int, rho_ratio, rows, nss=6, part=3):
    """Rows of the permuted PMCHWT matrix: for test vertex i in ``rows`` the
    returned arrays R1, R2 (len(rows), 2 n_v) are rows i and n_v + i."""
    V0, K0, T0, D0 = assemble_rows(verts, tris, k_ext, rows, nss, part)
    V1, K1, T1, D1 = assemble_rows(verts, tris, k_int, rows, nss, part)
    R1 = np.concatenate([V0 + rho_ratio * V1, -K0 - K1], axis=1)
    R2 = np.concatenate([T0 + T1, D0 + D1 / rho_ratio], axis=1)
    return R1, R2


def mass_stiffness(verts, tris):
    """Sparse (CSR) P1 mass M and Laplace-Beltrami stiffness S."""
    import scipy.sparse as sp

    v, t = _mesh(verts, tris)
    nt = t.shape[0]
    ri = np.zeros(9 * nt, dtype=np.int32)
    ci = np.zeros(9 * nt, dtype=np.int32)
    mv = np.zeros(9 * nt)
    sv = np.zeros(9 * nt)
    lib().orc_mass_stiffness_coo(_dp(v), _ip(t), nt, _ip(ri), _ip(ci), _dp(mv), _dp(sv))
    nv = v.shape[0]
    M = sp.coo_matrix((mv, (ri, ci)), shape=(nv, nv)).tocsr()
    S = sp.coo_matrix((sv, (ri, ci)), shape=(nv, nv)).tocsr()
    return M, S


def rhs(verts, tris, k_ext, kind="planewave", src=(0.0, 0.0, 1.0)):
    """[<u_inc, phi_i>; <du_inc/dn, phi_i>] (6-point rule), complex (2 n_v,)."""
    v, t = _mesh(verts, tris)
    s = np.ascontiguousarray(src, dtype=np.float64)
    out = np.zeros(4 * v.shape[0])
    lib().orc_rhs(_dp(v), v.shape[0], _ip(t), t.shape[0], float(np.real(k_ext)),
                  float(np.imag(k_ext)), 0 if kind == "planewave" else 1, _dp(s), _dp(out))
    return out.view(np.complex128).copy()


def potentials(verts, tris, k, psi, phi, pts):
    """(SLP psi, DLP phi) at points off the surface, 6-point rule per triangle:
    SLP psi(x) = int G(x, y) psi(y) dy, DLP phi(x) = int dG/dn_y phi(y) dy with
    G = exp(ikr)/(4 pi r) (Sec. 2.2); psi, phi P1 coefficients (n_v,)."""
    v, t = _mesh(verts, tris)
    P = np.ascontiguousarray(np.atleast_2d(pts), dtype=np.float64)
    ps = np.ascontiguousarray(psi, dtype=np.complex128)
    ph = np.ascontiguousarray(phi, dtype=np.complex128)
    n = P.shape[0]
    S = np.zeros(2 * n)
    D = np.zeros(2 * n)
    lib().orc_potentials(_dp(v), v.shape[0], _ip(t), t.shape[0], float(np.real(k)),
                         float(np.imag(k)), _dp(ps.view(np.float64)), _dp(ph.view(np.float64)),
                         _dp(P), n, _dp(S), _dp(D))
    return S.view(np.complex128).copy(), D.view(np.complex128).copy()


def inside(verts, tris, pts):
    """Region of each point: the Laplace double layer of the constant 1,
    -DLP_0 1 = 1 inside the closed surface and 0 outside (Gauss)."""
    nv = np.asarray(verts).shape[0]
    _, D = potentials(verts, tris, 0.0, np.zeros(nv), np.ones(nv), pts)
    return -D.real > 0.5


def field(verts, tris, k_ext, k_int, rho_ratio, x, pts, inc="planewave", src=(0.0, 0.0, 1.0)):
    """Total pressure at points from a solution x = [psi; phi] of the permuted
    PMCHWT system (psi = exterior normal derivative, phi = trace of the total
    field, outward normal).  Outside (Sec. 2.2, exterior representation of the
    scattered field plus the incident field):
        u = u_inc + DLP_0 phi - SLP_0 psi;
    inside (interior representation with the interior traces phi and
    rho psi from the transmission conditions, rho = rho_int / rho_ext):
        u = rho SLP_1 psi - DLP_1 phi.
    Returns (u, inside mask)."""
    P = np.atleast_2d(np.asarray(pts, dtype=np.float64))
    nv = np.asarray(verts).shape[0]
    psi, phi = np.asarray(x)[:nv], np.asarray(x)[nv:]
    ins = inside(verts, tris, P)
    S0, D0 = potentials(verts, tris, k_ext, psi, phi, P)
    S1, D1 = potentials(verts, tris, k_int, psi, phi, P)
    s = np.asarray(src, dtype=np.float64)
    if inc == "planewave":
        uinc = np.exp(1j * k_ext * (P @ s))
    else:
        R = np.linalg.norm(P - s[None, :], axis=1)
        uinc = np.exp(1j * k_ext * R) / (4.0 * math.pi * R)
    u = np.where(ins, rho_ratio * S1 - D1, uinc + D0 - S0)
    return u, ins


def field_objects(verts, tris, k_ext, k_int, rho_ratio, x, pts, inc="planewave",
                  src=(0.0, 0.0, 1.0)):
    """Total pressure at points for disjoint objects with their own materials
    (k_int[m], rho_ratio[m]): outside every object the exterior
    representation over all surfaces plus the incident field; inside object m
    the interior representation over its own surface only.  Returns (u,
    region) with region m + 1 inside object m and 0 outside."""
    P = np.atleast_2d(np.asarray(pts, dtype=np.float64))
    t = np.asarray(tris)
    tc, _ = components(t)
    nv = np.asarray(verts).shape[0]
    psi, phi = np.asarray(x)[:nv], np.asarray(x)[nv:]
    region = np.zeros(P.shape[0], dtype=int)
    for m in range(tc.max() + 1):
        region[inside(verts, t[tc == m], P)] = m + 1
    S0, D0 = potentials(verts, t, k_ext, psi, phi, P)
    s = np.asarray(src, dtype=np.float64)
    if inc == "planewave":
        uinc = np.exp(1j * k_ext * (P @ s))
    else:
        R = np.linalg.norm(P - s[None, :], axis=1)
        uinc = np.exp(1j * k_ext * R) / (4.0 * math.pi * R)
    u = uinc + D0 - S0
    for m in range(tc.max() + 1):
        sel = region == m + 1
        if sel.any():
            Sm, Dm = potentials(verts, t[tc == m], k_int[m], psi, phi, P[sel])
            u[sel] = rho_ratio[m] * Sm - Dm
    return u, region


# --------------------------------------------------------------------------
# OSRC preconditioner (Sec. 2.6)
# --------------------------------------------------------------------------
def pade(n_pade, theta):
    """Coefficients of sqrt(1+z) ~ C0 + sum_j A_j z / (1 + B_j z).

    Real Pade of sqrt(1+x): a_j = 2/(2N+1) sin^2(j pi/(2N+1)),
    b_j = cos^2(j pi/(2N+1)).  The branch cut is rotated by theta through
    sqrt(1+z) = e^{i theta/2} sqrt(1 + ((1+z) e^{-i theta} - 1)); expanding
    that in z with zeta0 = e^{-i theta} - 1 gives
        C0  = e^{i theta/2} (1 + sum_j a_j zeta0 / (1 + b_j zeta0))
        A_j = e^{-i theta/2} a_j / (1 + b_j zeta0)^2
        B_j = e^{-i theta} b_j / (1 + b_j zeta0)."""
    N = int(n_pade)
    j = np.arange(1, N + 1)
    a = 2.0 / (2 * N + 1) * np.sin(j * math.pi / (2 * N + 1)) ** 2
    b = np.cos(j * math.pi / (2 * N + 1)) ** 2
    z0 = np.exp(-1j * theta) - 1.0
    C0 = np.exp(0.5j * theta) * (1.0 + np.sum(a * z0 / (1.0 + b * z0)))
    A = np.exp(-0.5j * theta) * a / (1.0 + b * z0) ** 2
    B = np.exp(-1j * theta) * b / (1.0 + b * z0)
    return C0, A, B


def pade_eval(z, n_pade, theta):
    C0, A, B = pade(n_pade, theta)
    z = np.asarray(z, dtype=np.complex128)
    return C0 + np.sum(A[:, None] * z[None, :] / (1.0 + B[:, None] * z[None, :]), axis=0)


def ntd_partial_fractions(n_pade, theta):
    """R(z)/(1+z) = g0/(1+z) + sum_j g_j/(1+B_j z) with R the rotated Pade
    approximant: g0 = R(-1) = C0 - sum_j A_j/(1-B_j), g_j = A_j/(1-B_j)."""
    C0, A, B = pade(n_pade, theta)
    g = A / (1.0 - B)
    return C0 - np.sum(g), g, B


def mean_edge_length(verts, tris):
    t = np.asarray(tris)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    e = np.unique(np.sort(e, axis=1), axis=0)
    return float(np.linalg.norm(verts[e[:, 0]] - verts[e[:, 1]], axis=1).mean())


def damped_wavenumber(k, R):
    """k_eps = k (1 + 0.4 i (k R)^(-2/3)) = k + 0.4 i k^(1/3) R^(-2/3)."""
    return k * (1.0 + 0.4j * (k * R) ** (-2.0 / 3.0))


class _ShiftedSolver:
    """Direct (sparse LU) solves of (M - beta S) w = f."""

    def __init__(self, M, S):
        self.M, self.S = M, S
        self._lu = {}

    def solve(self, beta, f):
        import scipy.sparse.linalg as spla

        key = complex(beta)
        lu = self._lu.get(key)
        if lu is None:
            A = (self.M - beta * self.S).astype(np.complex128).tocsc()
            lu = spla.splu(A)
            self._lu[key] = lu
        return lu.solve(np.asarray(f, dtype=np.complex128))


def osrc_apply(M, S, u1, u2, k, k_eps, n_pade, theta, solver=None):
    """Strong-form OSRC maps on coefficient vectors (Sec. 2.6, 2.7), with
    X = Delta_Gamma / k_eps^2 represented by -M^{-1} S / k_eps^2:
      DtN u1 = i k [C0 u1 + sum_j A_j w_j],   (M - B_j S/k_eps^2) w_j = -S u1/k_eps^2
      NtD u2 = 1/(i k) [g0 v_0 + sum_j g_j v_j],
               (M - S/k_eps^2) v_0 = M u2,    (M - B_j S/k_eps^2) v_j = M u2
    (NtD as the Pade square root times (1+X)^{-1}, in partial fractions)."""
    solver = solver or _ShiftedSolver(M, S)
    C0, A, B = pade(n_pade, theta)
    ke2 = k_eps * k_eps
    f1 = -(S @ u1) / ke2
    z1 = C0 * u1
    for j in range(len(A)):
        z1 = z1 + A[j] * solver.solve(B[j] / ke2, f1)
    z1 = 1j * k * z1
    g0, g, B2 = ntd_partial_fractions(n_pade, theta)
    f2 = M @ u2
    z2 = g0 * solver.solve(1.0 / ke2, f2)
    for j in range(len(g)):
        z2 = z2 + g[j] * solver.solve(B2[j] / ke2, f2)
    z2 = z2 / (1j * k)
    return z1, z2


def strong_apply(M, y):
    """M^{-1} on both block rows (mass preconditioning, Sec. 2.4)."""
    import scipy.sparse.linalg as spla

    nv = M.shape[0]
    lu = spla.splu(M.astype(np.complex128).tocsc())
    y = np.asarray(y, dtype=np.complex128)
    return np.concatenate([lu.solve(y[:nv]), lu.solve(y[nv:])])


def gmres(apply, c, tol, maxit):
    """GMRES without restart, x0 = 0, modified Gram-Schmidt Arnoldi and
    Givens rotations; stops when the residual estimate |g_{j+1}| <= tol |c|.
    Returns (x, iterations, residual history)."""
    n = c.shape[0]
    beta = np.linalg.norm(c)
    if beta == 0.0:
        return np.zeros(n, dtype=np.complex128), 0, [0.0]
    Vb = np.zeros((maxit + 1, n), dtype=np.complex128)
    H = np.zeros((maxit + 1, maxit), dtype=np.complex128)
    cs = np.zeros(maxit)
    sn = np.zeros(maxit, dtype=np.complex128)
    g = np.zeros(maxit + 1, dtype=np.complex128)
    g[0] = beta
    Vb[0] = c / beta
    hist = [1.0]
    j = 0
    for j in range(maxit):
        w = apply(Vb[j])
        for i in range(j + 1):
            H[i, j] = np.vdot(Vb[i], w)
            w = w - H[i, j] * Vb[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] != 0.0:
            Vb[j + 1] = w / H[j + 1, j]
        for i in range(j):
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        a, b = H[j, j], H[j + 1, j]
        nu = math.hypot(abs(a), abs(b))
        if abs(a) == 0.0:
            cs[j], sn[j] = 0.0, 1.0
        else:
            cs[j] = abs(a) / nu
            sn[j] = (a / abs(a)) * np.conj(b) / nu
        H[j, j] = cs[j] * a + sn[j] * b
        H[j + 1, j] = 0.0
        g[j + 1] = -np.conj(sn[j]) * g[j]
        g[j] = cs[j] * g[j]
        res = abs(g[j + 1]) / beta
        hist.append(res)
        if res <= tol:
            j += 1
            break
    else:
        j = maxit
    y = np.linalg.solve(np.triu(H[:j, :j]), g[:j])
    x = Vb[:j].T @ y
    return x, j, hist


class Problem:
    """Dense oracle of one transmission problem: the permuted PMCHWT matrix,
    M, S and the OSRC preconditioner; meant for meshes of a few thousand
    vertices at most."""

    def __init__(self, verts, tris, k_ext, k_int, rho_ratio, n_pade=4,
                 theta=math.pi / 3, damping_R=None, osrc_side=1, nss=6, precond="osrc",
                 objects=None, formulation="pmchwt"):
        """objects = (k_int list, rho_ratio list): one material per connected
        component (disjoint objects); k_int and rho_ratio are then unused."""
        self.verts = np.asarray(verts, dtype=np.float64)
        self.tris = np.asarray(tris, dtype=np.int32)
        self.nv = self.verts.shape[0]
        self.k_ext, self.k_int, self.rho = k_ext, k_int, rho_ratio
        self.n_pade, self.theta, self.nss = n_pade, theta, nss
        self.R = damping_R if damping_R else mean_edge_length(self.verts, self.tris)
        self.objects = objects
        if objects is None:
            self.k_osrc = k_int if osrc_side == 1 else k_ext
            self.k_eps = damped_wavenumber(self.k_osrc, self.R)
            self.B = pmchwt_matrix(self.verts, self.tris, k_ext, k_int, rho_ratio, nss,
                                   formulation=formulation)
        else:
            _, self.vcomp = components(self.tris)
            kl = list(objects[0])
            self.k_osrc_obj = [kl[m] if osrc_side == 1 else k_ext for m in range(len(kl))]
            self.B = pmchwt_matrix_objects(self.verts, self.tris, k_ext, kl, list(objects[1]), nss,
                                           formulation=formulation)
        self.M, self.S = mass_stiffness(self.verts, self.tris)
        self._solver = _ShiftedSolver(self.M, self.S)
        self.precond_kind = precond

    def rhs(self, kind="planewave", src=(0.0, 0.0, 1.0)):
        return rhs(self.verts, self.tris, self.k_ext, kind, src)

    def precond(self, y):
        """P u on strong-form coefficient vectors: diag(DtN, NtD) u (OSRC,
        Sec. 2.6); u itself (mass preconditioning only, Sec. 2.4); or the
        Calderon preconditioner of Sec. 2.5 for one object, C = A_0 + A^_1,
        which is the PMCHWT operator in the unpermuted ordering [phi; psi]:
        with the permuted B acting on [psi; phi], P u = M^-1 B [u2; u1]."""
        nv = self.nv
        if self.precond_kind == "mass":
            return np.asarray(y).copy()
        if self.precond_kind == "calderon":
            y = np.asarray(y)
            return strong_apply(self.M, self.B @ np.concatenate([y[nv:], y[:nv]]))
        if self.objects is not None:
            # block-diagonal OSRC: each object with its own wavenumber
            y = np.asarray(y)
            z1 = np.zeros(nv, dtype=complex)
            z2 = np.zeros(nv, dtype=complex)
            for m, k in enumerate(self.k_osrc_obj):
                idx = np.nonzero(self.vcomp == m)[0]
                Mm = self.M[idx][:, idx]
                Sm = self.S[idx][:, idx]
                z1[idx], z2[idx] = osrc_apply(Mm, Sm, y[idx], y[nv + idx], k,
                                              damped_wavenumber(k, self.R), self.n_pade,
                                              self.theta)
            return np.concatenate([z1, z2])
        z1, z2 = osrc_apply(self.M, self.S, y[:nv], y[nv:], self.k_osrc,
                            self.k_eps, self.n_pade, self.theta, self._solver)
        return np.concatenate([z1, z2])

    def apply_preconditioned(self, x):
        """P M^{-1} B x (Sec. 2.7 with mass preconditioning, Sec. 3.1)."""
        return self.precond(strong_apply(self.M, self.B @ x))

    def solve_direct(self, b):
        return np.linalg.solve(self.B, b)

    def solve_gmres(self, b, tol=1e-8, maxit=500):
        c = self.precond(strong_apply(self.M, b))
        return gmres(self.apply_preconditioned, c, tol, maxit)
