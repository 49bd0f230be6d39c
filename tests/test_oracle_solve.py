"""Pins of the whole oracle solve: the permuted PMCHWT system of Sec. 2.7
reproduces the Mie series of a penetrable sphere (Sec. 3.2), with error
decreasing O(h^2); OSRC-preconditioned GMRES (Sec. 3.1) reproduces the direct
solution."""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre, spherical_jn, spherical_yn

import oracle as O
from paper_2104_04609_gb300.inputs import icosphere


def mie_traces(k0, k1, rho, a, cth):
    """phi = gamma_D u_tot and psi = gamma_N^+ u_tot on a sphere of radius a
    for the plane wave exp(i k0 z); rho = rho_int/rho_ext."""
    L = int(k0 * a + 4 * (k0 * a) ** (1 / 3) + 15)
    phi = np.zeros_like(cth, dtype=complex)
    psi = np.zeros_like(cth, dtype=complex)
    for l in range(L):
        j0, j0p = spherical_jn(l, k0 * a), spherical_jn(l, k0 * a, True)
        h0 = j0 + 1j * spherical_yn(l, k0 * a)
        h0p = j0p + 1j * spherical_yn(l, k0 * a, True)
        j1, j1p = spherical_jn(l, k1 * a), spherical_jn(l, k1 * a, True)
        al = ((k1 / rho) * j1p * j0 - k0 * j1 * j0p) / (k0 * j1 * h0p - (k1 / rho) * j1p * h0)
        P = eval_legendre(l, cth)
        phi += (2 * l + 1) * 1j ** l * (j0 + al * h0) * P
        psi += k0 * (2 * l + 1) * 1j ** l * (j0p + al * h0p) * P
    return phi, psi


def mie_field(k0, k1, rho, a, pts):
    """Total field of the penetrable sphere of radius a for the plane wave
    exp(i k0 z): outside sum (2l+1) i^l [j_l(k0 r) + a_l h_l(k0 r)] P_l(cos th),
    inside sum (2l+1) i^l c_l j_l(k1 r) P_l(cos th) with c_l from continuity of
    the pressure at r = a."""
    P = np.atleast_2d(pts)
    r = np.linalg.norm(P, axis=1)
    cth = np.where(r > 0, P[:, 2] / np.where(r > 0, r, 1.0), 1.0)
    L = int(max(abs(k0), abs(k1)) * max(a, r.max()) + 4 * (abs(k1) * a) ** (1 / 3) + 20)
    u = np.zeros(P.shape[0], dtype=complex)
    out = r > a
    for l in range(L):
        j0, j0p = spherical_jn(l, k0 * a), spherical_jn(l, k0 * a, True)
        h0 = j0 + 1j * spherical_yn(l, k0 * a)
        h0p = j0p + 1j * spherical_yn(l, k0 * a, True)
        j1, j1p = spherical_jn(l, k1 * a), spherical_jn(l, k1 * a, True)
        al = ((k1 / rho) * j1p * j0 - k0 * j1 * j0p) / (k0 * j1 * h0p - (k1 / rho) * j1p * h0)
        cl = (j0 + al * h0) / j1
        Pl = eval_legendre(l, cth)
        ro = np.where(out, r, a)
        ext = spherical_jn(l, k0 * ro) + al * (spherical_jn(l, k0 * ro) + 1j * spherical_yn(l, k0 * ro))
        inn = cl * spherical_jn(l, k1 * np.where(out, a, r))
        u += (2 * l + 1) * 1j ** l * np.where(out, ext, inn) * Pl
    return u


def _merr(M, a, e):
    d = a - e
    return math.sqrt(abs(np.vdot(d, M @ d)) / abs(np.vdot(e, M @ e)))


@pytest.mark.slow
def test_mie_sphere():
    errs = []
    for lev in (2, 3):
        v, t = icosphere(lev)
        P = O.Problem(v, t, 2.0, 3.0, 1.5)
        b = P.rhs()
        x = P.solve_direct(b)
        nv = v.shape[0]
        phi_ex, psi_ex = mie_traces(2.0, 3.0, 1.5, 1.0, v[:, 2])
        errs.append((_merr(P.M, x[nv:], phi_ex), _merr(P.M, x[:nv], psi_ex)))
        if lev == 3:
            xg, it, hist = P.solve_gmres(b, tol=1e-8, maxit=200)
            assert hist[-1] <= 1e-8
            assert np.linalg.norm(xg - x) / np.linalg.norm(x) < 1e-6
            assert it < 60
    (p2, s2), (p3, s3) = errs
    assert p3 < 0.015 and s3 < 0.015
    assert p3 < 0.35 * p2 and s3 < 0.35 * s2


def test_gmres_small_dense():
    rng = np.random.default_rng(5)
    n = 40
    A = np.eye(n) * 3 + rng.standard_normal((n, n)) * 0.3 + 1j * rng.standard_normal((n, n)) * 0.3
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, it, hist = O.gmres(lambda y: A @ y, b, 1e-12, 100)
    assert np.linalg.norm(A @ x - b) / np.linalg.norm(b) < 1e-11
    assert it <= n
