"""Pins of the oracle's Galerkin operators (Sec. 2.2) against mathematics
that does not depend on the oracle: Gauss' solid-angle identity, null spaces,
symmetries, a brute-force separated pair and the sphere spectra (spherical
harmonics are eigenfunctions of V, K, T, D with Bessel/Hankel eigenvalues)."""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre, spherical_jn, spherical_yn

import oracle as O
from paper_2104_04609_gb300.inputs import icosphere


@pytest.fixture(scope="module")
def sphere2():
    v, t = icosphere(2)
    return v, t


def test_laplace_identities(sphere2):
    v, t = sphere2
    V, K, T, D = O.assemble(v, t, 0.0)
    M, S = O.mass_stiffness(v, t)
    one = np.ones(v.shape[0])
    m1 = M @ one
    # Gauss: int_Gamma dG/dn_y(x, y) dy = -1/2 for x on a closed surface
    assert np.abs(K @ one + 0.5 * m1).max() / np.abs(m1).max() < 1e-5
    assert np.abs(one @ T + 0.5 * m1).max() / np.abs(m1).max() < 1e-5
    # the hypersingular operator annihilates constants at k = 0
    assert np.abs(D @ one).max() < 1e-13
    assert np.abs(S @ one).max() < 1e-13
    # sum of the mass matrix = surface area of the polyhedron
    p0, p1, p2 = (v[t[:, i]] for i in range(3))
    area = 0.5 * np.linalg.norm(np.cross(p1 - p0, p2 - p0), axis=1).sum()
    assert abs(M.sum() - area) < 1e-12


@pytest.mark.parametrize("k", [0.0, 2.5, 1.5 + 0.3j])
def test_symmetries(sphere2, k):
    v, t = sphere2
    V, K, T, D = O.assemble(v, t, k)
    assert np.abs(V - V.T).max() / np.abs(V).max() < 1e-8   # complex symmetric
    assert np.abs(D - D.T).max() / np.abs(D).max() < 1e-8
    assert np.abs(T - K.T).max() / np.abs(K).max() < 1e-6   # T = K^T
    if k != 0:
        assert np.abs(V - V.conj().T).max() / np.abs(V).max() > 1e-3  # not Hermitian


def _tri_rule(n):
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    U, W = np.meshgrid(x, x, indexing="ij")
    WU, WW = np.meshgrid(w, w, indexing="ij")
    bary = np.stack([1.0 - U, U * (1.0 - W), U * W], -1).reshape(-1, 3)
    return bary, (2.0 * WU * WW * U).ravel()   # weights sum to 1


def test_separated_pair_brute_force():
    """Well-separated triangles: the 6x6 rule agrees with a 30x30-per-triangle
    collapsed Gauss evaluation of the operator definitions to the rule's
    accuracy; any dropped term, sign or transposed index shows up at O(1)."""
    verts = np.array([[0.0, 0.0, 0.0], [0.3, 0.05, 0.02], [0.1, 0.28, -0.03],
                      [1.0, 0.2, 0.5], [1.1, 0.45, 0.4], [0.9, 0.3, 0.8]])
    tris = np.array([[0, 1, 2], [3, 4, 5]], dtype=np.int32)
    k = 4.0
    kase, V, K, T, D = O.pair_matrices(verts, tris, 0, 1, k)
    assert kase == 0
    b, w = _tri_rule(30)
    P, Q = verts[:3], verts[3:]
    def geom(X):
        n = np.cross(X[1] - X[0], X[2] - X[0]); a = 0.5 * np.linalg.norm(n); n = n / (2 * a)
        grads = [np.cross(n, X[(i + 2) % 3] - X[(i + 1) % 3]) / (2 * a) for i in range(3)]
        curls = [np.cross(n, g) for g in grads]
        return n, a, np.array(curls)
    nx, ax, cx = geom(P)
    ny, ay, cy = geom(Q)
    x = b @ P
    y = b @ Q
    d = x[:, None, :] - y[None, :, :]
    r = np.linalg.norm(d, axis=-1)
    G = np.exp(1j * k * r) / (4 * math.pi * r)
    dGdny = G * (1j * k * r - 1) / r ** 2 * np.einsum("pqj,j->pq", -d, ny)
    dGdnx = G * (1j * k * r - 1) / r ** 2 * np.einsum("pqj,j->pq", d, nx)
    W = np.outer(w, w) * ax * ay
    ref = {}
    ref["V"] = np.einsum("pq,pa,qb->ab", W * G, b, b)
    ref["K"] = np.einsum("pq,pa,qb->ab", W * dGdny, b, b)
    ref["T"] = np.einsum("pq,pa,qb->ab", W * dGdnx, b, b)
    ref["D"] = (cx @ cy.T) * (W * G).sum() - k * k * np.dot(nx, ny) * ref["V"]
    for name, mat in zip("VKTD", (V, K, T, D)):
        e = np.abs(mat - ref[name]).max() / np.abs(ref[name]).max()
        assert e < 1e-4, (name, e)


def _sphere_eigs(l, k, a=1.0):
    x = k * a
    j, jp = spherical_jn(l, x), spherical_jn(l, x, True)
    h = j + 1j * spherical_yn(l, x)
    hp = jp + 1j * spherical_yn(l, x, True)
    lv = 1j * k * a * a * j * h
    lk = 0.5 + 1j * k * k * a * a * j * hp
    ld = -1j * k ** 3 * a * a * jp * hp
    return lv, lk, ld


def test_sphere_eigenvalue_closed_forms():
    # Calderon projector on the sphere: lambda_K^2 + lambda_V lambda_D = 1/4
    for k in (0.5, 2.0, 7.3):
        for l in range(6):
            lv, lk, ld = _sphere_eigs(l, k)
            assert abs(lk * lk + lv * ld - 0.25) < 1e-12
    # k -> 0 limits: a/(2l+1), -1/(2(2l+1)), l(l+1)/((2l+1) a)
    for l in range(1, 5):
        lv, lk, ld = _sphere_eigs(l, 1e-4)
        assert abs(lv - 1.0 / (2 * l + 1)) < 1e-6
        assert abs(lk + 0.5 / (2 * l + 1)) < 1e-6
        assert abs(ld - l * (l + 1) / (2 * l + 1)) < 1e-6


@pytest.mark.slow
def test_sphere_spectra_converge():
    """Galerkin Rayleigh quotients of interpolated Y_l0 converge O(h^2) to the
    sphere eigenvalues for V, K, T, D at k = 2."""
    k = 2.0
    errs = {}
    for lev in (2, 3):
        v, t = icosphere(lev)
        V, K, T, D = O.assemble(v, t, k)
        M, _ = O.mass_stiffness(v, t)
        for l in range(4):
            u = eval_legendre(l, v[:, 2])
            den = u @ (M @ u)
            lv, lk, ld = _sphere_eigs(l, k)
            for name, A, e in (("V", V, lv), ("K", K, lk), ("T", T, lk), ("D", D, ld)):
                errs[(lev, l, name)] = abs((u @ (A @ u)) / den - e) / max(abs(e), 0.5)
    for l in range(4):
        for name in "VKTD":
            e2, e3 = errs[(2, l, name)], errs[(3, l, name)]
            assert e3 < 0.02, (l, name, e3)
            assert e3 < 0.35 * e2, (l, name, e2, e3)
