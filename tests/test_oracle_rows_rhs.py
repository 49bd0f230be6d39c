"""Pins of two oracle functions that the full-size parity tests rest on.

1. Row assembly (``assemble_rows`` / ``pmchwt_rows``): the rows of the
   permuted PMCHWT matrix of Sec. 2.7 for selected test vertices.  Its own
   loop (test-vertex search, scatter into the row, the far / near / all
   mask) must give exactly the rows of the dense assembler, which is pinned
   elsewhere by the solid-angle identity, symmetries, brute force and the
   sphere spectra.

2. Point-source right-hand side (``rhs(kind="pointsource")``): the data of
   Sec. 2.7 for the incident field G_0(x, x0) = exp(i k |x - x0|)/(4 pi |x - x0|)
   (the synthetic stand-in for the transducer of Sec. 3.6).  Pinned against
   mathematics that the oracle does not contain:
     - Gauss' flux identity at k = 0: the integral of dG_0/dn over a closed
       surface is -1 for a source inside and 0 outside; it holds exactly on
       the flat-triangle surface, so only the 6-point rule's error remains;
     - the addition theorem on a sphere of radius a: for |x0| = d,
       int G = i k a^2 j_0(k r<) h_0(k r>), int dG/dn = i k^2 a^2 j_0(k d) h_0'(k a)
       (source inside) or i k^2 a^2 j_0'(k a) h_0(k d) (outside), and the
       first moments int y_z G, int y_z dG/dn with j_1, h_1 and cos(theta_0);
       the polyhedral sphere converges to these O(h^2).  Weighting the vertex
       values by z_i tests how the right-hand side is spread over the
       vertices (sum_i z_i phi_i = z exactly on flat triangles);
     - a 20 x 20 collapsed Gauss integral of the same integrands against the
       hat functions, triangle by triangle, on a small tetrahedron.
"""
import math

import numpy as np
import pytest
from scipy.special import spherical_jn, spherical_yn

import oracle as O
from paper_2104_04609_gb300.inputs import fibonacci_hull, icosphere


# --------------------------------------------------------------------------
# 1. row assembly
# --------------------------------------------------------------------------
@pytest.fixture(scope="module", params=["icosphere2", "fib150"])
def mesh(request):
    if request.param == "icosphere2":
        return icosphere(2)
    return fibonacci_hull(150)


@pytest.mark.parametrize("part", [1, 2, 3])
def test_pmchwt_rows_equal_dense_rows(mesh, part):
    v, t = mesh
    nv = v.shape[0]
    k0, k1, rho = 2.5, 4.0 + 0.3j, 1.7
    A = O.pmchwt_matrix(v, t, k0, k1, rho, nss=4, part=part)
    rng = np.random.default_rng(7)
    rows = np.unique(np.concatenate([[0, nv - 1], rng.choice(nv, 10, replace=False)]))
    R1, R2 = O.pmchwt_rows(v, t, k0, k1, rho, rows, nss=4, part=part)
    scale = np.abs(A).max()
    assert R1.shape == (len(rows), 2 * nv) and R2.shape == (len(rows), 2 * nv)
    assert np.abs(R1 - A[rows]).max() < 1e-14 * scale
    assert np.abs(R2 - A[nv + rows]).max() < 1e-14 * scale
    # the mask really selects: far and near parts add up to the whole and
    # neither is empty
    if part != 3:
        other = O.pmchwt_rows(v, t, k0, k1, rho, rows, nss=4, part=3 - part)
        full = O.pmchwt_rows(v, t, k0, k1, rho, rows, nss=4, part=3)
        assert np.abs(R1).max() > 1e-3 * scale and np.abs(other[0]).max() > 1e-3 * scale
        assert np.abs(R1 + other[0] - full[0]).max() < 1e-14 * scale
        assert np.abs(R2 + other[1] - full[1]).max() < 1e-14 * scale


def test_assemble_rows_operator_blocks(mesh):
    """Each of V, K, T, D separately, at a real and a complex wavenumber."""
    v, t = mesh
    rows = np.array([3, 17, 41], dtype=np.int32)
    for k in (3.0, 2.0 + 0.5j):
        full = O.assemble(v, t, k, nss=4, part=3)
        part_rows = O.assemble_rows(v, t, k, rows, nss=4, part=3)
        for F, Rw in zip(full, part_rows):
            assert np.abs(Rw - F[rows]).max() < 1e-14 * np.abs(F).max()


# --------------------------------------------------------------------------
# 2. point-source right-hand side
# --------------------------------------------------------------------------
def _h(l, z, deriv=False):
    return spherical_jn(l, z, deriv) + 1j * spherical_yn(l, z, deriv)


def _sphere_moments(k, a, x0):
    """(int G, int y_z G, int dG/dn, int y_z dG/dn) over the sphere of radius
    a for the point source at x0 (addition theorem, see the module doc)."""
    d = float(np.linalg.norm(x0))
    cth = x0[2] / d
    if d < a:
        m0 = 1j * k * a ** 2 * spherical_jn(0, k * d) * _h(0, k * a)
        m1 = 1j * k * a ** 3 * spherical_jn(1, k * d) * _h(1, k * a) * cth
        n0 = 1j * k ** 2 * a ** 2 * spherical_jn(0, k * d) * _h(0, k * a, True)
        n1 = 1j * k ** 2 * a ** 3 * spherical_jn(1, k * d) * _h(1, k * a, True) * cth
    else:
        m0 = 1j * k * a ** 2 * spherical_jn(0, k * a) * _h(0, k * d)
        m1 = 1j * k * a ** 3 * spherical_jn(1, k * a) * _h(1, k * d) * cth
        n0 = 1j * k ** 2 * a ** 2 * spherical_jn(0, k * a, True) * _h(0, k * d)
        n1 = 1j * k ** 2 * a ** 3 * spherical_jn(1, k * a, True) * _h(1, k * d) * cth
    return m0, m1, n0, n1


@pytest.mark.parametrize("x0,inside", [((0.2, -0.1, 0.3), True), ((0.0, 0.0, 0.0), True),
                                       ((3.0, 0.0, 0.0), False), ((1.1, 0.9, -0.7), False)])
def test_pointsource_gauss_flux_k0(x0, inside):
    errs = []
    for level in (2, 3, 4):
        v, t = icosphere(level)
        b = O.rhs(v, t, 0.0, kind="pointsource", src=x0)
        nv = v.shape[0]
        flux = b[nv:].sum()
        assert abs(flux.imag) < 1e-15
        errs.append(abs(flux.real - (-1.0 if inside else 0.0)))
    # exact on the polyhedron up to the 6-point rule's error, which falls
    # fast with h for a source away from the surface
    assert errs[-1] < 1e-6, errs
    assert errs[2] <= errs[0], errs


@pytest.mark.parametrize("k", [0.0, 1.5, 4.0])
@pytest.mark.parametrize("x0", [(0.15, -0.2, 0.35), (1.2, 2.0, 1.5)])
def test_pointsource_sphere_closed_forms(k, x0):
    x0 = np.array(x0)
    kk = k if k > 0 else 1e-9
    ref = _sphere_moments(kk, 1.0, x0)
    errs = []
    for level in (2, 3, 4):
        v, t = icosphere(level)
        nv = v.shape[0]
        b = O.rhs(v, t, k, kind="pointsource", src=x0)
        z = v[:, 2]
        got = (b[:nv].sum(), z @ b[:nv], b[nv:].sum(), z @ b[nv:])
        errs.append([abs(g - r) / max(abs(r), 1e-3) for g, r in zip(got, ref)])
    errs = np.array(errs)
    # polyhedral sphere -> sphere: O(h^2), a factor about 4 per level
    assert (errs[2] < 6e-3).all(), errs
    ratio = errs[1] / np.maximum(errs[2], 1e-12)
    assert (ratio > 2.5).all() or (errs[2] < 1e-6).all(), errs


def _collapsed_gauss(n):
    """n x n rule on the reference triangle {0 <= l2, l1 + l2 <= 1} by the
    collapsed map (u, v) -> (u, v (1 - u)); returns (l1, l2), weights (sum 1/2)."""
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    U, Vv = np.meshgrid(x, x, indexing="ij")
    WU, WV = np.meshgrid(w, w, indexing="ij")
    l1 = U.ravel()
    l2 = (Vv * (1.0 - U)).ravel()
    wt = (WU * WV * (1.0 - U)).ravel()
    return np.stack([l1, l2], axis=1), wt


def _tet_brute(scale, k, x0):
    v = scale * np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 0.9, 0.1], [0.3, 0.3, 0.8]])
    t = np.array([[0, 2, 1], [0, 1, 3], [1, 2, 3], [0, 3, 2]], dtype=np.int32)
    b = O.rhs(v, t, k, kind="pointsource", src=x0)
    pts, wts = _collapsed_gauss(20)
    ref = np.zeros(8, dtype=complex)
    for tri in t:
        P0, P1, P2 = v[tri]
        nrm = np.cross(P1 - P0, P2 - P0)
        area2 = np.linalg.norm(nrm)
        n = nrm / area2
        for (l1, l2), wq in zip(pts, wts):
            y = P0 + l1 * (P1 - P0) + l2 * (P2 - P0)
            d = y - x0
            R = np.linalg.norm(d)
            e = np.exp(1j * k * R)
            G = e / (4 * math.pi * R)
            dG = e * (1j * k * R - 1.0) / (4 * math.pi * R ** 3) * (d @ n)
            lam = (1.0 - l1 - l2, l1, l2)
            for a in range(3):
                ref[tri[a]] += wq * area2 * lam[a] * G
                ref[4 + tri[a]] += wq * area2 * lam[a] * dG
    return np.abs(b - ref).max() / np.abs(ref).max()


def test_pointsource_brute_force_tetrahedron():
    """Vertex by vertex against a 20^2 collapsed Gauss rule per triangle:
    b1_i = int G_0(., x0) phi_i and b2_i = int dG_0/dn(., x0) phi_i.  The
    difference is the 6-point rule's error: small (a wrong sign, factor or
    vertex would be of order one) and falling fast as the triangles shrink
    (degree-4 rule)."""
    x0 = np.array([0.9, -0.4, 0.6])
    e1 = _tet_brute(0.2, 6.0, x0)
    e2 = _tet_brute(0.1, 6.0, x0)
    assert e1 < 1e-4, e1
    assert e2 < e1 / 8, (e1, e2)
