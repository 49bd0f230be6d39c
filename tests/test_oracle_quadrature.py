"""Pins of the oracle's quadrature against exact integrals.

- 6-point rule: exact for every monomial of degree <= 4 on a triangle.
- Gauss-Legendre: equal to numpy's independent Golub-Welsch nodes.
- Sauter-Schwab transformations (Sauter & Schwab, Sec. 5.2): each case's point
  set integrates polynomials on That x That exactly (the maps tile the 4-D
  domain with the right Jacobian), and singular integrals converge to
  closed forms / brute force."""
import math

import numpy as np
import pytest

import oracle as O


def test_quad6_degree4_exact():
    b, w = O.quad6()
    assert abs(w.sum() - 1.0) < 1e-15
    # int over the unit right triangle of l1^a l2^b = a! b! / (a+b+2)!, area 1/2
    for a in range(6):
        for c in range(6 - a):
            got = (w * b[:, 1] ** a * b[:, 2] ** c).sum()
            exact = 2.0 * math.factorial(a) * math.factorial(c) / math.factorial(a + c + 2)
            if a + c <= 4:
                assert abs(got - exact) < 1e-14, (a, c)
    # degree 5 is not integrated exactly (the rule is degree 4, not higher)
    got = (w * b[:, 1] ** 5).sum()
    assert abs(got - 2.0 * math.factorial(5) / math.factorial(7)) > 1e-6


@pytest.mark.parametrize("n", [1, 2, 5, 8, 13])
def test_gauss_legendre_matches_numpy(n):
    x, w = O.gauss_legendre(n)
    t, tw = np.polynomial.legendre.leggauss(n)
    ref_x = np.sort(0.5 * (t + 1.0))
    order = np.argsort(x)
    assert np.allclose(x[order], ref_x, atol=1e-14)
    assert np.allclose(w[order], 0.5 * tw[np.argsort(0.5 * (t + 1.0))], atol=1e-14)


def _tri_moment(a, b):
    # int_{0<=x2<=x1<=1} x1^a x2^b
    return 1.0 / ((b + 1) * (a + b + 2))


@pytest.mark.parametrize("kase", [1, 2, 3])
def test_sauter_schwab_polynomial_moments(kase):
    P, w = O.ss_rule(kase, 6)
    assert abs(w.sum() - 0.25) < 1e-14
    for a in range(4):
        for b in range(4 - a):
            for c in range(4 - a - b):
                for d in range(4 - a - b - c):
                    got = (w * P[:, 0] ** a * P[:, 1] ** b * P[:, 2] ** c * P[:, 3] ** d).sum()
                    assert abs(got - _tri_moment(a, b) * _tri_moment(c, d)) < 1e-14


@pytest.mark.parametrize("kase", [1, 2, 3])
def test_sauter_schwab_points_inside(kase):
    P, _ = O.ss_rule(kase, 5)
    assert (P[:, 1] >= -1e-15).all() and (P[:, 1] <= P[:, 0] + 1e-15).all()
    assert (P[:, 3] >= -1e-15).all() and (P[:, 3] <= P[:, 2] + 1e-15).all()
    assert (P[:, 0] <= 1 + 1e-15).all() and (P[:, 2] <= 1 + 1e-15).all()


def _wilton_inplane(x, tri):
    """int_T 1/|x-y| dS_y for x in the plane of T (inside), by summing over
    the edges  d_i ln((R+ + l+)/(R- + l-))  (polar integration about x)."""
    tot = 0.0
    for i in range(3):
        A, B = tri[i], tri[(i + 1) % 3]
        u = (B - A) / np.linalg.norm(B - A)
        lm, lp = np.dot(A - x, u), np.dot(B - x, u)
        foot = A + np.dot(x - A, u) * u
        d = np.linalg.norm(x - foot)
        Rm, Rp = np.linalg.norm(A - x), np.linalg.norm(B - x)
        tot += d * math.log((Rp + lp) / (Rm + lm))
    return tot


def _duffy_rule(n):
    """Collapsed tensor Gauss rule on the unit right triangle (weights sum 1/2)."""
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    U, Vv = np.meshgrid(x, x, indexing="ij")
    WU, WV = np.meshgrid(w, w, indexing="ij")
    l1 = U * (1.0 - Vv)
    l2 = U * Vv
    return np.stack([l1.ravel(), l2.ravel()], 1), (WU * WV * U).ravel()


def test_coincident_laplace_single_layer_closed_form():
    """Sum of the 3x3 coincident V at k = 0 equals (1/4 pi) int_T Phi(x) dx
    with Phi the closed-form potential of a flat triangle."""
    verts = np.array([[0.0, 0.0, 0.0], [1.0, 0.2, 0.0], [0.3, 0.9, 0.0]])
    tris = np.array([[0, 1, 2]], dtype=np.int32)
    kase, V, K, T, D = O.pair_matrices(verts, tris, 0, 0, 0.0, nss=10)
    assert kase == 3
    pts, w = _duffy_rule(40)
    P0, P1, P2 = verts
    area = 0.5 * np.linalg.norm(np.cross(P1 - P0, P2 - P0))
    ref = 0.0
    for (l1, l2), wi in zip(pts, w):
        x = P0 + l1 * (P1 - P0) + l2 * (P2 - P0)
        ref += wi * 2.0 * area * _wilton_inplane(x, verts)
    ref /= 4.0 * math.pi
    assert abs(V.sum().real - ref) / ref < 2e-6
    assert abs(V.sum().imag) < 1e-15
    # flat coincident triangles: (x - y).n = 0, so K and T vanish identically
    assert np.abs(K).max() < 1e-15 and np.abs(T).max() < 1e-15


@pytest.mark.parametrize("pair", ["coincident", "edge", "vertex"])
def test_sauter_schwab_exponential_convergence(pair):
    verts = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 0.9, 0.1],
                      [0.6, -0.8, 0.3], [-0.7, -0.2, 0.4]])
    tris = np.array([[0, 1, 2], [1, 0, 3], [0, 3, 4]], dtype=np.int32)
    s = {"coincident": 0, "edge": 1, "vertex": 2}[pair]
    vals = []
    for n in (4, 6, 8, 12):
        kase, V, K, T, D = O.pair_matrices(verts, tris, 0, s, 3.0, nss=n)
        vals.append(np.concatenate([V.ravel(), K.ravel(), T.ravel(), D.ravel()]))
    assert kase == {"coincident": 3, "edge": 2, "vertex": 1}[pair]
    scale = np.abs(vals[-1]).max()
    e = [np.abs(v - vals[-1]).max() / scale for v in vals[:-1]]
    assert e[0] < 1e-3 and e[1] < 1e-5 and e[2] < 1e-7, e
    assert e[2] < e[1] < e[0]


def test_sauter_schwab_edge_pair_brute_force():
    """Edge-adjacent pair, k = 0: Sauter-Schwab V equals a brute-force
    integral that integrates the closed-form potential of the source triangle
    (out of its plane) over the test triangle."""
    verts = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.3, 0.8, 0.0], [0.5, -0.6, 0.5]])
    tris = np.array([[0, 1, 2], [1, 0, 3]], dtype=np.int32)
    kase, V, K, T, D = O.pair_matrices(verts, tris, 0, 1, 0.0, nss=10)
    assert kase == 2
    src = verts[[1, 0, 3]]
    n = np.cross(src[1] - src[0], src[2] - src[0])
    n /= np.linalg.norm(n)

    def potential(x):
        # int_T 1/|x-y| dS for x off the plane (Wilton et al. 1984)
        w = np.dot(x - src[0], n)
        xp = x - w * n
        tot = 0.0
        for i in range(3):
            A, B = src[i], src[(i + 1) % 3]
            u = (B - A) / np.linalg.norm(B - A)
            m = np.cross(u, n)  # outward in-plane edge normal for CCW src
            lm, lp = np.dot(A - xp, u), np.dot(B - xp, u)
            P0 = np.dot(A - xp, m)
            R0sq = P0 * P0 + w * w
            Rm = math.sqrt(lm * lm + R0sq)
            Rp = math.sqrt(lp * lp + R0sq)
            if abs(P0) > 1e-14:
                tot += P0 * math.log((Rp + lp) / (Rm + lm))
                tot -= abs(w) * (math.atan(P0 * lp / (R0sq + abs(w) * Rp)) -
                                 math.atan(P0 * lm / (R0sq + abs(w) * Rm)))
        return tot

    pts, wq = _duffy_rule(60)
    P0, P1, P2 = verts[[0, 1, 2]]
    area_t = 0.5 * np.linalg.norm(np.cross(P1 - P0, P2 - P0))
    ref = 0.0
    # collapse towards P2 so that the shared edge P0P1 is sampled densely
    for (l1, l2), wi in zip(pts, wq):
        x = P2 + l1 * (P0 - P2) + l2 * (P1 - P2)
        ref += wi * 2.0 * area_t * potential(x)
    ref /= 4.0 * math.pi
    assert abs(V.sum().real - ref) / abs(ref) < 1e-5


def test_quad6_matches_published_table():
    """The oracle's 6-point rule equals Dunavant's published degree-4 table
    (tests/golden/dunavant_p4_n6.txt) up to the order of the points."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "dunavant_p4_n6.txt")
    rows = [list(map(float, l.split())) for l in open(path) if l.strip() and not l.startswith("#")]
    ref = []
    for w, a, b, c in rows:
        for perm in {(a, b, c), (b, c, a), (c, a, b)}:
            ref.append((w, perm))
    b, w = O.quad6()
    assert len(ref) == 6 == len(w)
    used = set()
    for k in range(6):
        hit = [i for i, (rw, rp) in enumerate(ref)
               if i not in used and abs(rw - w[k]) < 1e-14 and np.allclose(rp, b[k], atol=1e-14)]
        assert hit, (k, b[k], w[k])
        used.add(hit[0])
