"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module only *generates* inputs: surface meshes shaped like the paper's
workloads (spheres, ellipsoids, a bumpy elongated body standing in for the
tibia section of Sec. 3.6), incident-field parameters and request streams.
It contains none of the boundary-element arithmetic (no quadrature, no
kernels, no operators) so that the oracle and the GPU library can both use
it without sharing any of the method's code.

Meshes are returned as ``(verts, tris)`` with ``verts`` a float64 ``(n_v, 3)``
array and ``tris`` an int32 ``(n_t, 3)`` array whose vertex order is
counter-clockwise seen from outside (outward normals, Sec. 2.1).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "icosphere",
    "fibonacci_hull",
    "ellipsoid",
    "bumpy_ellipsoid",
    "plane_wave_dirs",
    "serving_requests",
    "orient_outward",
    "workload",
]


def _icosahedron():
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array(
        [
            [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
            [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
            [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
        ],
        dtype=np.float64,
    )
    f = np.array(
        [
            [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
            [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
            [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
            [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
        ],
        dtype=np.int64,
    )
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


def icosphere(level: int, radius: float = 1.0):
    """Icosahedron refined ``level`` times by midpoint subdivision, every new
    vertex projected onto the sphere. Level 3: 642 vertices / 1280 triangles;
    level 5: 10242 / 20480."""
    v, f = _icosahedron()
    verts = [tuple(p) for p in v]
    for _ in range(level):
        cache = {}
        new_f = []

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            idx = cache.get(key)
            if idx is None:
                p = (np.asarray(verts[a]) + np.asarray(verts[b])) * 0.5
                p /= np.linalg.norm(p)
                idx = len(verts)
                verts.append(tuple(p))
                cache[key] = idx
            return idx

        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new_f += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        f = np.asarray(new_f, dtype=np.int64)
    verts = np.asarray(verts, dtype=np.float64) * radius
    return verts, orient_outward(verts, f.astype(np.int32))


def orient_outward(verts, tris):
    """Flip triangles whose vertex order gives a normal pointing towards the
    centroid of the (star-shaped) body."""
    tris = np.array(tris, dtype=np.int32, copy=True)
    c = verts.mean(axis=0)
    p0, p1, p2 = (verts[tris[:, i]] for i in range(3))
    n = np.cross(p1 - p0, p2 - p0)
    cen = (p0 + p1 + p2) / 3.0 - c
    bad = np.einsum("ij,ij->i", n, cen) < 0
    tris[bad] = tris[bad][:, [0, 2, 1]]
    return tris


def fibonacci_hull(n: int):
    """``n`` Fibonacci-lattice points on the unit sphere joined by their convex
    hull: a closed genus-0 triangulation with 2n-4 triangles."""
    from scipy.spatial import ConvexHull

    i = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * i / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    golden = math.pi * (3.0 - math.sqrt(5.0))
    phi = golden * i
    pts = np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)
    hull = ConvexHull(pts)
    tris = orient_outward(pts, hull.simplices.astype(np.int32))
    return pts, tris


def ellipsoid(n_v: int, axes=(1.0, 0.7, 0.5)):
    """Fibonacci-hull sphere mesh scaled to the given semi-axes."""
    pts, tris = fibonacci_hull(n_v)
    return pts * np.asarray(axes, dtype=np.float64)[None, :], tris


def bumpy_ellipsoid(n_v: int, axes=(2.0, 1.0, 1.0), n_bumps: int = 32,
                    amplitude: float = 0.05, width: float = 0.2, seed: int = 3):
    """Ellipsoid with seeded radial Gaussian bumps: each unit-sphere point x is
    moved to x (1 + A sum_b exp(-|x - c_b|^2 / (2 w^2))) before scaling, with
    bump centres c_b uniform on the sphere."""
    pts, tris = fibonacci_hull(n_v)
    rng = np.random.default_rng(seed)
    c = rng.standard_normal((n_bumps, 3))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    d2 = ((pts[:, None, :] - c[None, :, :]) ** 2).sum(-1)
    bump = amplitude * np.exp(-d2 / (2.0 * width * width)).sum(1)
    pts = pts * (1.0 + bump)[:, None]
    return pts * np.asarray(axes, dtype=np.float64)[None, :], tris


def plane_wave_dirs(n: int, seed: int = 1):
    """``n`` unit directions uniform on the sphere (normalised Gaussians)."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def serving_requests(n: int = 1000, rate: float = 50.0, seed: int = 2):
    """Poisson stream of solve requests: arrival time, mesh size (log-uniform
    2k..40k vertices), ka in [5, 40], density ratio in [1, 2], wave-speed
    ratio in [0.4, 1.5], 1..16 plane-wave right-hand sides."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    for i in range(n):
        nv = int(round(math.exp(rng.uniform(math.log(2000), math.log(40000)))))
        shape = "sphere" if rng.uniform() < 0.5 else "ellipsoid"
        axes = (1.0, float(rng.uniform(0.5, 1.0)), float(rng.uniform(0.5, 1.0)))
        out.append(
            dict(
                t=float(t[i]), n_v=nv, shape=shape,
                axes=(1.0, 1.0, 1.0) if shape == "sphere" else axes,
                ka=float(rng.uniform(5.0, 40.0)),
                rho_ratio=float(rng.uniform(1.0, 2.0)),
                c_ratio=float(rng.uniform(0.4, 1.5)),
                nrhs=int(rng.integers(1, 17)),
                seed=int(rng.integers(0, 2**31 - 1)),
            )
        )
    return out


def menger_sponge(level: int = 2, sub: int = 1, edge: float = 2.0):
    """Surface of a level-``level`` Menger sponge (a cube of side ``edge``,
    centred at the origin, from which the middle cells are removed
    recursively: a cell of the 3^level grid is kept when no level has more
    than one of its three base-3 digits equal to 1).  Every boundary face of
    a kept cell is split into sub x sub squares on the global lattice and each
    square into two triangles, counter-clockwise seen from outside."""
    n = 3 ** level
    keep = np.ones((n, n, n), dtype=bool)
    idx = np.arange(n)
    for d in range(level):
        dig = (idx // 3 ** d) % 3 == 1
        ones = dig[:, None, None].astype(int) + dig[None, :, None] + dig[None, None, :]
        keep &= ones <= 1
    N = n * sub
    vid = {}
    verts, tris = [], []

    def vertex(p):
        if p not in vid:
            vid[p] = len(verts)
            verts.append(p)
        return vid[p]

    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        for cell in zip(*np.nonzero(keep)):
            for side in (0, 1):
                nb = list(cell)
                nb[a] += 1 if side else -1
                if 0 <= nb[a] < n and keep[tuple(nb)]:
                    continue
                base = [int(cell[0]) * sub, int(cell[1]) * sub, int(cell[2]) * sub]
                base[a] += sub if side else 0
                for u in range(sub):
                    for w in range(sub):
                        def corner(du, dw):
                            q = list(base)
                            q[b] += u + du
                            q[c] += w + dw
                            return vertex(tuple(q))
                        p00, p10, p11, p01 = corner(0, 0), corner(1, 0), corner(1, 1), corner(0, 1)
                        if side:  # outward normal +e_a: (e_b, e_c) right-handed
                            tris += [(p00, p10, p11), (p00, p11, p01)]
                        else:
                            tris += [(p00, p11, p10), (p00, p01, p11)]
    V = np.asarray(verts, dtype=np.float64) * (edge / N) - edge / 2.0
    return V, np.asarray(tris, dtype=np.int32)


def workload(name: str):
    """The named synthetic workloads: mesh + physical parameters.

    ``k_int = k_ext / c_ratio`` with ``c_ratio = c_int / c_ext``."""
    if name == "sphere642":
        v, t = icosphere(3)
        return dict(verts=v, tris=t, k_ext=2.0, k_int=3.0, rho_ratio=1.5,
                    dirs=np.array([[0.0, 0.0, 1.0]]))
    if name == "sphere10242":
        v, t = icosphere(5)
        return dict(verts=v, tris=t, k_ext=20.0, k_int=26.0, rho_ratio=1.5,
                    dirs=np.array([[0.0, 0.0, 1.0]]))
    if name == "ellipsoid8000":
        v, t = ellipsoid(8000)
        return dict(verts=v, tris=t, k_ext=15.0, k_int=15.0 * 3600.0 / 1500.0,
                    rho_ratio=1.9, dirs=plane_wave_dirs(128, seed=1))
    if name == "bumpy80000":
        v, t = bumpy_ellipsoid(80000)
        return dict(verts=v, tris=t, k_ext=60.0, k_int=60.0 * 3600.0 / 1500.0,
                    rho_ratio=1.9, src=np.array([[3.0, 0.0, 0.0]]))
    raise KeyError(name)
