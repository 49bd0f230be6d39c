"""Checks of the synthetic geometry generators: closed, consistently
oriented surfaces with the enclosed volume the construction fixes."""
import numpy as np
import pytest

import oracle as O
from paper_2104_04609_gb300.inputs import menger_sponge


def _volume(v, t):
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    return np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0


@pytest.mark.parametrize("level,sub", [(1, 1), (1, 2), (2, 1)])
def test_menger_sponge_closed_oriented(level, sub):
    v, t = menger_sponge(level, sub, edge=2.0)
    edges = {}
    for tri in t:
        for k in range(3):
            e = (tri[k], tri[(k + 1) % 3])
            assert e not in edges  # each directed edge once: consistent orientation
            edges[e] = 1
    assert all((b, a) in edges for a, b in edges)  # closed
    assert abs(_volume(v, t) - 8.0 * (20.0 / 27.0) ** level) < 1e-12


def test_menger_sponge_region():
    v, t = menger_sponge(1, 1, edge=2.0)
    solid = np.array([[-0.9, -0.9, -0.9], [0.0, -0.9, -0.9]])  # corner and edge cells
    tunnel = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.9]])       # removed centre column
    assert O.inside(v, t, solid).all() and not O.inside(v, t, tunnel).any()
