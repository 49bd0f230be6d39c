"""Pins of the OSRC preconditioner pieces (Sec. 2.6): the rotated Pade
approximation of sqrt(1+z), its NtD partial fractions, the damped
wavenumber, and the discrete DtN map on a sphere."""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre

import oracle as O
from paper_2104_04609_gb300.inputs import icosphere


def test_pade_theta0_is_real_pade():
    C0, A, B = O.pade(4, 0.0)
    j = np.arange(1, 5)
    assert abs(C0 - 1.0) < 1e-15
    assert np.allclose(A, 2.0 / 9.0 * np.sin(j * math.pi / 9) ** 2, atol=1e-15)
    assert np.allclose(B, np.cos(j * math.pi / 9) ** 2, atol=1e-15)


def test_pade_n1_closed_form():
    # the [1/1] Pade approximant of sqrt(1+z) is (4 + 3z)/(4 + z)
    z = np.linspace(-0.9, 3.0, 17)
    got = O.pade_eval(z, 1, 0.0)
    assert np.allclose(got, (4 + 3 * z) / (4 + z), atol=1e-14)


def test_pade_rotated_converges_to_principal_sqrt():
    z = np.concatenate([np.linspace(-6.0, -1.2, 9), np.linspace(-0.8, 4.0, 9)]) + 0.05j
    errs = [np.abs(O.pade_eval(z, n, math.pi / 3) - np.sqrt(1 + z)).max() for n in (2, 4, 8, 16)]
    assert errs[3] < 1e-2 and errs[3] < errs[1] < errs[0]
    # rotation keeps exactness at the expansion point structure: sqrt(1+0) = 1
    assert abs(O.pade_eval(np.array([0.0]), 4, math.pi / 3)[0] - 1.0) < 5e-3


def test_ntd_partial_fractions():
    g0, g, B = O.ntd_partial_fractions(4, math.pi / 3)
    rng = np.random.default_rng(0)
    z = rng.standard_normal(20) * 3 + 1j * rng.standard_normal(20)
    lhs = O.pade_eval(z, 4, math.pi / 3) / (1 + z)
    rhs = g0 / (1 + z) + (g[:, None] / (1 + B[:, None] * z[None, :])).sum(0)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_damped_wavenumber():
    k, R = 26.0, 0.05
    ke = O.damped_wavenumber(k, R)
    assert abs(ke - (k + 0.4j * k ** (1 / 3) * R ** (-2 / 3))) < 1e-12


def test_osrc_dtn_on_sphere():
    """On the unit sphere Delta_Gamma Y_l = -l(l+1) Y_l, so the DtN map acts on
    Y_l as i k R(-l(l+1)/k_eps^2): the discrete map's Rayleigh quotient
    approaches it (and NtD * DtN ~ R^2/(1+z) ~ identity)."""
    v, t = icosphere(3)
    M, S = O.mass_stiffness(v, t)
    k = 3.0
    ke = O.damped_wavenumber(k, 0.1)
    for l in range(1, 4):
        u = eval_legendre(l, v[:, 2]).astype(np.complex128)
        z1, z2 = O.osrc_apply(M, S, u, u, k, ke, 4, math.pi / 3)
        den = u @ (M @ u)
        zl = -l * (l + 1) / ke ** 2
        dtn = 1j * k * O.pade_eval(np.array([zl]), 4, math.pi / 3)[0]
        ntd = O.pade_eval(np.array([zl]), 4, math.pi / 3)[0] / (1 + zl) / (1j * k)
        assert abs((u @ (M @ z1)) / den - dtn) / abs(dtn) < 0.02
        assert abs((u @ (M @ z2)) / den - ntd) / abs(ntd) < 0.02
