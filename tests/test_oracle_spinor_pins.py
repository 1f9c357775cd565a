"""Pins of the oracle's spinor harmonics (Sec. II, Eq. 7) to sources other
than the oracle itself: Clebsch-Gordan coupling of Y_l with a spin-1/2
state (sympy's exact coefficients, scipy's harmonics), the closure relation
of each j-shell, orthonormality of the two-component functions on an exact
quadrature, and the textbook p_1/2 spinor.
"""
import math

import numpy as np
import pytest

from paper_2510_05282_b300 import inputs

LMAX = 9


def angles(pts):
    rho = np.hypot(pts[:, 0], pts[:, 1])
    return np.arctan2(rho, pts[:, 2]), np.arctan2(pts[:, 1], pts[:, 0])


def shell_bound(l):
    return math.sqrt((2 * l + 1) / (4 * math.pi))


def test_layout_and_count(oracle_mod):
    pts = inputs.random_sphere_points(7, stream="tests", with_axes=False)
    S = oracle_mod.spinor_sh(pts, 4)
    assert S.shape == (7, 50, 2)
    seen = set()
    for l in range(5):
        for s in ((1,) if l == 0 else (-1, 1)):
            tj = 2 * l + s
            for tmj in range(-tj, tj + 1, 2):
                seen.add(oracle_mod.spinor_index(l, s, tmj))
    assert seen == set(range(50))


def test_clebsch_gordan_coupling(oracle_mod):
    """S_{l j m_j} = sum_sigma <l, m_j - sigma; 1/2, sigma | j m_j> Y_l^{m_j - sigma} chi_sigma,
    upper component sigma = +1/2, lower sigma = -1/2 (Condon-Shortley phases)."""
    sympy = pytest.importorskip("sympy")
    special = pytest.importorskip("scipy.special")
    from sympy.physics.quantum.cg import CG
    half = sympy.Rational(1, 2)
    pts = np.concatenate([inputs.random_sphere_points(200, stream="tests", with_axes=False),
                          inputs.edge_points()[:12]])
    pts = pts[np.linalg.norm(pts, axis=1) > 0]
    th, ph = angles(pts)
    S = oracle_mod.spinor_sh(pts, LMAX)
    for l in range(LMAX + 1):
        for s in ((1,) if l == 0 else (-1, 1)):
            tj = 2 * l + s
            for tmj in range(-tj, tj + 1, 2):
                q = oracle_mod.spinor_index(l, s, tmj)
                for c, tsig in ((0, 1), (1, -1)):
                    m = (tmj - tsig) // 2
                    if abs(m) > l:
                        ref = np.zeros(len(pts), dtype=complex)
                    else:
                        cg = float(CG(l, m, half, sympy.Rational(tsig, 2), sympy.Rational(tj, 2),
                                      sympy.Rational(tmj, 2)).doit())
                        ref = cg * special.sph_harm_y(l, m, th, ph)
                    err = np.max(np.abs(S[:, q, c] - ref))
                    assert err <= 1e-13 * shell_bound(l), (l, s, tmj, c, err)


def test_p_one_half_textbook_form(oracle_mod):
    """l = 1, j = 1/2, m_j = +1/2: (-sqrt(1/3) Y_1^0, sqrt(2/3) Y_1^1); Y_1^0 and
    Y_1^1 written out: sqrt(3/4pi) z/r and -sqrt(3/8pi) (x + i y)/r."""
    pts = inputs.random_sphere_points(100, stream="tests", with_axes=False)
    r = np.linalg.norm(pts, axis=1)
    x, y, z = (pts / r[:, None]).T
    Y10 = math.sqrt(3 / (4 * math.pi)) * z
    Y11 = -math.sqrt(3 / (8 * math.pi)) * (x + 1j * y)
    S = oracle_mod.spinor_sh(pts, 1)
    q = oracle_mod.spinor_index(1, -1, 1)
    np.testing.assert_allclose(S[:, q, 0], -math.sqrt(1 / 3) * Y10, atol=1e-15)
    np.testing.assert_allclose(S[:, q, 1], math.sqrt(2 / 3) * Y11, atol=1e-15)
    # s_1/2 (l = 0, j = 1/2): spin up and down times Y_0^0
    c = 1 / math.sqrt(4 * math.pi)
    np.testing.assert_allclose(S[:, oracle_mod.spinor_index(0, 1, 1)], np.array([[c, 0]] * 100), atol=1e-16)
    np.testing.assert_allclose(S[:, oracle_mod.spinor_index(0, 1, -1)], np.array([[0, c]] * 100), atol=1e-16)


def test_closure_of_each_j_shell(oracle_mod):
    """sum over m_j of S S^dagger = (2j+1)/(8 pi) times the 2 x 2 identity."""
    pts = inputs.random_sphere_points(300, stream="tests", with_axes=False)
    S = oracle_mod.spinor_sh(pts, LMAX)
    for l in range(LMAX + 1):
        for s in ((1,) if l == 0 else (-1, 1)):
            tj = 2 * l + s
            qs = [oracle_mod.spinor_index(l, s, t) for t in range(-tj, tj + 1, 2)]
            block = S[:, qs, :]                                   # [n, 2j+1, 2]
            M = np.einsum("nqa,nqb->nab", block, block.conj())
            ref = (tj + 1) / (8 * math.pi) * np.eye(2)
            assert np.max(np.abs(M - ref)) <= 1e-14 * (tj + 1), (l, s)


def test_orthonormality_on_exact_quadrature(oracle_mod):
    """<S_a, S_b> = sum_c int S_a^c* S_b^c dOmega = delta_ab; 12 x 24
    Gauss-Legendre x uniform-phi points integrate degree <= 2 lmax exactly."""
    L = 9
    xg, wg = np.polynomial.legendre.leggauss(12)
    ph = 2 * np.pi * np.arange(24) / 24
    ct = np.repeat(xg, 24)
    st = np.sqrt(1 - ct * ct)
    p = np.tile(ph, 12)
    q = np.stack([st * np.cos(p), st * np.sin(p), ct], axis=1)
    w = np.repeat(wg, 24) * (2 * np.pi / 24)
    S = oracle_mod.spinor_sh(q, L).reshape(len(q), -1)        # [n, 2 * nspinors]
    n = S.shape[1] // 2
    G = np.zeros((n, n), dtype=complex)
    for c in range(2):
        Sc = S[:, c::2]
        G += (Sc.conj() * w[:, None]).T @ Sc
    assert np.max(np.abs(G - np.eye(n))) <= 1e-13


def test_origin_keeps_only_l0(oracle_mod):
    S = oracle_mod.spinor_sh(np.zeros((2, 3)), 3)
    c = 1 / math.sqrt(4 * math.pi)
    ref = np.zeros((2, 32, 2), dtype=complex)
    ref[:, 0, 1] = c
    ref[:, 1, 0] = c
    assert np.array_equal(S, ref)
