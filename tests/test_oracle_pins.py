"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check is a printed value
(Tables II and III of App. D), an independent evaluation (the App. C closed
forms with the App. B rotations, a 40-digit mpmath evaluation of the explicit
Legendre sum, scipy's complex harmonics through Eq. 6), or an identity that
holds for the true functions (addition theorem, parity, orthonormality on an
exact quadrature, axis values, the r = 0 convention of Sec. II).
"""
import math
import os

import numpy as np
import pytest

from appc_formulas import real_sh_appc
from paper_2510_05282_b300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
LMAX = 9
L_OF_K = np.array([int(math.isqrt(k)) for k in range((LMAX + 1) ** 2)])
M_OF_K = np.array([k - L_OF_K[k] ** 2 - L_OF_K[k] for k in range((LMAX + 1) ** 2)])
NORM_BOUND = np.sqrt((2 * L_OF_K + 1) / (4 * np.pi))   # max |R_l^m| by the addition theorem


def normwise(a, b):
    """max over points of |a - b| / sqrt((2l+1)/4pi), per column."""
    return np.abs(a - b) / NORM_BOUND[: a.shape[1]]


def read_table(name):
    rows = []
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            l, m, a, b = line.split()
            rows.append((int(l), int(m), float(a), None if b == "-" else float(b)))
    return rows


@pytest.mark.parametrize("name,theta,phi", [
    # Table II caption
    ("table2_point1.txt", 2.12160245947564796, -1.82732370250979703),
    # Table III caption, decimal point of phi restored (see the fixture header)
    ("table3_point2.txt", 1.69050041976591414, 0.758228122208986166),
])
def test_printed_reference_values(oracle_mod, name, theta, phi):
    rows = read_table(name)
    assert len(rows) == 55
    R = oracle_mod.real_sh_angles([theta], [phi], LMAX)[0]
    # same point through the Cartesian interface, at an arbitrary radius
    xyz = 2.75 * np.array([[math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi), math.cos(theta)]])
    Rc = oracle_mod.real_sh(xyz, LMAX)[0]
    for l, m, cos_col, sin_col in rows:
        assert abs(R[l * l + l + m] - cos_col) <= 2e-15, (l, m)
        assert abs(Rc[l * l + l + m] - cos_col) <= 4e-15, (l, m)
        if m > 0:
            assert abs(R[l * l + l - m] - sin_col) <= 2e-15, (l, -m)
            assert abs(Rc[l * l + l - m] - sin_col) <= 4e-15, (l, -m)


def test_appendix_c_closed_forms(oracle_mod):
    pts = inputs.random_sphere_points(4000, stream="tests")
    err = normwise(oracle_mod.real_sh(pts, LMAX), real_sh_appc(pts))
    # the printed formulas in binary64 reach ~1.5e-14 at l = 9 near the poles
    assert err.max() <= 5e-14, err.max()


def test_appendix_c_closed_forms_near_poles(oracle_mod):
    g = inputs.rng("tests", 11)
    eps = 10.0 ** g.uniform(-9, -2, size=500)
    ang = g.uniform(0, 2 * np.pi, size=500)
    sgn = np.where(g.uniform(size=500) < 0.5, -1.0, 1.0)
    pts = np.stack([eps * np.cos(ang), eps * np.sin(ang), sgn * np.ones(500)], axis=1)
    err = normwise(oracle_mod.real_sh(pts, LMAX), real_sh_appc(pts))
    assert err.max() <= 5e-14, err.max()


def _legendre_mp(l, m, x, mp):
    """(1 - x^2)^(m/2) d^m/dx^m P_l(x) without the Condon-Shortley sign, from
    the explicit sum P_l(x) = 2^-l sum_k (-1)^k C(l,k) C(2l-2k,l) x^(l-2k)."""
    s = mp.mpf(0)
    for k in range(l // 2 + 1):
        e = l - 2 * k
        if e < m:
            continue
        c = mp.mpf((-1) ** k * math.comb(l, k) * math.comb(2 * l - 2 * k, l)) / mp.mpf(2) ** l
        s += c * mp.mpf(math.perm(e, m)) * x ** (e - m)
    return mp.power(1 - x * x, mp.mpf(m) / 2) * s


def test_against_40_digit_explicit_sum(oracle_mod):
    mp = pytest.importorskip("mpmath").mp
    mp.dps = 40
    g = inputs.rng("tests", 3)
    pts = np.concatenate([g.standard_normal((150, 3)), inputs.axis_points()[:12]])
    O = oracle_mod.real_sh(pts, LMAX)
    worst = 0.0
    for i, (x, y, z) in enumerate(pts):
        X, Y, Z = mp.mpf(x), mp.mpf(y), mp.mpf(z)
        r = mp.sqrt(X * X + Y * Y + Z * Z)
        ct = Z / r
        phi = mp.atan2(Y, X)
        for l in range(LMAX + 1):
            for m in range(0, l + 1):
                N = mp.sqrt(mp.mpf(2 * l + 1) / (4 * mp.pi) * mp.factorial(l - m) / mp.factorial(l + m))
                P = _legendre_mp(l, m, ct, mp)
                if m == 0:
                    vals = {0: N * P}
                else:
                    vals = {m: mp.sqrt(2) * N * P * mp.cos(m * phi), -m: mp.sqrt(2) * N * P * mp.sin(m * phi)}
                for mm, v in vals.items():
                    e = abs(float(v) - O[i, l * l + l + mm]) / NORM_BOUND[l * l + l + mm]
                    worst = max(worst, e)
    assert worst <= 1e-14, worst


def test_against_scipy_complex_harmonics(oracle_mod):
    special = pytest.importorskip("scipy.special")
    pts = inputs.random_sphere_points(500, stream="tests", with_axes=False)
    r = np.linalg.norm(pts, axis=1)
    theta = np.arccos(np.clip(pts[:, 2] / r, -1, 1))
    phi = np.arctan2(pts[:, 1], pts[:, 0])
    O = oracle_mod.real_sh(pts, LMAX)
    for l in range(LMAX + 1):
        for m in range(-l, l + 1):
            a = abs(m)
            Y = special.sph_harm_y(l, a, theta, phi)   # includes (-1)^m, as Eq. 5
            if m == 0:
                ref = Y.real
            elif m > 0:   # Eq. 6 with Y_l^{-m} = (-1)^m conj(Y_l^m):  (-1)^m sqrt2 Re Y_l^m
                ref = (-1) ** a * math.sqrt(2) * Y.real
            else:         # (-1)^m sqrt2 Im Y_l^{|m|}
                ref = (-1) ** a * math.sqrt(2) * Y.imag
            k = l * l + l + m
            assert np.max(np.abs(O[:, k] - ref)) / NORM_BOUND[k] <= 1e-13, (l, m)


def test_addition_theorem(oracle_mod):
    pts = np.concatenate([inputs.random_sphere_points(3000, stream="tests"), inputs.edge_points()[2:14]])
    R = oracle_mod.real_sh(pts, LMAX)
    for l in range(LMAX + 1):
        s = np.sum(R[:, l * l: (l + 1) ** 2] ** 2, axis=1)
        np.testing.assert_allclose(s, (2 * l + 1) / (4 * np.pi), rtol=2e-14, atol=0)


def test_parity_and_scale_invariance(oracle_mod):
    pts = inputs.random_sphere_points(2000, stream="tests")
    R = oracle_mod.real_sh(pts, LMAX)
    Rm = oracle_mod.real_sh(-pts, LMAX)
    sign = (-1.0) ** L_OF_K
    assert np.max(normwise(Rm, sign * R)) <= 1e-14
    # a power-of-two scale changes no rounding: bit-identical
    assert np.array_equal(oracle_mod.real_sh(pts * 8.0, LMAX), R)
    assert np.max(normwise(oracle_mod.real_sh(pts * 3.7, LMAX), R)) <= 1e-14


def test_orthonormality_on_exact_quadrature(oracle_mod):
    # Gauss-Legendre in cos(theta) (16 nodes) x 32 uniform phi integrates
    # products of degree <= 18 exactly.
    xg, wg = np.polynomial.legendre.leggauss(16)
    ph = 2 * np.pi * np.arange(32) / 32
    ct = np.repeat(xg, 32)
    st = np.sqrt(1 - ct * ct)
    p = np.tile(ph, 16)
    pts = np.stack([st * np.cos(p), st * np.sin(p), ct], axis=1)
    w = np.repeat(wg, 32) * (2 * np.pi / 32)
    R = oracle_mod.real_sh(pts, LMAX)
    G = (R * w[:, None]).T @ R
    assert np.max(np.abs(G - np.eye(G.shape[0]))) <= 1e-13


def test_special_values(oracle_mod):
    # l = 0 is constant and l = 1 is sqrt(3/4pi) (y, z, x)/r
    pts = inputs.random_sphere_points(200, stream="tests")
    R = oracle_mod.real_sh(pts, 1)
    r = np.linalg.norm(pts, axis=1)
    assert np.max(np.abs(R[:, 0] - 1 / math.sqrt(4 * math.pi))) <= 1e-16
    c = math.sqrt(3 / (4 * math.pi))
    for k, comp in ((1, 1), (2, 2), (3, 0)):
        assert np.max(np.abs(R[:, k] - c * pts[:, comp] / r)) <= 1e-15
    # on the z axis: R_l^0 = (+-1)^l sqrt((2l+1)/4pi), every m != 0 is 0 (the oracle
    # reaches the south pole through sin(pi) ~ 1.2e-16, hence a rounding-level bound
    # that grows with l: |dP_l^1/dx| = l(l+1)/2 at x = -1)
    for zs in (1.0, -1.0):
        R = oracle_mod.real_sh(np.array([[0.0, 0.0, 2.5 * zs]]), LMAX)[0]
        for k in range(100):
            if M_OF_K[k] == 0:
                assert abs(R[k] - zs ** L_OF_K[k] * NORM_BOUND[k]) <= 1e-15
            else:
                assert abs(R[k]) <= 1e-14 * NORM_BOUND[k]
    # on the +x axis (phi = 0): R_l^{m<0} = 0 and R_l^{m>0} = sqrt2 N_l^m P_l^m(0) with
    # P_l^m(0) = (-1)^((l-m)/2) (l+m-1)!! / (l-m)!! for l+m even, else 0 (no CS sign)
    def dfact(n):
        return 1 if n <= 0 else n * dfact(n - 2)
    R = oracle_mod.real_sh(np.array([[0.7, 0.0, 0.0]]), LMAX)[0]
    for l in range(LMAX + 1):
        for m in range(-l, l + 1):
            k = l * l + l + m
            a = abs(m)
            if m < 0:
                assert abs(R[k]) <= 1e-16
                continue
            P0 = 0.0 if (l + a) % 2 else (-1) ** ((l - a) // 2) * dfact(l + a - 1) / dfact(l - a)
            N = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - a) / math.factorial(l + a))
            ref = (math.sqrt(2) if m > 0 else 1.0) * N * P0
            assert abs(R[k] - ref) <= 2e-15, (l, m)


def test_origin_convention_and_nan(oracle_mod):
    R = oracle_mod.real_sh(np.array([[0.0, 0.0, 0.0], [-0.0, 0.0, -0.0]]), LMAX)
    for row in R:
        assert row[0] == 1 / math.sqrt(4 * math.pi)
        assert np.all(row[1:] == 0.0)
    R = oracle_mod.real_sh(np.array([[np.nan, 0.0, 1.0]]), 3)
    assert np.all(np.isnan(R[0, 1:]))


def test_rejects_bad_lmax(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.real_sh(np.ones((1, 3)), 17)
    with pytest.raises(ValueError):
        oracle_mod.real_sh(np.ones((1, 3)), -1)


@pytest.mark.parametrize("lmax", [0, 1, 2, 5, 9])
def test_prefix_property(oracle_mod, lmax):
    # a smaller lmax gives exactly the leading columns of lmax = 9
    pts = inputs.random_sphere_points(100, stream="tests")
    full = oracle_mod.real_sh(pts, LMAX)
    part = oracle_mod.real_sh(pts, lmax)
    assert np.array_equal(part, full[:, : (lmax + 1) ** 2])


def test_complex_harmonics_against_scipy_and_eq10(oracle_mod):
    special = pytest.importorskip("scipy.special")
    pts = inputs.random_sphere_points(800, stream="tests")
    r = np.linalg.norm(pts, axis=1)
    theta = np.arccos(np.clip(pts[:, 2] / r, -1, 1))
    phi = np.arctan2(pts[:, 1], pts[:, 0])
    Y = oracle_mod.complex_sh(pts, LMAX)
    for l in range(LMAX + 1):
        for m in range(-l, l + 1):
            ref = special.sph_harm_y(l, m, theta, phi)       # Condon-Shortley included, as Eq. 5
            k = l * l + l + m
            assert np.max(np.abs(Y[:, k] - ref)) <= 1e-13 * NORM_BOUND[k], (l, m)
            if m > 0:  # Eq. 10
                assert np.array_equal(Y[:, l * l + l - m], (-1) ** m * np.conj(Y[:, k]))
    # the addition theorem for |Y|^2 and the link to the real harmonics (Eq. 6)
    R = oracle_mod.real_sh(pts, LMAX)
    for l in range(LMAX + 1):
        np.testing.assert_allclose(np.sum(np.abs(Y[:, l * l:(l + 1) ** 2]) ** 2, axis=1),
                                   (2 * l + 1) / (4 * np.pi), rtol=2e-14)
        for m in range(1, l + 1):
            k = l * l + l + m
            re = (-1) ** m * np.sqrt(2) * Y[:, k].real
            im = (-1) ** m * np.sqrt(2) * Y[:, k].imag
            assert np.max(np.abs(re - R[:, k])) <= 1e-14 * NORM_BOUND[k]
            assert np.max(np.abs(im - R[:, l * l + l - m])) <= 1e-14 * NORM_BOUND[k]


# ---------------------------------------------------------------- beyond l = 9

def test_high_l_against_scipy_and_identities(oracle_mod):
    """l up to 16 (the recurrence has no l limit): scipy's complex harmonics
    through Eq. 6, the addition theorem and orthonormality on an exact
    24 x 48 Gauss-Legendre x uniform-phi quadrature (degree <= 47)."""
    special = pytest.importorskip("scipy.special")
    L = 16
    nb = np.sqrt((2 * np.array([int(math.isqrt(k)) for k in range((L + 1) ** 2)]) + 1) / (4 * np.pi))
    pts = inputs.random_sphere_points(300, stream="tests", with_axes=False)
    R = oracle_mod.real_sh(pts, L)
    r = np.linalg.norm(pts, axis=1)
    theta = np.arccos(np.clip(pts[:, 2] / r, -1, 1))
    phi = np.arctan2(pts[:, 1], pts[:, 0])
    for l in range(10, L + 1):
        for m in range(-l, l + 1):
            a = abs(m)
            Y = special.sph_harm_y(l, a, theta, phi)
            ref = Y.real if m == 0 else (-1) ** a * math.sqrt(2) * (Y.real if m > 0 else Y.imag)
            k = l * l + l + m
            assert np.max(np.abs(R[:, k] - ref)) <= 1e-13 * nb[k], (l, m)
        s = np.sum(R[:, l * l:(l + 1) ** 2] ** 2, axis=1)
        np.testing.assert_allclose(s, (2 * l + 1) / (4 * np.pi), rtol=4e-14)
    xg, wg = np.polynomial.legendre.leggauss(24)
    ph = 2 * np.pi * np.arange(48) / 48
    ct = np.repeat(xg, 48)
    st = np.sqrt(1 - ct * ct)
    p = np.tile(ph, 24)
    q = np.stack([st * np.cos(p), st * np.sin(p), ct], axis=1)
    w = np.repeat(wg, 48) * (2 * np.pi / 48)
    Rq = oracle_mod.real_sh(q, L)
    G = (Rq * w[:, None]).T @ Rq
    assert np.max(np.abs(G - np.eye(G.shape[0]))) <= 1e-12


def test_high_l_against_40_digit_explicit_sum(oracle_mod):
    mp = pytest.importorskip("mpmath").mp
    mp.dps = 40
    g = inputs.rng("tests", 4)
    pts = g.standard_normal((40, 3))
    L = 16
    O = oracle_mod.real_sh(pts, L)
    worst = 0.0
    for i, (x, y, z) in enumerate(pts):
        X, Y, Z = mp.mpf(x), mp.mpf(y), mp.mpf(z)
        rr = mp.sqrt(X * X + Y * Y + Z * Z)
        ct, phi = Z / rr, mp.atan2(Y, X)
        for l in (10, 13, 16):
            for m in range(0, l + 1):
                N = mp.sqrt(mp.mpf(2 * l + 1) / (4 * mp.pi) * mp.factorial(l - m) / mp.factorial(l + m))
                P = _legendre_mp(l, m, ct, mp)
                vals = {0: N * P} if m == 0 else {m: mp.sqrt(2) * N * P * mp.cos(m * phi),
                                                  -m: mp.sqrt(2) * N * P * mp.sin(m * phi)}
                for mm, v in vals.items():
                    worst = max(worst, abs(float(v) - O[i, l * l + l + mm]) / math.sqrt((2 * l + 1) / (4 * math.pi)))
    assert worst <= 4e-14, worst


def test_thread_count_resets_to_all_processors(oracle_mod):
    """nthreads = 0 means every processor, also right after a 1-thread call
    (the CPU baselines time both)."""
    import os
    assert oracle_mod.max_threads(1) == 1
    full = oracle_mod.max_threads(0)
    assert full >= 1 and full == oracle_mod.max_threads(0)
    if (os.cpu_count() or 1) > 1:
        assert full > 1
