"""Second, independent evaluation of R_l^m used only to pin the oracle.

The explicit factorised polynomials of App. C (m <= 0, l <= 9, in normalised
Cartesian coordinates xb, yb, zb) and the m > 0 rotation rules of App. B,
restated in numpy.  p(a, b) = (a - b)(a + b) is the root-pair factor of
Eq. 16.  Three printed formulas are taken in a corrected reading, each
checked against the theta/phi definition:

* R_5^0: the two z-roots are sqrt((5 -+ 2 sqrt(10/7)) / 9) (the roots of
  63 z^4 - 70 z^2 + 15); the printed "/3" gives values off by O(1).
* R_8^{-1}: the Horner form is used; the printed factored form lacks an overall
  minus sign (its three p(root, z) factors flip the sign of the leading term).
* R_9^{-7}: the factored form is used; the first printed line lacks the yb
  factor.
"""
import math

import numpy as np

PI = math.pi
S2, S3, S5, S7 = math.sqrt(2), math.sqrt(3), math.sqrt(5), math.sqrt(7)


def p(a, b):
    return (a - b) * (a + b)


def sq(v):
    return math.sqrt(v)


def _neg_m_formulas(x, y, z):
    """dict (l, m) -> values for m <= 0."""
    R = {}
    R[0, 0] = np.full_like(z, 1.0 / sq(4 * PI))
    R[1, -1] = sq(3 / (4 * PI)) * y
    R[1, 0] = sq(3 / (4 * PI)) * z
    R[2, -2] = 0.5 * sq(15 / PI) * x * y
    R[2, -1] = 0.5 * sq(15 / PI) * y * z
    R[2, 0] = 0.25 * sq(5 / PI) * p(S3 * z, 1.0)
    R[3, -3] = (1 / 8) * sq(70 / PI) * y * p(S3 * x, y)
    R[3, -2] = 0.5 * sq(105 / PI) * x * y * z
    R[3, -1] = (1 / 8) * sq(42 / PI) * y * p(S5 * z, 1.0)
    R[3, 0] = 0.25 * sq(7 / PI) * p(S5 * z, S3) * z
    R[4, -4] = 0.75 * sq(35 / PI) * x * y * p(x, y)
    R[4, -3] = (3 / 8) * sq(70 / PI) * y * p(S3 * x, y) * z
    R[4, -2] = 0.75 * sq(5 / PI) * x * y * p(S7 * z, 1.0)
    R[4, -1] = (3 / 8) * sq(10 / PI) * y * z * p(S7 * z, S3)
    R[4, 0] = (105 / 16) * sq(1 / PI) * p(sq((3 + 2 * sq(6 / 5)) / 7), z) * p(sq((3 - 2 * sq(6 / 5)) / 7), z)
    R[5, -5] = (30 / 64) * sq(154 / PI) * y * p(sq(1 - 2 / S5) * y, x) * p(sq(1 + 2 / S5) * y, x)
    R[5, -4] = 0.75 * sq(385 / PI) * p(x, y) * y * z * x
    R[5, -3] = (1 / 32) * sq(770 / PI) * y * p(y, S3 * x) * p(1.0, 3 * z)
    R[5, -2] = 0.25 * sq(1155 / PI) * x * y * p(S3 * z, 1.0) * z
    R[5, -1] = (21 / 16) * sq(165 / PI) * y * p(sq((7 - 2 * S7) / 21), z) * p(sq((7 + 2 * S7) / 21), z)
    R[5, 0] = (63 / 16) * sq(11 / PI) * z * p(sq((5 - 2 * sq(10 / 7)) / 9), z) * p(sq((5 + 2 * sq(10 / 7)) / 9), z)
    R[6, -6] = (1 / 32) * sq(6006 / PI) * x * y * p(x, S3 * y) * p(S3 * x, y)
    R[6, -5] = (3 / 32) * sq(2002 / PI) * y * z * p(sq(5 - 2 * S5) * x, y) * p(sq(5 + 2 * S5) * x, y)
    R[6, -4] = (3 / 8) * sq(91 / PI) * x * y * p(x, y) * p(sq(11) * z, 1.0)
    R[6, -3] = (1 / 32) * sq(2730 / PI) * y * z * p(S3 * x, y) * p(sq(11) * z, S3)
    R[6, -2] = (33 / 32) * sq(2730 / PI) * x * y * p(sq((3 - 4 / S3) / 11), z) * p(sq((3 + 4 / S3) / 11), z)
    R[6, -1] = (33 / 16) * sq(273 / PI) * y * z * p(sq((15 - 2 * sq(15)) / 33), z) * p(sq((15 + 2 * sq(15)) / 33), z)
    z2 = z * z
    R[6, 0] = (1 / 32) * sq(13 / PI) * (z2 * ((231 * z2 - 315) * z2 + 105) - 5)
    hept = 7 * x**6 - 35 * x**4 * y**2 + 21 * x**2 * y**4 - y**6
    R[7, -7] = (3 / 64) * sq(715 / PI) * y * hept
    R[7, -6] = (3 / 32) * sq(10010 / PI) * x * y * z * p(x, S3 * y) * p(S3 * x, y)
    R[7, -5] = (3 / 64) * sq(385 / PI) * y * p(sq(13) * z, 1.0) * p(sq(5 - 2 * S5) * x, y) * p(sq(5 + 2 * S5) * x, y)
    R[7, -4] = (3 / 8) * sq(385 / PI) * x * y * z * p(x, y) * p(sq(13) * z, S3)
    R[7, -3] = (429 / 64) * sq(35 / PI) * y * p(S3 * x, y) * p(sq((33 - 2 * sq(165)) / 143), z) * p(sq((33 + 2 * sq(165)) / 143), z)
    R[7, -2] = (429 / 32) * sq(70 / PI) * x * y * z * p(sq((55 - 4 * sq(55)) / 143), z) * p(sq((55 + 4 * sq(55)) / 143), z)
    R[7, -1] = (1 / 64) * sq(105 / PI) * y * (z2 * ((429 * z2 - 495) * z2 + 135) - 5)
    R[7, 0] = (1 / 32) * sq(15 / PI) * z * (-35 + z2 * (315 + z2 * (-693 + 429 * z2)))
    R[8, -8] = (12 / 128) * sq(12155 / PI) * x * y * p(x, y) * p((1 + S2) * x, y) * p((1 - S2) * x, y)
    R[8, -7] = (3 / 64) * sq(12155 / PI) * y * z * hept
    R[8, -6] = (1 / 64) * sq(14586 / PI) * x * y * p(x, S3 * y) * p(S3 * x, y) * p(sq(15) * z, 1.0)
    R[8, -5] = (3 / 64) * sq(17017 / PI) * y * z * p(S5 * z, 1.0) * p(sq(5 + 2 * S5) * x, y) * p(sq(5 - 2 * S5) * x, y)
    R[8, -4] = (195 / 32) * sq(1309 / PI) * x * y * p(x, y) * p(sq((13 - 2 * sq(26)) / 65), z) * p(sq((13 + 2 * sq(26)) / 65), z)
    R[8, -3] = (39 / 64) * sq(19635 / PI) * y * z * p(S3 * x, y) * p(sq((1 - 2 / sq(13)) / 3), z) * p(sq((1 + 2 / sq(13)) / 3), z)
    R[8, -2] = (3 / 64) * sq(1190 / PI) * x * y * (z2 * ((143 * z2 - 143) * z2 + 33) - 1)
    R[8, -1] = (3 / 64) * sq(17 / PI) * y * z * (z2 * ((715 * z2 - 1001) * z2 + 385) - 35)
    R[8, 0] = (1 / 256) * sq(17 / PI) * ((z2 * ((6435 * z2 - 12012) * z2 + 6930) - 1260) * z2 + 35)
    R[9, -9] = (1 / 512) * sq(461890 / PI) * y * p(S3 * x, y) * (3 * x**6 - 27 * x**4 * y**2 + 33 * x**2 * y**4 - y**6)
    R[9, -8] = (3 / 32) * sq(230945 / PI) * x * y * z * p(x, y) * p((1 + S2) * x, y) * p((1 - S2) * x, y)
    R[9, -7] = ((3 / 512) * sq(27170 / PI) * y * p(1.0, sq(17) * z)
                * p(y, 0.481574618807528644332162353056970575219 * x)
                * p(y, 1.253960337662703837570910978336464443221 * x)
                * p(y, 4.381286267534823072404689085032695444150 * x))
    R[9, -6] = (1 / 64) * sq(81510 / PI) * x * y * z * p(x, S3 * y) * p(S3 * x, y) * p(sq(17) * z, S3)
    R[9, -5] = ((255 / 256) * sq(5434 / PI) * y * p(sq(5 - 2 * S5) * x, y) * p(sq(5 + 2 * S5) * x, y)
                * p(sq((15 - 2 * sq(35)) / 85), z) * p(sq((15 + 2 * sq(35)) / 85), z))
    R[9, -4] = (51 / 32) * sq(95095 / PI) * x * y * z * p(x, y) * p(sq((5 - 2 * S2) / 17), z) * p(sq((5 + 2 * S2) / 17), z)
    R[9, -3] = (1 / 256) * sq(43890 / PI) * y * p(S3 * x, y) * (z2 * ((221 * z2 - 195) * z2 + 39) - 1)
    R[9, -2] = -(3 / 64) * sq(2090 / PI) * x * y * z * ((z2 * (273 - 221 * z2) - 91) * z2 + 7)
    R[9, -1] = (3 / 256) * sq(95 / PI) * y * ((z2 * ((2431 * z2 - 4004) * z2 + 2002) - 308) * z2 + 7)
    R[9, 0] = (1 / 256) * sq(19 / PI) * z * ((z2 * ((12155 * z2 - 25740) * z2 + 18018) - 4620) * z2 + 315)
    return R


def real_sh_appc(xyz: np.ndarray, lmax: int = 9) -> np.ndarray:
    """[n, (lmax+1)^2] by App. C (m <= 0) and the App. B rotations (m > 0).
    Points must be nonzero; they are normalised here."""
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    r = np.linalg.norm(xyz, axis=1)
    x, y, z = (xyz[:, i] / r for i in range(3))
    out = np.zeros((xyz.shape[0], (lmax + 1) ** 2))
    base = _neg_m_formulas(x, y, z)
    # odd m = 2n+1: R_l^m(x, y, z) = (-1)^n R_l^{-m}(-y, x, z)
    rot90 = _neg_m_formulas(-y, x, z)
    # m = 2(2n+1): R_l^m(x, y, z) = (-1)^n R_l^{-m}((x - y)/sqrt2, (x + y)/sqrt2, z)
    rot45 = _neg_m_formulas((x - y) / S2, (x + y) / S2, z)
    # m = 4, 8: rotation by pi/(2m) with constant cos/sin
    rotm = {}
    for m in (4, 8):
        c, s = math.cos(PI / (2 * m)), math.sin(PI / (2 * m))
        rotm[m] = _neg_m_formulas(c * x - s * y, s * x + c * y, z)
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            k = l * l + l + m
            if m <= 0:
                out[:, k] = base[l, m]
            elif m % 2 == 1:
                n = (m - 1) // 2
                out[:, k] = (-1) ** n * rot90[l, -m]
            elif (m // 2) % 2 == 1:
                n = (m // 2 - 1) // 2
                out[:, k] = (-1) ** n * rot45[l, -m]
            else:
                out[:, k] = rotm[m][l, -m]
    return out
