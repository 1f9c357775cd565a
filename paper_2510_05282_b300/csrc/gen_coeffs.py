"""Generate sh_coeffs.h: the constants of the Cartesian evaluation scheme.

Run from the repository root:  python paper_2510_05282_b300/csrc/gen_coeffs.py

Tables run to l = 16: the paper's formulas stop at l = 9, the recurrence
does not (the paper's conclusion names recurrences as the way past l = 9).

Scheme (normalised Cartesian coordinates xb, yb, zb, Sec. II Eq. 8):
  R_l^{+m} = S_lm * Qh_l^m(zb) * A_m,   R_l^{-m} = S_lm * Qh_l^m(zb) * B_m,
  R_l^0    = S_l0 * Qh_l^0(zb),
  A_m + i B_m = (xb + i yb)^m   (= sin^m(theta) e^{i m phi}),
  Qh_m^m = 1,  Qh_{m+1}^m = zb,  Qh_l^m = zb Qh_{l-1}^m - G_lm q Qh_{l-2}^m,
where q = xb^2 + yb^2 + zb^2 (= 1 on the sphere; the homogeneous form keeps
q so that rounding of the coordinates off the sphere costs only l ulps), and
  G_lm = (l+m-1)(l-m-1) / ((2l-1)(2l-3)),
  S_lm = K_lm * sigma_lm,
  K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) times sqrt(2) for m > 0 (Eq. 5-6).
Qh_l^m is d^m P_l / dx^m divided by sigma_lm, where sigma_mm = (2m-1)!! and
sigma_lm = (2l-1)/(l-m) sigma_{l-1,m}; this rescaling makes the leading
coefficient of the three-term recurrence 1.  All constants are computed in
exact rational arithmetic and 40-digit mpmath, then rounded once.
"""
import math
import os
from fractions import Fraction

import mpmath as mp

LMAX = 16
mp.mp.dps = 50


def sigma(l, m):
    s = Fraction(math.prod(range(1, 2 * m, 2)) if m > 0 else 1)
    for ll in range(m + 1, l + 1):
        s *= Fraction(2 * ll - 1, ll - m)
    return s


def G(l, m):
    return Fraction((l + m - 1) * (l - m - 1), (2 * l - 1) * (2 * l - 3))


def K(l, m):
    v = mp.sqrt(mp.mpf(2 * l + 1) / (4 * mp.pi) * mp.factorial(l - m) / mp.factorial(l + m))
    return v * mp.sqrt(2) if m > 0 else v


def S(l, m):
    s = sigma(l, m)
    return K(l, m) * mp.mpf(s.numerator) / s.denominator


def SC(l, m):
    """S_lm / sqrt2 for m > 0 (the complex harmonics, Y = (R + i R')/sqrt2), S_l0 for m = 0."""
    return S(l, m) / mp.sqrt(2) if m > 0 else S(l, m)


def fmt64(v):
    return mp.nstr(mp.mpf(v), 21, min_fixed=-1, max_fixed=-1)


def split_hi_lo(v):
    """float hi + float lo with hi = fl32(v), lo = fl32(v - hi)."""
    import numpy as np
    hi = np.float32(float(v))
    lo = np.float32(float(mp.mpf(v) - mp.mpf(float(hi))))
    return float(hi), float(lo)


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    lines = [
        "// Generated by gen_coeffs.py -- do not edit.",
        "// Constants of the Cartesian recurrence for the real spherical harmonics",
        "// (normalised Cartesian coordinates, Sec. II Eq. 8 and App. C of arXiv",
        "// 2510.05282); see gen_coeffs.py for the scheme and derivation.",
        "#pragma once",
        f"#define SHM_COEFF_LMAX {LMAX}",
        "",
        "// G[l][m] for l >= m + 2 (0 elsewhere)",
        f"__device__ constexpr double SHM_G[{LMAX + 1}][{LMAX + 1}] = {{",
    ]
    for l in range(LMAX + 1):
        row = []
        for m in range(LMAX + 1):
            row.append(fmt64(mp.mpf(G(l, m).numerator) / G(l, m).denominator) if l >= m + 2 else "0.0")
        lines.append("  {" + ", ".join(row) + "},")
    lines.append("};")
    lines.append("// S[l][m] for m <= l (0 elsewhere)")
    lines.append(f"__device__ constexpr double SHM_S[{LMAX + 1}][{LMAX + 1}] = {{")
    for l in range(LMAX + 1):
        lines.append("  {" + ", ".join(fmt64(S(l, m)) if m <= l else "0.0" for m in range(LMAX + 1)) + "},")
    lines.append("};")
    lines.append("// SC[l][m] = S[l][m] / sqrt2 for m > 0 (complex harmonics), S[l][0] for m = 0")
    lines.append(f"__device__ constexpr double SHM_SC[{LMAX + 1}][{LMAX + 1}] = {{")
    for l in range(LMAX + 1):
        lines.append("  {" + ", ".join(fmt64(SC(l, m)) if m <= l else "0.0" for m in range(LMAX + 1)) + "},")
    lines.append("};")
    # float hi/lo splits for the compensated FP32 path
    for name, fn in (("G", lambda l, m: mp.mpf(G(l, m).numerator) / G(l, m).denominator if l >= m + 2 else 0),
                     ("S", lambda l, m: S(l, m) if m <= l else 0),
                     ("SC", lambda l, m: SC(l, m) if m <= l else 0)):
        his, los = [], []
        for l in range(LMAX + 1):
            hr, lr = [], []
            for m in range(LMAX + 1):
                h, lo = split_hi_lo(fn(l, m))
                hr.append(repr(h) + "f")
                lr.append(repr(lo) + "f")
            his.append("  {" + ", ".join(hr) + "},")
            los.append("  {" + ", ".join(lr) + "},")
        lines.append(f"__device__ constexpr float SHM_{name}_HI[{LMAX + 1}][{LMAX + 1}] = {{")
        lines += his
        lines.append("};")
        lines.append(f"__device__ constexpr float SHM_{name}_LO[{LMAX + 1}][{LMAX + 1}] = {{")
        lines += los
        lines.append("};")
    nk = (LMAX + 1) ** 2
    lines.append("// l of the flat index k = l*l + l + m (a table, so a constant k folds at compile time)")
    lines.append(f"__device__ constexpr int SHM_L_OF_K[{nk}] = {{")
    ls = [str(int(math.isqrt(k))) for k in range(nk)]
    for i in range(0, nk, 25):
        lines.append("    " + ", ".join(ls[i:i + 25]) + ",")
    lines.append("};")
    with open(os.path.join(here, "sh_coeffs.h"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
