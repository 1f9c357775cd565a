"""Pins of the projector oracle (grid index -> minimum image -> log-grid cubic
Lagrange interpolation of f_{s,l} -> times R_l^m).

The independent side here is a brute-force numpy/scipy restatement: numpy
minimum image, numpy.polyfit through the four table nodes for the
interpolation, and scipy's complex harmonics through Eq. 6 for the angular
part; plus exactness of 4-point Lagrange on cubic data and invariance under
lattice translations of the atoms.
"""
import math

import numpy as np
import pytest

from paper_2510_05282_b300 import inputs


def small_problem(extra=0, **kw):
    args = dict(n_atoms=5, box=6.0, h=0.25, rc_range=(1.0, 2.0), n_species=3,
                lmax_choices=(2, 3, 4), n_rad=200, r_min=1e-3, r_max=3.0, extra=extra)
    args.update(kw)
    return inputs.projector_problem(**args)


def real_sh_scipy(d, lmax):
    special = pytest.importorskip("scipy.special")
    r = np.linalg.norm(d, axis=1)
    theta = np.arccos(np.clip(d[:, 2] / r, -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    out = np.zeros((d.shape[0], (lmax + 1) ** 2))
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            Y = special.sph_harm_y(l, abs(m), theta, phi)
            s = (-1) ** abs(m) * math.sqrt(2)
            out[:, l * l + l + m] = Y.real if m == 0 else (s * Y.real if m > 0 else s * Y.imag)
    return out


def brute_force(prob):
    out = np.zeros(prob.n_values)
    ng = prob.ng
    for a in range(prob.n_atoms):
        s = prob.atom_species[a]
        lmax = int(prob.species_lmax[s])
        idx = prob.point_index[prob.point_offsets[a]:prob.point_offsets[a + 1]].astype(np.int64)
        gi, gj, gk = idx // (ng * ng), (idx // ng) % ng, idx % ng
        d = np.stack([gi, gj, gk], axis=1) * prob.h - prob.atom_pos[a]
        d -= prob.box * np.round(d / prob.box)
        r = np.linalg.norm(d, axis=1)
        t = np.clip(np.log(r / prob.r_min) / prob.dlog, 0, prob.n_rad - 1)
        Y = real_sh_scipy(d, lmax)
        L2 = (lmax + 1) ** 2
        block = np.zeros((idx.shape[0], L2))
        for l in range(lmax + 1):
            F = prob.radial[s, l]
            f = np.empty(idx.shape[0])
            for q in range(idx.shape[0]):
                i0 = min(max(int(math.floor(t[q])) - 1, 0), prob.n_rad - 4)
                nodes = np.arange(i0, i0 + 4, dtype=np.float64)
                coef = np.polyfit(nodes - i0, F[i0:i0 + 4], 3)
                f[q] = np.polyval(coef, t[q] - i0)
            block[:, l * l:(l + 1) ** 2] = f[:, None] * Y[:, l * l:(l + 1) ** 2]
        out[prob.out_offsets[a]:prob.out_offsets[a + 1]] = block.reshape(-1)
    return out


def test_problem_layout():
    prob = small_problem()
    assert prob.point_offsets[0] == 0 and prob.out_offsets[0] == 0
    n = np.diff(prob.point_offsets)
    L2 = (prob.atom_lmax().astype(np.int64) + 1) ** 2
    assert np.array_equal(np.diff(prob.out_offsets), n * L2)
    assert prob.point_index.min() >= 0 and prob.point_index.max() < prob.ng ** 3


def test_projector_oracle_vs_brute_force(oracle_mod):
    prob = small_problem()
    O = oracle_mod.projectors(prob)
    B = brute_force(prob)
    scale = np.abs(prob.radial).max()
    assert np.max(np.abs(O - B)) <= 1e-12 * scale


def test_lagrange_exact_on_cubic_tables(oracle_mod):
    prob = small_problem(extra=1)
    i = np.arange(prob.n_rad, dtype=np.float64)
    # f_{s,l} tabulated as a cubic in the table index is reproduced exactly
    # (up to rounding) by 4-point Lagrange interpolation
    cub = 1.0 + 0.01 * i - 2e-5 * i * i + 3e-8 * i ** 3
    prob.radial[:] = cub
    O = oracle_mod.projectors(prob)
    ng = prob.ng
    for a in range(prob.n_atoms):
        lmax = int(prob.atom_lmax()[a])
        L2 = (lmax + 1) ** 2
        idx = prob.point_index[prob.point_offsets[a]:prob.point_offsets[a + 1]].astype(np.int64)
        d = np.stack([idx // (ng * ng), (idx // ng) % ng, idx % ng], axis=1) * prob.h - prob.atom_pos[a]
        d -= prob.box * np.round(d / prob.box)
        r = np.linalg.norm(d, axis=1)
        t = np.clip(np.log(r / prob.r_min) / prob.dlog, 0, prob.n_rad - 1)
        f = 1.0 + 0.01 * t - 2e-5 * t * t + 3e-8 * t ** 3
        Y = oracle_mod.real_sh(d, lmax)
        ref = (f[:, None] * Y).reshape(-1)
        got = O[prob.out_offsets[a]:prob.out_offsets[a + 1]]
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.abs(cub).max(), a
        assert got.shape[0] == idx.shape[0] * L2


def test_lattice_translation_invariance(oracle_mod):
    prob = small_problem(extra=2)
    O = oracle_mod.projectors(prob)
    shift = np.array([1, -2, 3])[None, :] * prob.box
    prob.atom_pos = prob.atom_pos + shift
    O2 = oracle_mod.projectors(prob)
    assert np.max(np.abs(O - O2)) <= 1e-12 * np.abs(prob.radial).max()


def test_interpolation_tracks_analytic_radial(oracle_mod):
    # with l = 0 only, value * sqrt(4 pi) is the interpolated radial function;
    # against f evaluated analytically it is accurate to the log-grid step
    g = inputs.rng("tests", 21)
    prob = small_problem(extra=3, lmax_choices=(0,), n_rad=2000, r_min=1e-4, r_max=6.0)
    tab, dlog, a, alpha = inputs.radial_tables(g, prob.radial.shape[0], 1, 2000, 1e-4, 6.0)
    prob.radial = tab
    prob.dlog = dlog
    O = oracle_mod.projectors(prob)
    ng = prob.ng
    for at in range(prob.n_atoms):
        s = prob.atom_species[at]
        idx = prob.point_index[prob.point_offsets[at]:prob.point_offsets[at + 1]].astype(np.int64)
        d = np.stack([idx // (ng * ng), (idx // ng) % ng, idx % ng], axis=1) * prob.h - prob.atom_pos[at]
        d -= prob.box * np.round(d / prob.box)
        r = np.linalg.norm(d, axis=1)
        f = (a[s, 0, 0] + a[s, 0, 1] * r + a[s, 0, 2] * r * r) * np.exp(-alpha[s, 0] * r * r)
        got = O[prob.out_offsets[at]:prob.out_offsets[at + 1]] * math.sqrt(4 * math.pi)
        assert np.max(np.abs(got - f)) <= 1e-8 * np.abs(tab[s, 0]).max()
