"""Seeded synthetic inputs shared by the tests, the oracle checks and bench.py.

This module holds input generation only (point sets, grids, atom layouts,
radial tables, request streams).  It contains none of the harmonic or
projector arithmetic: that lives in the CUDA library on one side and in the
oracle on the other.

All generators are seeded numpy PCG64 streams derived from BASE_SEED, one
stream per workload, so every run and every machine sees the same inputs.

Workloads (the paper measures on synthetic random points, Sec. IV, and
motivates the method by DFT projector grids, Sec. I; no public dataset is
involved):

* ``random_sphere_points``  directions uniform on the unit sphere, radii
  log-uniform in [1e-3, 10] bohr, plus 64 points on the +-x/+-y/+-z axes.
* ``dft_grid_points``       a uniform cubic grid of spacing 0.3 bohr centred on
  an atom displaced by a seeded offset in [0, 0.3)^3 (no point at r = 0).
* ``projector_problem``     atoms in a periodic box with per-atom spheres,
  per-species lmax and tabulated radial functions.
* ``serving_requests`` and ``counter_points``  the request stream of the
  serving workload and the counter-based point generator its requests use.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 20251005

# one independent stream per workload
_STREAM = {"sphere": 1, "grid": 2, "sphere32": 3, "projectors": 4, "serving": 5, "tests": 6}


def rng(stream: str | int, extra: int = 0) -> np.random.Generator:
    key = _STREAM[stream] if isinstance(stream, str) else int(stream)
    return np.random.Generator(np.random.PCG64([BASE_SEED, key, int(extra)]))


# --------------------------------------------------------------------------- points

def axis_points() -> np.ndarray:
    """64 special points: +-x, +-y, +-z at 10 radii 10^(-3 + 4 (k + 1/2) / 10),
    plus +-z at the end radii 1e-3 and 10 bohr."""
    radii = 10.0 ** (-3.0 + 4.0 * (np.arange(10) + 0.5) / 10.0)
    dirs = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=np.float64)
    pts = [d * r for r in radii for d in dirs]
    for r in (1e-3, 10.0):
        pts.append(np.array([0.0, 0.0, r]))
        pts.append(np.array([0.0, 0.0, -r]))
    return np.asarray(pts, dtype=np.float64)


def random_sphere_points(n: int, stream: str = "sphere", with_axes: bool = True,
                         r_lo: float = 1e-3, r_hi: float = 10.0) -> np.ndarray:
    """[n (+64), 3] float64: directions = normalised N(0,1)^3, radii log-uniform."""
    g = rng(stream, n)
    v = g.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    r = np.exp(g.uniform(math.log(r_lo), math.log(r_hi), size=(n, 1)))
    pts = v * r
    if with_axes:
        pts = np.concatenate([pts, axis_points()], axis=0)
    return np.ascontiguousarray(pts)


def dft_grid_points(n_side: int = 192, spacing: float = 0.3, stream: str = "grid") -> np.ndarray:
    """[n_side^3, 3] float64: (i - n/2, j - n/2, k - n/2) * spacing - R, R ~ U[0, spacing)^3,
    row order i-major (i, j, k)."""
    g = rng(stream, n_side)
    R = g.uniform(0.0, spacing, size=3)
    idx = (np.arange(n_side, dtype=np.float64) - n_side // 2) * spacing
    X = idx[:, None, None] - R[0]
    Y = idx[None, :, None] - R[1]
    Z = idx[None, None, :] - R[2]
    pts = np.empty((n_side, n_side, n_side, 3), dtype=np.float64)
    pts[..., 0] = X
    pts[..., 1] = Y
    pts[..., 2] = Z
    return pts.reshape(-1, 3)


def edge_points() -> np.ndarray:
    """Degenerate and awkward inputs: r = 0, poles, axes, diagonals, tiny and
    huge radii, points 1e-9 off the poles, negative zeros."""
    base = [
        [0.0, 0.0, 0.0], [-0.0, 0.0, -0.0],
        [0.0, 0.0, 1.0], [0.0, 0.0, -1.0], [1.0, 0.0, 0.0], [-1.0, 0.0, 0.0],
        [0.0, 1.0, 0.0], [0.0, -1.0, 0.0], [1.0, 1.0, 1.0], [-1.0, 1.0, -1.0],
        [1e-9, 0.0, 1.0], [0.0, -1e-9, -1.0], [1e-9, 1e-9, 1.0], [3e-8, -2e-8, -1.0],
        [1e-12, 2e-12, -3e-12], [1e-30, -1e-30, 1e-30], [1e30, 2e30, -3e30],
        [0.3, -0.4, 0.5], [1e-3, 0.0, 0.0], [0.0, 0.0, 1e-3], [-2.5, 1e-300, 0.0],
    ]
    return np.asarray(base, dtype=np.float64)


# --------------------------------------------------------------------------- projectors

@dataclasses.dataclass
class ProjectorProblem:
    """Atoms in a cubic periodic box with a real-space grid of ng^3 points of
    spacing h (box = ng * h).  Atom a has species atom_species[a]; species s has
    angular cutoff species_lmax[s] and radial functions radial[s, l, :]
    tabulated at r_i = r_min * exp(i * dlog), i < n_rad.  point_index lists the
    linear grid indices ((i*ng + j)*ng + k) of every atom's sphere points, atom
    by atom (CSR by point_offsets); out_offsets[a] is where atom a's
    [n_a, (lmax_a+1)^2] block starts in the flat output."""
    atom_pos: np.ndarray        # [A, 3] float64
    atom_species: np.ndarray    # [A] int32
    atom_rc: np.ndarray         # [A] float64 sphere radii
    species_lmax: np.ndarray    # [S] int32
    radial: np.ndarray          # [S, lstride, n_rad] float64
    r_min: float
    dlog: float
    box: float
    ng: int
    h: float
    point_offsets: np.ndarray   # [A+1] int64
    point_index: np.ndarray     # [P] int32
    out_offsets: np.ndarray     # [A+1] int64

    @property
    def n_atoms(self) -> int:
        return int(self.atom_pos.shape[0])

    @property
    def n_points(self) -> int:
        return int(self.point_offsets[-1])

    @property
    def n_values(self) -> int:
        return int(self.out_offsets[-1])

    @property
    def n_rad(self) -> int:
        return int(self.radial.shape[2])

    def atom_lmax(self) -> np.ndarray:
        return self.species_lmax[self.atom_species]


def radial_tables(g: np.random.Generator, n_species: int, lstride: int, n_rad: int,
                  r_min: float, r_max: float):
    """f_{s,l}(r) = r^l (a0 + a1 r + a2 r^2) exp(-alpha r^2), a ~ N(0,1),
    alpha ~ U[0.3, 1.5], tabulated on the log grid r_i = r_min exp(i dlog)."""
    dlog = math.log(r_max / r_min) / (n_rad - 1)
    r = r_min * np.exp(dlog * np.arange(n_rad))
    a = g.standard_normal((n_species, lstride, 3))
    alpha = g.uniform(0.3, 1.5, size=(n_species, lstride))
    tab = np.empty((n_species, lstride, n_rad), dtype=np.float64)
    for s in range(n_species):
        for l in range(lstride):
            tab[s, l] = r ** l * (a[s, l, 0] + a[s, l, 1] * r + a[s, l, 2] * r * r) * np.exp(-alpha[s, l] * r * r)
    return tab, dlog, a, alpha


def sphere_lists(atom_pos: np.ndarray, atom_rc: np.ndarray, ng: int, h: float, box: float):
    """Per-atom grid points within rc of the atom (minimum image), in
    lexicographic (i, j, k) order over the atom's bounding box."""
    offsets = [0]
    chunks = []
    for a in range(atom_pos.shape[0]):
        p, rc = atom_pos[a], atom_rc[a]
        lo = np.ceil((p - rc) / h).astype(np.int64)
        hi = np.floor((p + rc) / h).astype(np.int64)
        ii = np.arange(lo[0], hi[0] + 1)
        jj = np.arange(lo[1], hi[1] + 1)
        kk = np.arange(lo[2], hi[2] + 1)
        dx = (ii * h - p[0])[:, None, None]
        dy = (jj * h - p[1])[None, :, None]
        dz = (kk * h - p[2])[None, None, :]
        inside = dx * dx + dy * dy + dz * dz <= rc * rc
        I, J, K = np.nonzero(inside)
        gi = np.mod(ii[I], ng)
        gj = np.mod(jj[J], ng)
        gk = np.mod(kk[K], ng)
        lin = (gi * ng + gj) * ng + gk
        chunks.append(lin.astype(np.int32))
        offsets.append(offsets[-1] + lin.shape[0])
    return np.asarray(offsets, dtype=np.int64), np.concatenate(chunks) if chunks else np.zeros(0, np.int32)


def projector_problem(n_atoms: int = 512, box: float = 40.0, h: float = 0.2,
                      rc_range=(2.0, 5.0), n_species: int = 8, lmax_choices=(2, 3, 4),
                      n_rad: int = 2000, r_min: float = 1e-4, r_max: float = 6.0,
                      stream: str = "projectors", extra: int = 0) -> ProjectorProblem:
    """The fused-projector workload: by default 512 atoms at seeded positions in a
    40 bohr periodic box, grid spacing 0.2 bohr (200^3 grid), sphere radii
    U[2, 5] bohr, 8 species with lmax drawn from {2, 3, 4}, radial functions on
    a 2000-point log grid from 1e-4 to 6 bohr."""
    g = rng(stream, extra * 1000003 + n_atoms)
    ng = int(round(box / h))
    if abs(ng * h - box) > 1e-9 * box:
        raise ValueError("box must be a whole number of grid spacings")
    if rc_range[1] >= box / 2:
        raise ValueError("sphere radius must stay below half the box (minimum image)")
    atom_pos = g.uniform(0.0, box, size=(n_atoms, 3))
    species_lmax = g.choice(np.asarray(lmax_choices, dtype=np.int32), size=n_species).astype(np.int32)
    atom_species = g.integers(0, n_species, size=n_atoms).astype(np.int32)
    atom_rc = g.uniform(rc_range[0], rc_range[1], size=n_atoms)
    lstride = int(max(lmax_choices)) + 1
    radial, dlog, _, _ = radial_tables(g, n_species, lstride, n_rad, r_min, r_max)
    point_offsets, point_index = sphere_lists(atom_pos, atom_rc, ng, h, box)
    nh = (species_lmax[atom_species].astype(np.int64) + 1) ** 2
    counts = np.diff(point_offsets)
    out_offsets = np.concatenate([[0], np.cumsum(counts * nh)]).astype(np.int64)
    return ProjectorProblem(atom_pos=atom_pos, atom_species=atom_species, atom_rc=atom_rc,
                            species_lmax=species_lmax, radial=radial, r_min=r_min, dlog=dlog,
                            box=box, ng=ng, h=h, point_offsets=point_offsets,
                            point_index=point_index, out_offsets=out_offsets)


# --------------------------------------------------------------------------- serving

MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter: np.ndarray) -> np.ndarray:
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) used as a counter-based
    generator: word(seed, c) = mix(seed + (c + 1) * GAMMA) with GAMMA the 64-bit
    golden-ratio increment and mix the published 30/27/31 xor-shift multiply
    finaliser."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counter.astype(np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def counter_points(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Points start..start+n-1 of the serving request with this seed, [n, 3] float64.

    Point i uses the four words c = 4i .. 4i+3 of splitmix64(seed, c) and only
    correctly rounded IEEE +, -, * on doubles assembled from bits, so any IEEE
    binary64 implementation reproduces it bit for bit:
      s = v(w0) - 3, t = v(w1) - 3, v(w) = double with bits (w >> 12) | 0x4000000000000000;
      direction (2s (1 - t^2), 2s 2t, (1 - s^2)(1 + t^2)) (length (1 + s^2)(1 + t^2)),
      x negated when bit 0 of w3 is 1, z when bit 1 is;
      radius = double with bits ((e + 1023) << 52) | (w2 >> 12), e = -10 + ((w3 >> 32) mod 14);
      point = direction * radius.
    """
    i = np.arange(start, start + n, dtype=np.uint64)
    w0 = splitmix64(seed, np.uint64(4) * i)
    w1 = splitmix64(seed, np.uint64(4) * i + np.uint64(1))
    w2 = splitmix64(seed, np.uint64(4) * i + np.uint64(2))
    w3 = splitmix64(seed, np.uint64(4) * i + np.uint64(3))
    hi = np.uint64(0x4000000000000000)
    s = ((w0 >> np.uint64(12)) | hi).view(np.float64) - 3.0
    t = ((w1 >> np.uint64(12)) | hi).view(np.float64) - 3.0
    s2, t2 = s * s, t * t
    s_2, t_2 = s + s, t + t
    dx = s_2 * (1.0 - t2)
    dy = s_2 * t_2
    dz = (1.0 - s2) * (1.0 + t2)
    dx = np.where((w3 & np.uint64(1)) == np.uint64(1), -dx, dx)
    dz = np.where((w3 & np.uint64(2)) == np.uint64(2), -dz, dz)
    e = (w3 >> np.uint64(32)) % np.uint64(14)
    radius = (((e + np.uint64(1013)) << np.uint64(52)) | (w2 >> np.uint64(12))).view(np.float64)
    pts = np.empty((n, 3), dtype=np.float64)
    pts[:, 0] = dx * radius
    pts[:, 1] = dy * radius
    pts[:, 2] = dz * radius
    return pts


@dataclasses.dataclass
class RequestSpec:
    arrival_s: float
    n: int
    lmax: int
    dtype: str      # "f32" or "f64"
    seed: int


def serving_requests(rate_per_s: float, duration_s: float, n_lo: int = 1000, n_hi: int = 4_000_000,
                     lmax_hi: int = 9, extra: int = 0) -> list[RequestSpec]:
    """Poisson arrivals at ``rate_per_s`` for ``duration_s`` seconds; sizes
    log-uniform in [n_lo, n_hi], lmax uniform in 0..lmax_hi, dtype 50/50."""
    g = rng("serving", extra * 7919 + int(rate_per_s))
    out: list[RequestSpec] = []
    t = 0.0
    while True:
        t += g.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            break
        n = int(round(math.exp(g.uniform(math.log(n_lo), math.log(n_hi)))))
        out.append(RequestSpec(arrival_s=t, n=n, lmax=int(g.integers(0, lmax_hi + 1)),
                               dtype="f32" if g.integers(0, 2) == 0 else "f64",
                               seed=int(g.integers(0, 2**63 - 1))))
    return out
