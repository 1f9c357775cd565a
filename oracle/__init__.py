"""CPU FP64 oracle for the real spherical harmonics and the fused projectors.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product package ``paper_2510_05282_b300`` never imports it, and
this package imports nothing from the product package.

The arithmetic lives in ``sh_oracle.c`` (plain C, binary64), which is written
from the paper's theta/phi definition (Eq. 3-6 and Eq. 10 of arXiv 2510.05282,
with the r = 0 convention of Sec. II); this module only marshals numpy arrays
through ctypes.  ``build()`` compiles it with gcc (OpenMP over points).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SHM_ORACLE_SRC / SHM_ORACLE_BUILD_DIR let the mutation tests build a copy of
# the oracle with a planted mistake and check that the pins catch it.
_SRC = os.environ.get("SHM_ORACLE_SRC", os.path.join(_HERE, "sh_oracle.c"))
_BUILD_DIR = os.environ.get("SHM_ORACLE_BUILD_DIR", os.path.join(_HERE, "_build"))
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

LMAX_CAP = 16

_lib = None


def build(force: bool = False) -> str:
    """Compile ``sh_oracle.c`` into ``oracle/_build/liboracle.so`` (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, i32, dp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        lib.oracle_real_sh.argtypes = [dp, i64, i32, dp, i32]
        lib.oracle_real_sh.restype = i32
        lib.oracle_real_sh_angles.argtypes = [dp, dp, i64, i32, dp]
        lib.oracle_real_sh_angles.restype = i32
        lib.oracle_complex_sh.argtypes = [dp, i64, i32, dp, i32]
        lib.oracle_complex_sh.restype = i32
        lib.oracle_spinor_sh.argtypes = [dp, i64, i32, dp, i32]
        lib.oracle_spinor_sh.restype = i32
        lib.oracle_max_threads.argtypes = [i32]
        lib.oracle_max_threads.restype = i32
        lib.oracle_projectors.argtypes = [i64, dp, dp, dp, i32, dp, i32, i32, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, i32, ctypes.c_double,
                                          dp, dp, dp, dp, i32]
        lib.oracle_projectors.restype = i32
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def n_harmonics(lmax: int) -> int:
    return (lmax + 1) * (lmax + 1)


def max_threads(nthreads: int = 0) -> int:
    """Threads the oracle's OpenMP loops use for ``nthreads`` (0 = OpenMP default)."""
    return int(_load().oracle_max_threads(int(nthreads)))


def real_sh(points, lmax: int, nthreads: int = 0) -> np.ndarray:
    """R_l^m for l <= lmax at Cartesian points [n, 3] (float64) -> [n, (lmax+1)^2]."""
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    out = np.empty((pts.shape[0], n_harmonics(lmax)), dtype=np.float64)
    rc = _load().oracle_real_sh(_ptr(pts), pts.shape[0], int(lmax), _ptr(out), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_real_sh rejected its arguments (lmax={lmax})")
    return out


def complex_sh(points, lmax: int, nthreads: int = 0) -> np.ndarray:
    """Complex Y_l^m (Eq. 5, Eq. 10) at Cartesian points -> [n, (lmax+1)^2] complex128."""
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    out = np.empty((pts.shape[0], n_harmonics(lmax), 2), dtype=np.float64)
    rc = _load().oracle_complex_sh(_ptr(pts), pts.shape[0], int(lmax), _ptr(out), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_complex_sh rejected its arguments (lmax={lmax})")
    return out[..., 0] + 1j * out[..., 1]


def n_spinors(lmax: int) -> int:
    """Spinor harmonics per point: j = l +- 1/2 for l <= lmax, 2 (lmax+1)^2."""
    return 2 * (lmax + 1) ** 2


def spinor_index(l: int, s: int, two_mj: int) -> int:
    """Position of the spinor (l, j = l + s/2, m_j = two_mj/2) in a row."""
    two_j = 2 * l + s
    return 2 * l * l + (0 if s < 0 else 2 * l) + (two_mj + two_j) // 2


def spinor_sh(points, lmax: int, nthreads: int = 0) -> np.ndarray:
    """Spinor harmonics (Eq. 7) at Cartesian points -> [n, 2 (lmax+1)^2, 2]
    complex128: (upper, lower) component of each spinor, order spinor_index."""
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    out = np.empty((pts.shape[0], n_spinors(lmax), 2, 2), dtype=np.float64)
    rc = _load().oracle_spinor_sh(_ptr(pts), pts.shape[0], int(lmax), _ptr(out), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_spinor_sh rejected its arguments (lmax={lmax})")
    return out[..., 0] + 1j * out[..., 1]


def real_sh_angles(theta, phi, lmax: int) -> np.ndarray:
    """R_l^m at angular inputs (theta, phi) -> [n, (lmax+1)^2] (float64)."""
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
    ph = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
    if th.shape != ph.shape:
        raise ValueError("theta and phi differ in length")
    out = np.empty((th.shape[0], n_harmonics(lmax)), dtype=np.float64)
    rc = _load().oracle_real_sh_angles(_ptr(th), _ptr(ph), th.shape[0], int(lmax), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_real_sh_angles rejected its arguments (lmax={lmax})")
    return out


def projectors(prob, nthreads: int = 0) -> np.ndarray:
    """Fused projector values f_{s,l}(|d|) R_l^m(d/|d|) for a projector problem.

    ``prob`` is a ``ProjectorProblem`` (see ``paper_2510_05282_b300.inputs``) or any
    object with the same fields; the output is the flat CSR value array.
    """
    pos = np.ascontiguousarray(prob.atom_pos, dtype=np.float64)
    spec = np.ascontiguousarray(prob.atom_species, dtype=np.int32)
    slmax = np.ascontiguousarray(prob.species_lmax, dtype=np.int32)
    rad = np.ascontiguousarray(prob.radial, dtype=np.float64)
    poff = np.ascontiguousarray(prob.point_offsets, dtype=np.int64)
    pidx = np.ascontiguousarray(prob.point_index, dtype=np.int32)
    ooff = np.ascontiguousarray(prob.out_offsets, dtype=np.int64)
    out = np.empty(int(ooff[-1]), dtype=np.float64)
    rc = _load().oracle_projectors(
        pos.shape[0], _ptr(pos), _ptr(spec), _ptr(slmax), slmax.shape[0],
        _ptr(rad), rad.shape[1], rad.shape[2], float(prob.r_min), float(prob.dlog),
        float(prob.box), int(prob.ng), float(prob.h),
        _ptr(poff), _ptr(pidx), _ptr(ooff), _ptr(out), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_projectors rejected its arguments")
    return out
