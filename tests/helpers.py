"""Shared test utilities: error measures and tolerances.

Tolerance (normwise per l): |R_gpu - R_oracle| <= tol * sqrt((2l+1)/(4 pi)).
sqrt((2l+1)/(4 pi)) bounds |R_l^m| by the addition theorem, so this is a
relative error against the size of the l-shell, well defined on the nodal
lines where a pointwise relative error is not.  FP64: tol = 1e-13, FP32:
tol = 2e-6 (the FP32 reference is the oracle at the FP32 inputs upcast
exactly to FP64).
"""
import math

import numpy as np

TOL_F64 = 1e-13
TOL_F32 = 2e-6


def l_of_k(nh):
    return np.array([int(math.isqrt(k)) for k in range(nh)])


def norm_bound(nh):
    l = l_of_k(nh)
    return np.sqrt((2 * l + 1) / (4 * np.pi))


def normwise_err(got, ref):
    """[n, nh] array of |got - ref| / sqrt((2l+1)/4pi)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(got - ref) / norm_bound(ref.shape[1])[None, :]


def per_l_max(err):
    l = l_of_k(err.shape[1])
    return [float(err[:, l == ll].max()) if err.shape[0] else 0.0 for ll in range(int(l.max()) + 1)]


def per_l_mean(err):
    l = l_of_k(err.shape[1])
    return [float(err[:, l == ll].mean()) if err.shape[0] else 0.0 for ll in range(int(l.max()) + 1)]


def per_l_report(err):
    """'l: max/mean' of a normwise error array, for the printed accuracy reports."""
    return " ".join(f"{ll}:{a:.1e}/{b:.1e}" for ll, (a, b) in enumerate(zip(per_l_max(err), per_l_mean(err))))


def assert_normwise(got, ref, tol, what=""):
    err = normwise_err(got, ref)
    if err.size == 0:
        return
    worst = float(np.nanmax(err))
    assert not np.isnan(err).any(), f"{what}: NaN mismatch"
    assert worst <= tol, f"{what}: max normwise error {worst:.3e} > {tol:.1e}; per l {per_l_max(err)}"
