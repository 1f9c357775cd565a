"""GPU parity of shm_eval_complex (complex Y_l^m, Eq. 5 and Eq. 10) against
the oracle's complex harmonics, normwise per l as for the real ones."""
import numpy as np
import pytest

from helpers import TOL_F32, TOL_F64, norm_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2510_05282_b300 as shm  # noqa: E402
from paper_2510_05282_b300 import inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_05282_b300 import build
    build.build()
    shm.lib()


def check(got, ref, tol, what):
    nb = norm_bound(ref.shape[1])
    err = np.abs(got.astype(np.complex128) - ref) / nb
    assert not np.isnan(err).any(), what
    assert float(err.max()) <= tol, f"{what}: {float(err.max()):.3e}"


@pytest.mark.parametrize("lmax", [0, 1, 4, 9])
@pytest.mark.parametrize("n", [1, 129, 5003])
def test_complex_fp64(oracle_mod, lmax, n):
    pts = np.concatenate([inputs.random_sphere_points(n, stream="tests", with_axes=False), inputs.edge_points()])
    got = shm.eval_complex(torch.from_numpy(pts).cuda(), lmax).cpu().numpy()
    finite = np.all(np.isfinite(pts), axis=1)
    check(got[finite], oracle_mod.complex_sh(pts[finite], lmax), TOL_F64, f"FP64 lmax={lmax}")


@pytest.mark.parametrize("lmax", [0, 3, 9])
def test_complex_fp32(oracle_mod, lmax):
    pts = inputs.random_sphere_points(20000, stream="tests").astype(np.float32)
    got = shm.eval_complex(torch.from_numpy(pts).cuda(), lmax).cpu().numpy()
    check(got, oracle_mod.complex_sh(pts.astype(np.float64), lmax), TOL_F32, f"FP32 lmax={lmax}")


def test_complex_matches_real_rows_exactly_where_it_must():
    """Y_l^0 equals R_l^0 bitwise; |Y_l^m|^2 sums to (2l+1)/4pi."""
    pts = inputs.random_sphere_points(4000, stream="tests")
    p = torch.from_numpy(pts).cuda()
    Y = shm.eval_complex(p, 9).cpu().numpy()
    shm.set_eval_variant(9, torch.float64, 7)            # a hybrid variant: same m = 0 code
    try:
        R = shm.eval_sh(p, 9).cpu().numpy()
    finally:
        shm.set_eval_variant(9, torch.float64, -1)
    for l in range(10):
        k = l * l + l
        assert np.array_equal(Y[:, k].real, R[:, k]) and np.all(Y[:, k].imag == 0)
        s = np.sum(np.abs(Y[:, l * l:(l + 1) ** 2]) ** 2, axis=1)
        assert np.max(np.abs(s - (2 * l + 1) / (4 * np.pi))) <= 4e-13 * (2 * l + 1) / (4 * np.pi)


def test_complex_full_grid_sampled(oracle_mod):
    pts = inputs.dft_grid_points(192)
    Y = shm.eval_complex(torch.from_numpy(pts).cuda(), 9)
    torch.cuda.synchronize()
    rows = np.unique(inputs.rng("tests", 79).integers(0, pts.shape[0], 20000))
    got = Y[torch.from_numpy(rows).cuda()].cpu().numpy()
    check(got, oracle_mod.complex_sh(pts[rows], 9), TOL_F64, "complex 192^3 sample")
