"""GPU parity of shm_eval_spinor (spin-1/2 spinor harmonics, Eq. 7) against
the oracle's spinors.  Tolerance per value: tol * sqrt((2l+1)/4pi) for the
orbital l of the spinor (every coupling coefficient is <= 1, so this is the
l-shell bound of the harmonics it is made of)."""
import math

import numpy as np
import pytest

from helpers import TOL_F32, TOL_F64

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


def spinor_l(lmax):
    """Orbital l of each spinor of a row."""
    return np.array([l for l in range(lmax + 1) for _ in range(4 * l + 2)])


def check(got, ref, tol, what):
    L = int(round(math.sqrt(ref.shape[1] / 2))) - 1
    nb = np.sqrt((2 * spinor_l(L) + 1) / (4 * np.pi))[None, :, None]
    err = np.abs(got.astype(np.complex128) - ref) / nb
    assert not np.isnan(err).any(), what
    worst = float(err.max()) if err.size else 0.0
    assert worst <= tol, f"{what}: {worst:.3e}"
    return worst


@pytest.mark.parametrize("lmax", [0, 1, 4, 9])
@pytest.mark.parametrize("n", [1, 129, 5003])
def test_spinor_fp64(oracle_mod, lmax, n):
    pts = np.concatenate([inputs.random_sphere_points(n, stream="tests", with_axes=False), inputs.edge_points()])
    finite = np.all(np.isfinite(pts), axis=1)
    pts = pts[finite]
    got = shm.eval_spinor(torch.from_numpy(pts).cuda(), lmax).cpu().numpy()
    assert got.shape == (len(pts), 2 * (lmax + 1) ** 2, 2)
    check(got, oracle_mod.spinor_sh(pts, lmax), TOL_F64, f"FP64 lmax={lmax}")


@pytest.mark.parametrize("lmax", [0, 3, 9])
def test_spinor_fp32(oracle_mod, lmax):
    pts = inputs.random_sphere_points(20000, stream="tests").astype(np.float32)
    got = shm.eval_spinor(torch.from_numpy(pts).cuda(), lmax).cpu().numpy()
    check(got, oracle_mod.spinor_sh(pts.astype(np.float64), lmax), TOL_F32, f"FP32 lmax={lmax}")


def test_normalized_input_flag(oracle_mod):
    pts = inputs.random_sphere_points(3000, stream="tests", with_axes=False)
    u = pts / np.linalg.norm(pts, axis=1, keepdims=True)
    got = shm.eval_spinor(torch.from_numpy(u).cuda(), 9, normalized=True).cpu().numpy()
    check(got, oracle_mod.spinor_sh(u, 9), TOL_F64, "normalized")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_unaligned_output_takes_scalar_stores(oracle_mod, dtype):
    """An output that starts one element past a 16-byte boundary: same values."""
    pts = inputs.random_sphere_points(777, stream="tests")          # + the 64 axis points
    n = pts.shape[0]
    p = torch.from_numpy(pts).to(device="cuda", dtype=dtype)
    ns = shm.num_spinors(5)
    buf = torch.zeros(n * ns * 4 + 1, dtype=dtype, device="cuda")
    code = shm.SHM_F64 if dtype == torch.float64 else shm.SHM_F32
    shm.check(shm.lib().shm_eval_spinor(p.data_ptr(), n, 5, code, 0, buf[1:].data_ptr(), None))
    ref = shm.eval_spinor(p, 5)
    torch.cuda.synchronize()
    got = buf[1:].view(n, ns, 2, 2).cpu().numpy()
    assert np.array_equal(got[..., 0] + 1j * got[..., 1], ref.cpu().numpy())
    assert buf[0].item() == 0.0


def test_closure_and_origin_on_gpu():
    """sum over m_j of S S^dagger = (2j+1)/(8 pi) I for every (l, j); r = 0 keeps only l = 0."""
    pts = np.concatenate([inputs.random_sphere_points(2000, stream="tests", with_axes=False), np.zeros((3, 3))])
    S = shm.eval_spinor(torch.from_numpy(pts).cuda(), 9).cpu().numpy()
    q = 0
    for l in range(10):
        for s in ((1,) if l == 0 else (-1, 1)):
            tj = 2 * l + s
            blk = S[:-3, q:q + tj + 1]
            M = np.einsum("nqa,nqb->nab", blk, blk.conj())
            assert np.max(np.abs(M - (tj + 1) / (8 * np.pi) * np.eye(2))) <= 1e-13 * (tj + 1)
            q += tj + 1
    c = 1 / math.sqrt(4 * math.pi)
    ref = np.zeros((3, 200, 2), dtype=complex)
    ref[:, 0, 1] = c
    ref[:, 1, 0] = c
    assert np.array_equal(S[-3:], ref)


def test_bad_arguments():
    L = shm.lib()
    p = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    o = torch.zeros(4 * 200 * 4, dtype=torch.float64, device="cuda")
    assert L.shm_eval_spinor(p.data_ptr(), 4, 10, shm.SHM_F64, 0, o.data_ptr(), None) == 1
    assert L.shm_eval_spinor(p.data_ptr(), 4, 9, shm.SHM_F64, 8, o.data_ptr(), None) == 1
    assert L.shm_eval_spinor(None, 4, 9, shm.SHM_F64, 0, o.data_ptr(), None) == 1
    assert L.shm_eval_spinor(p.data_ptr(), 0, 9, shm.SHM_F64, 0, None, None) == 0


def test_spinor_full_grid_sampled(oracle_mod, capsys):
    """The 192^3 grid of the benchmark, FP64 (45 GB of output): 20,000 sampled
    rows against the oracle, in the benchmark's launch set-up."""
    pts = inputs.dft_grid_points(192)
    S = shm.eval_spinor(torch.from_numpy(pts).cuda(), 9)
    torch.cuda.synchronize()
    rows = np.unique(inputs.rng("tests", 83).integers(0, pts.shape[0], 20000))
    got = S[torch.from_numpy(rows).cuda()].cpu().numpy()
    del S
    torch.cuda.empty_cache()
    worst = check(got, oracle_mod.spinor_sh(pts[rows], 9), TOL_F64, "spinor 192^3 sample")
    with capsys.disabled():
        print(f"\nspinor FP64 192^3 sample: max normwise error {worst:.2e}")
