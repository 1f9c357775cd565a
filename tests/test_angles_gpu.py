"""GPU parity of shm_eval_angles (the angular interface): the paper's printed
reference values of Tables II and III (App. D, given at angles) and the
oracle's angular entry on random angles."""
import math
import os

import numpy as np
import pytest

from helpers import TOL_F32, TOL_F64, assert_normwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2510_05282_b300 as shm  # noqa: E402
from paper_2510_05282_b300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_05282_b300 import build
    build.build()
    shm.lib()


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
    ("table2_point1.txt", 2.12160245947564796, -1.82732370250979703),
    ("table3_point2.txt", 1.69050041976591414, 0.758228122208986166),   # decimal point of phi restored
])
def test_printed_reference_values_on_the_gpu(name, theta, phi):
    ang = torch.tensor([[theta, phi]], dtype=torch.float64, device="cuda")
    R = shm.eval_angles(ang, 9).cpu().numpy()[0]
    for l, m, cos_col, sin_col in read_table(name):
        nb = math.sqrt((2 * l + 1) / (4 * math.pi))
        assert abs(R[l * l + l + m] - cos_col) <= TOL_F64 * nb, (l, m)
        if m > 0:
            assert abs(R[l * l + l - m] - sin_col) <= TOL_F64 * nb, (l, -m)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, TOL_F64), (torch.float32, TOL_F32)])
@pytest.mark.parametrize("lmax", [0, 5, 9])
def test_random_angles_against_oracle(oracle_mod, dtype, tol, lmax):
    g = inputs.rng("tests", 31)
    n = 20000
    theta = np.arccos(g.uniform(-1, 1, n))
    phi = g.uniform(-np.pi, np.pi, n)
    theta[:4] = [0.0, np.pi, np.pi / 2, 1e-9]          # poles, equator, near a pole
    ang = np.stack([theta, phi], axis=1)
    a = torch.from_numpy(ang).to(device="cuda", dtype=dtype)
    got = shm.eval_angles(a, lmax).cpu().numpy()
    a64 = a.double().cpu().numpy()
    assert_normwise(got, oracle_mod.real_sh_angles(a64[:, 0], a64[:, 1], lmax), tol, f"angles {dtype}")


@pytest.mark.parametrize("lmax", [3, 9])
def test_wide_phi_range_against_oracle(oracle_mod, lmax):
    """FP64 rows over azimuths far outside [-pi, pi]: the float-float
    sine/cosine of phi (|phi| <= 800) with its argument reduction, the binary64
    one beyond, and azimuths on and next to the quadrant boundaries k pi/2
    and the switch at |phi| = 800.  The oracle evaluates cos(m phi) with m phi
    rounded in binary64, an error of up to m |phi| 2^-53 at large |phi|; R is
    2 pi-periodic in phi, so it is given phi reduced to [-pi, pi] in 120-bit
    arithmetic instead (within 2^-52 of the exact reduction)."""
    g = inputs.rng("tests", 37)
    n = 12000
    theta = np.arccos(g.uniform(-1, 1, n))
    phi = g.uniform(-1000.0, 1000.0, n)
    k = np.arange(-40, 41)
    edges = np.concatenate([k * np.pi / 2, k * np.pi / 2 + 1e-13, k * np.pi / 2 - 1e-9, k * np.pi / 4 + 509 * np.pi / 2,
                            [800.0, -800.0, np.nextafter(800.0, 1e3), np.nextafter(-800.0, -1e3), 0.0, -0.0, 1e-300,
                             -3e-8, 799.9999999, -254.5 * np.pi]])
    phi[:edges.size] = edges
    ang = np.stack([theta, phi], axis=1)
    a = torch.from_numpy(ang).to(device="cuda", dtype=torch.float64)
    got = shm.eval_angles(a, lmax).cpu().numpy()
    mpmath = pytest.importorskip("mpmath")
    with mpmath.workprec(120):
        two_pi = 2 * mpmath.pi
        phi_red = np.array([float(mpmath.mpf(float(v)) - two_pi * round(v / (2 * np.pi))) for v in phi])
    assert np.all(np.abs(phi_red) <= np.pi + 1e-9)
    assert_normwise(got, oracle_mod.real_sh_angles(ang[:, 0], phi_red, lmax), TOL_F64, "wide phi")
