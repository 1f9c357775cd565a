"""Host-side parts of serving that need no GPU: the counter-based point
generator agrees bit for bit between the library's host twin and the Python
input generator, and bad create/submit arguments are rejected before any CUDA
call."""
import ctypes

import numpy as np
import pytest

import paper_2510_05282_b300 as shm
from paper_2510_05282_b300 import _binding, inputs


@pytest.fixture(scope="module")
def L():
    from paper_2510_05282_b300 import build
    build.build()
    return shm.lib()


@pytest.mark.parametrize("seed", [0, 1, 12345, 2**63 - 1, 0xDEADBEEFCAFEF00D])
def test_generator_bitwise_host_vs_python(L, seed):
    idx = np.concatenate([np.arange(300), np.array([10**6, 4 * 10**6 - 1, 2**31 + 5])])
    py = np.concatenate([inputs.counter_points(seed, 1, start=int(i)) for i in idx])
    host = np.array([shm.serve_generated_point(seed, int(i)) for i in idx])
    assert np.array_equal(py, host)


def test_generator_distribution():
    """Directions (2s(1-t^2), 4st, (1-s^2)(1+t^2)) / ((1+s^2)(1+t^2)) with s, t
    uniform on [-1, 1): z = (1-s^2)/(1+s^2), so E[z] = 0 (random sign) and
    E[z^2] = int_0^1 ((1-s^2)/(1+s^2))^2 ds = 2 - pi/2 (checked by
    quadrature); radii 2^e (1+m) (1+s^2)(1+t^2) in [2^-10, 64)."""
    from scipy.integrate import quad
    pts = inputs.counter_points(7, 200_000)
    r = np.linalg.norm(pts, axis=1)
    assert r.min() >= 2.0 ** -10 * 0.999 and r.max() < 64.0
    u = pts / r[:, None]
    ez2 = quad(lambda s: ((1 - s * s) / (1 + s * s)) ** 2, 0, 1)[0]
    assert abs(ez2 - (2 - np.pi / 2)) < 1e-12
    assert abs(u[:, 2].mean()) < 0.01 and abs((u[:, 2] ** 2).mean() - ez2) < 0.01
    # every octant is populated
    octs = ((u > 0) * np.array([1, 2, 4])).sum(axis=1)
    assert np.bincount(octs, minlength=8).min() > 20_000


def test_create_and_submit_validation_without_gpu(L):
    h = ctypes.c_void_p()
    assert L.shm_serve_create(None, ctypes.byref(h)) == 1
    bad = _binding.ServeConfig(pool_bytes=1 << 20, max_slots=0, queue_capacity=1, batch_points=1,
                               chunk_points=1, inflight_batches=1, device=0)
    assert L.shm_serve_create(ctypes.byref(bad), ctypes.byref(h)) == 1
    req = _binding._Request(points=None, n=10, lmax=3, dtype=1, seed=0, flags=0)
    t = ctypes.c_uint64()
    assert L.shm_serve_submit(None, ctypes.byref(req), ctypes.byref(t)) == 1


def test_injected_tuner_allocation_failure_without_gpu(L, monkeypatch):
    """SHM_FAIL_ALLOC=autotune: the tuner's probe allocation fails before any
    CUDA call, with SHM_ENOMEM and a message naming the injection."""
    monkeypatch.setenv("SHM_FAIL_ALLOC", "autotune")
    best = ctypes.c_double(-1.0)
    assert L.shm_autotune(9, 1, 1000, ctypes.byref(best)) == 2
    assert "injected" in L.shm_last_error().decode()
    assert best.value == -1.0
    monkeypatch.setenv("SHM_FAIL_ALLOC", "serve_pool,autotune")
    assert L.shm_autotune_ex(5, 0, 0, 1000, ctypes.byref(best)) == 2
    monkeypatch.setenv("SHM_FAIL_ALLOC", "serve_pool")     # another site only: the tuner's own check passes
    st = L.shm_autotune(9, 1, 1000, ctypes.byref(best))
    assert "injected" not in L.shm_last_error().decode()
    assert st != 0                                           # no GPU here: a real failure


def test_request_flags_validated(L):
    """Unknown request flag bits are refused (SHM_REQ_DISCARD | SHM_REQ_STRICT_FP64 are the known ones)."""
    req = _binding._Request(points=None, n=10, lmax=3, dtype=1, seed=0, flags=0x4)
    t = ctypes.c_uint64()
    assert L.shm_serve_submit(ctypes.c_void_p(1), ctypes.byref(req), ctypes.byref(t)) == 1
