"""Serving on the GPU: results are the evaluator's results, alone or batched
with other requests; admission by slots and pool memory; back-pressure,
time-outs and release semantics."""
import time

import numpy as np
import pytest

from helpers import TOL_F32, TOL_F64, assert_normwise

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


def direct(points_np, lmax, dtype):
    """shm_eval on the same points (the unbatched evaluator)."""
    p = torch.from_numpy(points_np).to(device="cuda", dtype=dtype)
    out = shm.eval_sh(p, lmax)
    torch.cuda.synchronize()
    return out


def result(srv, ticket):
    r = srv.wait(ticket, timeout_ms=60_000)
    assert r.status == 0
    out = srv.result_tensor(r)
    torch.cuda.synchronize()
    return r, out


def test_generated_request_equals_evaluator_bitwise_and_oracle(oracle_mod):
    with shm.Server(pool_bytes=2 << 30) as srv:
        for dtype in (torch.float64, torch.float32):
            seed, n = 4242, 100_003
            t = srv.submit(n, 9, dtype, seed=seed)
            r, out = result(srv, t)
            pts = inputs.counter_points(seed, n)
            ref = direct(pts, 9, dtype)
            assert torch.equal(out, ref), f"{dtype}: batched rows differ from shm_eval"
            sample = np.arange(0, n, 97)
            p64 = pts[sample] if dtype == torch.float64 else pts[sample].astype(np.float32).astype(np.float64)
            assert_normwise(out.cpu().numpy()[sample], oracle_mod.real_sh(p64, 9),
                            TOL_F64 if dtype == torch.float64 else TOL_F32, f"serve {dtype}")
            srv.release(t)


def test_alone_and_in_the_mix_are_identical():
    g = inputs.rng("tests", 500)
    spec = dict(n=250_001, lmax=7, dtype=torch.float64, seed=99)
    with shm.Server(pool_bytes=8 << 30, batch_points=1 << 20, chunk_points=1 << 16, inflight_batches=3) as srv:
        t = srv.submit(spec["n"], spec["lmax"], spec["dtype"], seed=spec["seed"])
        _, alone = result(srv, t)
        alone = alone.clone()
        srv.release(t)
        # the same request again, submitted in the middle of 40 others of mixed
        # size, lmax and dtype so that their chunks share its batches
        others = []
        tickets = []
        for i in range(40):
            n = int(np.exp(g.uniform(np.log(1e3), np.log(3e5))))
            lmax = int(g.integers(0, 10))
            dt = torch.float32 if g.integers(0, 2) else torch.float64
            sd = int(g.integers(0, 2**62))
            others.append((n, lmax, dt, sd))
            tickets.append(srv.submit(n, lmax, dt, seed=sd))
            if i == 20:
                mid = srv.submit(spec["n"], spec["lmax"], spec["dtype"], seed=spec["seed"])
        _, mixed = result(srv, mid)
        assert torch.equal(mixed, alone)
        st = srv.stats()
        assert st["batches"] >= 2
        for (n, lmax, dt, sd), tk in zip(others, tickets):
            _, out = result(srv, tk)
            assert torch.equal(out, direct(inputs.counter_points(sd, n), lmax, dt)), (n, lmax, dt)
            srv.release(tk)
        srv.release(mid)


def test_user_points_requests():
    pts = inputs.random_sphere_points(70_000, stream="tests")
    with shm.Server(pool_bytes=1 << 30) as srv:
        for dtype in (torch.float64, torch.float32):
            p = torch.from_numpy(pts).to(device="cuda", dtype=dtype)
            t = srv.submit(p.shape[0], 5, dtype, points=p)
            _, out = result(srv, t)
            assert torch.equal(out, shm.eval_sh(p, 5))
            srv.release(t)


def test_admission_waits_for_pool_memory_and_release():
    n = 1 << 20
    row_bytes = 100 * 8
    # room for exactly one 800 MB output at a time
    with shm.Server(pool_bytes=n * row_bytes + 4096, max_slots=8) as srv:
        t1 = srv.submit(n, 9, torch.float64, seed=1)
        t2 = srv.submit(n, 9, torch.float64, seed=2)
        r1 = srv.wait(t1, timeout_ms=60_000)
        assert r1.status == 0
        st, r2 = srv.wait_status(t2, timeout_ms=200)     # cannot be admitted while t1 holds the pool
        assert st == 5 and r2.status == 5
        srv.release(t1)
        r2 = srv.wait(t2, timeout_ms=60_000)
        assert r2.status == 0 and r2.t_admit_ms >= r1.t_done_ms
        s = srv.stats()
        assert s["pool_peak"] <= s["pool_bytes"]
        srv.release(t2)


def test_backpressure_rejects_when_queue_full():
    with shm.Server(pool_bytes=256 << 20, max_slots=1, queue_capacity=4) as srv:
        got = [srv.submit(300_000, 9, torch.float64, seed=i, discard=True) for i in range(40)]
        rejected = sum(t is None for t in got)
        assert rejected > 0
        deadline = time.time() + 60
        while time.time() < deadline:
            s = srv.stats()
            if s["completed"] + s["rejected"] == s["submitted"]:
                break
            time.sleep(0.01)
        s = srv.stats()
        assert s["rejected"] == rejected and s["completed"] == 40 - rejected
        assert s["pool_in_use"] == 0            # discarded outputs went back to the pool


def test_ticket_errors_and_oversized_requests():
    with shm.Server(pool_bytes=64 << 20) as srv:
        with pytest.raises(shm.ShmError) as ei:
            srv.submit(10**6, 9, torch.float64, seed=1)      # 800 MB > 64 MB pool
        assert ei.value.status == 1
        t = srv.submit(1000, 3, torch.float64, seed=5)
        srv.wait(t, timeout_ms=60_000)
        srv.release(t)
        st, _ = srv.wait_status(t, timeout_ms=0)
        assert st == 7                                       # SHM_ENOTFOUND
        with pytest.raises(shm.ShmError) as ei:
            srv.release(t)
        assert ei.value.status == 7


def test_destroy_with_work_in_flight_drains():
    srv = shm.Server(pool_bytes=2 << 30)
    for i in range(10):
        srv.submit(200_000, 9, torch.float64, seed=i, discard=True)
    srv.close()                                              # returns after the admitted work drained


def test_latency_statistics():
    with shm.Server(pool_bytes=2 << 30) as srv:
        ts = [srv.submit(10_000 * (i + 1), i % 10, torch.float32, seed=i) for i in range(20)]
        for t in ts:
            srv.wait(t, timeout_ms=60_000)
            srv.release(t)
        s = srv.stats()
        assert s["completed"] == 20 and 0 < s["lat_p50_ms"] <= s["lat_p99_ms"] <= s["lat_max_ms"]
        assert s["harmonics_done"] == sum(10_000 * (i + 1) * ((i % 10) + 1) ** 2 for i in range(20))


def test_strict_fp64_requests_equal_strict_evaluator_bitwise(oracle_mod):
    """SHM_REQ_STRICT_FP64: the request's rows are the all-binary64 rows,
    bitwise those of shm_eval_ex with SHM_STRICT_FP64, alone and mixed with
    default FP64 and FP32 requests in the same batches."""
    g = inputs.rng("tests", 503)
    with shm.Server(pool_bytes=2 << 30, batch_points=1 << 16, chunk_points=1 << 14) as srv:
        tickets = []
        for i in range(12):
            n = int(g.integers(1000, 60_000))
            lmax = int(g.integers(0, 10))
            dtype = (torch.float64, torch.float32)[i % 2]
            strict = i % 4 == 0
            tickets.append((srv.submit(n, lmax, dtype, seed=1000 + i, strict=strict), n, lmax, dtype, strict, 1000 + i))
        for t, n, lmax, dtype, strict, seed in tickets:
            r, out = result(srv, t)
            pts = inputs.counter_points(seed, n)
            p = torch.from_numpy(pts).to(device="cuda", dtype=dtype)
            ref = shm.eval_sh(p, lmax, strict=strict)
            torch.cuda.synchronize()
            assert torch.equal(out, ref), (n, lmax, dtype, strict)
            if strict:
                assert_normwise(out.cpu().numpy()[::37], oracle_mod.real_sh(pts[::37], lmax), TOL_F64, "strict serve")
            srv.release(t)


def test_wait_any_returns_requests_in_completion_order_and_counts_client_latency():
    with shm.Server(pool_bytes=2 << 30) as srv:
        sizes = [400_000, 2_000, 3_000, 150_000, 1_000]
        tickets = {srv.submit(n, 9, torch.float64, seed=77 + i): n for i, n in enumerate(sizes)}
        seen = []
        while len(seen) < len(tickets):
            st, t, r = srv.wait_any(timeout_ms=60_000)
            assert st == 0 and t in tickets and r.status == 0
            assert t not in seen and r.n == tickets[t]
            seen.append(t)
        st, t, r = srv.wait_any(timeout_ms=20)       # nothing left to collect
        assert st == 5
        stats = srv.stats()
        assert stats["collected"] == len(sizes) and stats["completed"] == len(sizes)
        assert 0 < stats["client_lat_p50_ms"] <= stats["client_lat_max_ms"]
        # a wait on an already collected ticket still returns it, but counts it once
        assert srv.wait(seen[0], timeout_ms=10).status == 0
        assert srv.stats()["collected"] == len(sizes)
        for t in seen:
            srv.release(t)
        # discarded requests are never handed to wait_any
        srv.submit(5_000, 3, torch.float32, seed=1, discard=True)
        st, t, r = srv.wait_any(timeout_ms=2_000)
        assert st == 5


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("site", ["serve_pool", "serve_pinned", "serve_batch", "all"])
def test_injected_allocation_failure_at_create(site, monkeypatch):
    """SHM_FAIL_ALLOC makes the named allocation of shm_serve_create fail:
    SHM_ENOMEM, no server, nothing left allocated; without it the same
    create succeeds."""
    import ctypes
    from paper_2510_05282_b300 import _binding
    L = shm.lib()
    cfg = _binding.ServeConfig(pool_bytes=1 << 30, max_slots=8, queue_capacity=16, batch_points=1 << 16,
                               chunk_points=1 << 14, inflight_batches=2, device=torch.cuda.current_device())
    before = _free_bytes()
    monkeypatch.setenv("SHM_FAIL_ALLOC", site)
    h = ctypes.c_void_p(0)
    assert L.shm_serve_create(ctypes.byref(cfg), ctypes.byref(h)) == 2
    assert h.value is None
    assert "injected" in L.shm_last_error().decode()
    assert _free_bytes() >= before - (64 << 20)
    monkeypatch.delenv("SHM_FAIL_ALLOC")
    assert L.shm_serve_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    assert L.shm_serve_destroy(h) == 0


def test_injected_allocation_failure_in_the_tuner(monkeypatch):
    """The tuner's probe allocation fails: SHM_ENOMEM, the variant choice is
    unchanged and no probe kernel has run (the choice would otherwise move)."""
    before = shm.eval_variant(7, torch.float64)
    monkeypatch.setenv("SHM_FAIL_ALLOC", "autotune")
    with pytest.raises(shm.ShmError) as ei:
        shm.autotune(7, torch.float64, 1 << 14)
    assert ei.value.status == 2 and "injected" in str(ei.value)
    assert shm.eval_variant(7, torch.float64) == before
