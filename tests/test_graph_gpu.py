"""The evaluators can be captured into a CUDA graph and replayed: they
allocate nothing, check their arguments on the host, and only enqueue
kernels on the given stream.  Replayed results equal eager ones bit for bit."""
import numpy as np
import pytest

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


def capture_and_replay(fn, replays=3):
    """fn(stream) enqueues work on `stream`; returns after capturing it once and
    replaying the graph `replays` times."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn(s)                      # warm-up outside the capture (per-device set-up)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fn(s)
    for _ in range(replays):
        g.replay()
    torch.cuda.synchronize()
    return g


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_eval_graph_replay_bitwise(dtype):
    pts = inputs.random_sphere_points(50_000, stream="tests")
    p = torch.from_numpy(pts).to(device="cuda", dtype=dtype)
    ref = shm.eval_sh(p, 9).clone()
    out = torch.full_like(ref, float("nan"))
    capture_and_replay(lambda s: shm.eval_sh(p, 9, out=out, stream=s))
    assert torch.equal(torch.nan_to_num(out, nan=7.0), torch.nan_to_num(ref, nan=7.0))


def test_complex_spinor_angles_graph_replay_bitwise():
    pts = inputs.random_sphere_points(20_000, stream="tests", with_axes=False)
    p = torch.from_numpy(pts).cuda()
    r = np.linalg.norm(pts, axis=1)
    ang = torch.from_numpy(np.stack([np.arccos(pts[:, 2] / r), np.arctan2(pts[:, 1], pts[:, 0])], 1)).cuda()
    refs = (shm.eval_complex(p, 9).clone(), shm.eval_spinor(p, 9).clone(), shm.eval_angles(ang, 9).clone())
    outc = torch.empty((p.shape[0], 100, 2), dtype=torch.float64, device="cuda")
    outs = torch.empty((p.shape[0], 200, 2, 2), dtype=torch.float64, device="cuda")
    outa = torch.empty((p.shape[0], 100), dtype=torch.float64, device="cuda")

    def work(s):
        shm.eval_complex(p, 9, out=outc, stream=s)
        shm.eval_spinor(p, 9, out=outs, stream=s)
        shm.eval_angles(ang, 9, out=outa, stream=s)

    capture_and_replay(work)
    assert torch.equal(torch.view_as_complex(outc), refs[0])
    assert torch.equal(torch.view_as_complex(outs), refs[1])
    assert torch.equal(outa, refs[2])


def test_graph_replays_follow_new_input_values():
    """The graph holds pointers, not values: new points written into the same
    buffer give the new rows on the next replay."""
    a = inputs.random_sphere_points(10_000, stream="tests", with_axes=False)
    b = inputs.random_sphere_points(10_000, stream="sphere", with_axes=False)
    p = torch.from_numpy(a).cuda()
    out = torch.empty((p.shape[0], 100), dtype=torch.float64, device="cuda")
    g = capture_and_replay(lambda s: shm.eval_sh(p, 9, out=out, stream=s), replays=1)
    p.copy_(torch.from_numpy(b))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, shm.eval_sh(torch.from_numpy(b).cuda(), 9))
