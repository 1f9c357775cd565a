"""shm_projectors_noalloc: the projector entry point for callers that cannot
allocate device memory (for instance a host code whose framework already
holds the device memory in its own pool, or a time-step loop that must not
grow its footprint or synchronise through cudaMalloc).  It keeps its scratch
in a static device array of the library, so the caller passes only the
problem and the output.

Checked here through the C ABI against shm_projectors (which takes a caller
workspace), on two calls in a row: the two entry points run the same
launches with the same arithmetic, so the values must agree bit for bit.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2510_05282_b300 as shm  # noqa: E402
from paper_2510_05282_b300 import _binding, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_05282_b300 import build
    build.build()
    shm.lib()


def reference(d, dtype):
    ws = d.workspace(dtype)
    out = shm.projectors(d, dtype, workspace=ws)
    torch.cuda.synchronize()
    assert shm.projectors_check(ws) == 0
    return out


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("which", ["small", "full"])
def test_noalloc_matches_workspace_entry_point_twice(dtype, which):
    if which == "small":
        prob = inputs.projector_problem(n_atoms=6, box=6.0, h=0.25, rc_range=(1.0, 2.0), n_species=3,
                                        lmax_choices=(2, 3, 4), n_rad=200, r_min=1e-3, r_max=3.0, extra=9)
    else:
        prob = inputs.projector_problem()       # 512 atoms, 13.2M points
    d = shm.DeviceProjectors(prob)
    assert d.workspace_size(dtype) <= _binding.PROJ_NOALLOC_SCRATCH_BYTES
    ref = reference(d, dtype)
    L = shm.lib()
    code = shm.SHM_F64 if dtype == torch.float64 else shm.SHM_F32
    for call in range(2):
        out = torch.full((d.n_values,), float("nan"), dtype=dtype, device="cuda")
        st = L.shm_projectors_noalloc(ctypes.byref(d.c), code, out.data_ptr(), None)
        assert st == 0, L.shm_last_error()
        torch.cuda.synchronize()
        assert not torch.isnan(out).any(), f"call {call}: rows left unwritten"
        assert torch.equal(out, ref), f"call {call}: differs from shm_projectors"


def test_noalloc_rejects_problems_beyond_its_scratch():
    prob = inputs.projector_problem(n_atoms=6, box=6.0, h=0.25, rc_range=(1.0, 2.0), n_species=3,
                                    lmax_choices=(2, 3, 4), n_rad=200, r_min=1e-3, r_max=3.0, extra=10)
    d = shm.DeviceProjectors(prob)
    big = _binding._ProjProblem.from_buffer_copy(d.c)
    big.n_rad = 200_000          # FP32 interval cubics of 3 x 5 x 200000 nodes, 16 bytes each: 48 MB > 32 MiB
    out = torch.zeros(d.n_values, dtype=torch.float32, device="cuda")
    L = shm.lib()
    assert L.shm_projectors_noalloc(ctypes.byref(big), shm.SHM_F32, out.data_ptr(), None) == 1
    msg = L.shm_last_error().decode()
    assert "bytes of scratch" in msg and str(_binding.PROJ_NOALLOC_SCRATCH_BYTES) in msg
    torch.cuda.synchronize()
    assert torch.all(out == 0)
