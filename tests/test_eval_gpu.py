"""GPU parity of shm_eval against the CPU FP64 oracle (through the C ABI).

Tolerances (see helpers.py): normwise per l, 1e-13 for FP64 and 2e-6 for FP32
against the oracle at the FP32 inputs upcast exactly.
"""
import numpy as np
import pytest

from helpers import TOL_F32, TOL_F64, assert_normwise, normwise_err, per_l_max, per_l_report

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


def gpu_eval(pts_np, lmax, dtype=torch.float64, normalized=False):
    p = torch.from_numpy(np.ascontiguousarray(pts_np)).to(device="cuda", dtype=dtype)
    out = shm.eval_sh(p, lmax, normalized=normalized)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_random_sphere_fp64_all_points(oracle_mod, capsys):
    pts = inputs.random_sphere_points(65_536)          # 65,600 points incl. 64 on the axes
    got = gpu_eval(pts, 9)
    ref = oracle_mod.real_sh(pts, 9)
    with capsys.disabled():
        print("\nFP64 random sphere 65,600, normwise error per l (max/mean):", per_l_report(normwise_err(got, ref)))
    assert_normwise(got, ref, TOL_F64, "random sphere FP64")


@pytest.mark.parametrize("lmax", list(range(10)))
@pytest.mark.parametrize("n", [1, 127, 128, 129, 1000, 4099])
def test_every_lmax_and_ragged_sizes_fp64(oracle_mod, lmax, n):
    pts = inputs.random_sphere_points(n, stream="tests", with_axes=False)
    got = gpu_eval(pts, lmax)
    assert got.shape == (n, (lmax + 1) ** 2)
    assert_normwise(got, oracle_mod.real_sh(pts, lmax), TOL_F64, f"lmax={lmax} n={n}")


@pytest.mark.parametrize("lmax", [0, 3, 9])
@pytest.mark.parametrize("n", [1, 129, 4099])
def test_every_lmax_and_ragged_sizes_fp32(oracle_mod, lmax, n):
    pts32 = inputs.random_sphere_points(n, stream="tests", with_axes=False).astype(np.float32)
    got = gpu_eval(pts32, lmax, dtype=torch.float32)
    ref = oracle_mod.real_sh(pts32.astype(np.float64), lmax)
    assert_normwise(got, ref, TOL_F32, f"FP32 lmax={lmax} n={n}")


def test_edge_points_fp64(oracle_mod):
    pts = inputs.edge_points()
    got = gpu_eval(pts, 9)
    ref = oracle_mod.real_sh(pts, 9)
    assert_normwise(got, ref, TOL_F64, "edge points")
    # r = 0 rows are exactly [1/sqrt(4 pi), 0, ...] (Sec. II)
    for i in (0, 1):
        assert got[i, 0] == np.float64(0.28209479177387814347)
        assert np.all(got[i, 1:] == 0.0)
    # on the z axis every m != 0 harmonic is exactly zero
    l = np.array([int(np.sqrt(k)) for k in range(100)])
    m = np.arange(100) - l * l - l
    for i in (2, 3):
        assert np.all(got[i, m != 0] == 0.0)


def test_edge_points_fp32(oracle_mod):
    pts32 = inputs.edge_points()
    pts32 = pts32[np.all(np.abs(pts32) < 1e30, axis=1)].astype(np.float32)
    got = gpu_eval(pts32, 9, dtype=torch.float32)
    ref = oracle_mod.real_sh(pts32.astype(np.float64), 9)
    assert_normwise(got, ref, TOL_F32, "FP32 edge points")


def test_nan_propagates():
    got = gpu_eval(np.array([[np.nan, 0.0, 1.0], [0.0, 0.0, 1.0]]), 4)
    assert np.all(np.isnan(got[0, 1:]))
    assert not np.isnan(got[1]).any()


def _points_with_nonfinite(n=300):
    """n finite points with non-finite rows at the tile edges and inside."""
    pts = inputs.random_sphere_points(n, stream="tests", with_axes=False)
    bad_rows = {0: [np.nan, 0.0, 1.0], 1: [np.inf, 0.0, 0.0], 127: [0.0, -np.inf, 1.0],
                128: [1.0, 2.0, np.nan], 200: [np.inf, np.inf, -np.inf], n - 1: [np.nan, np.nan, np.nan]}
    for i, v in bad_rows.items():
        pts[i] = v
    return pts, np.array(sorted(bad_rows))


@pytest.mark.parametrize("lmax", [2, 9])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_nonfinite_points_give_nan_rows_every_variant(oracle_mod, lmax, dtype):
    """A NaN or infinite coordinate gives NaN in every value but the constant
    l = 0 one, on every launch variant and with the normalised-input flag;
    the finite rows of the same launch are unaffected."""
    pts, bad = _points_with_nonfinite()
    good = np.setdiff1d(np.arange(pts.shape[0]), bad)
    p = torch.from_numpy(pts).to(device="cuda", dtype=dtype)
    ref = oracle_mod.real_sh(p[torch.from_numpy(good).cuda()].double().cpu().numpy(), lmax)
    tol = TOL_F64 if dtype == torch.float64 else TOL_F32
    try:
        for v in range(shm.eval_variant_count()):
            shm.set_eval_variant(lmax, dtype, v)
            for normalized in (False, True):
                got = shm.eval_sh(p, lmax, normalized=normalized).cpu().numpy()
                what = f"{shm.eval_variant(lmax, dtype)} normalized={normalized}"
                assert np.allclose(got[bad, 0], 0.28209479177387814347, rtol=1e-7, atol=0), what
                assert np.all(np.isnan(got[bad, 1:])), what
                if not normalized:
                    assert_normwise(got[good], ref, tol, what)
    finally:
        shm.set_eval_variant(lmax, dtype, -1)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_nonfinite_points_complex_spinor_angles(oracle_mod, dtype):
    pts, bad = _points_with_nonfinite()
    good = np.setdiff1d(np.arange(pts.shape[0]), bad)
    tol = TOL_F64 if dtype == torch.float64 else TOL_F32
    y00 = 0.28209479177387814347
    p = torch.from_numpy(pts).to(device="cuda", dtype=dtype)
    cx = shm.eval_complex(p, 9).cpu().numpy()
    assert np.allclose(cx[bad, 0], y00, rtol=1e-7, atol=0)
    assert np.all(np.isnan(cx[bad, 1:].real))
    assert np.all(np.isfinite(cx[good]))
    sp = shm.eval_spinor(p, 9).cpu().numpy()           # [n, 200, 2]; spinors 0, 1 are the l = 0 block
    assert np.all(np.isfinite(sp[bad, :2]))
    assert np.all(np.isnan(sp[bad, 2:].real))
    assert np.all(np.isfinite(sp[good]))
    # angles: a NaN or infinite theta or phi
    ang = np.stack([np.arccos(np.clip(pts[:, 2] / np.linalg.norm(pts, axis=1), -1, 1)),
                    np.arctan2(pts[:, 1], pts[:, 0])], 1)
    bad_a = good[:3]
    ang[bad_a] = [[np.nan, 0.1], [0.3, np.inf], [-np.inf, np.nan]]
    fine = good[3:]
    a = torch.from_numpy(np.ascontiguousarray(ang)).to(device="cuda", dtype=dtype)
    got = shm.eval_angles(a, 9).cpu().numpy()
    assert np.allclose(got[bad_a, 0], y00, rtol=1e-7, atol=0)
    assert np.all(np.isnan(got[bad_a, 1:]))
    ref = oracle_mod.real_sh(pts[fine].astype(np.float32).astype(np.float64) if dtype == torch.float32 else pts[fine], 9)
    assert_normwise(got[fine], ref, 10 * tol if dtype == torch.float32 else tol, "angles next to non-finite rows")


def test_normalized_input_flag(oracle_mod):
    pts = inputs.random_sphere_points(5000, stream="tests", with_axes=False)
    unit = pts / np.linalg.norm(pts, axis=1, keepdims=True)
    got = gpu_eval(unit, 9, normalized=True)
    assert_normwise(got, oracle_mod.real_sh(pts, 9), TOL_F64, "normalized input")


def test_unaligned_output_uses_scalar_path(oracle_mod):
    """An output 8 but not 16 bytes aligned takes the scalar stores: same rows,
    bitwise, as the 16-byte path, for every launch variant."""
    pts = inputs.random_sphere_points(1001, stream="tests", with_axes=False)
    p = torch.from_numpy(pts).cuda()
    buf = torch.empty(1001 * 100 + 1, dtype=torch.float64, device="cuda")
    out = buf[1:]                                  # 8-byte but not 16-byte aligned
    assert out.data_ptr() % 16 == 8
    try:
        for v in range(shm.eval_variant_count()):
            shm.set_eval_variant(9, torch.float64, v)
            shm.eval_sh(p, 9, out=out)
            ref = shm.eval_sh(p, 9)
            torch.cuda.synchronize()
            assert torch.equal(out.view(1001, 100), ref), shm.eval_variant(9, torch.float64)
            assert_normwise(out.view(1001, 100).cpu().numpy(), oracle_mod.real_sh(pts, 9), TOL_F64, "unaligned")
    finally:
        shm.set_eval_variant(9, torch.float64, -1)


TMA_VARIANT = 12
TMA2_VARIANT = 13
COPY_OUT_VARIANT = 11
TMA_EMU_VARIANTS = {18: "phased-hybrid-tma-emu-o-128", 19: "phased-hybrid-tma-emu-os-128"}


def _tma_test_points(n):
    """Random-sphere points with, where n allows, origin and non-finite rows
    in the first tile, the middle and the ragged last tile."""
    pts = inputs.random_sphere_points(n, stream="tests", with_axes=False)
    special = {0: [0.0, 0.0, 0.0], 5: [np.nan, 1.0, 0.0], n // 2: [0.0, -0.0, 0.0], n - 1: [np.inf, 0.0, 1.0]}
    for i, v in special.items():
        if n > 8:
            pts[i] = v
    return pts


@pytest.mark.parametrize("variant", [TMA_VARIANT, TMA2_VARIANT])
@pytest.mark.parametrize("lmax", [1, 2, 3, 5, 7, 9, 11])
@pytest.mark.parametrize("n", [1, 127, 128, 129, 4099, 200_003])
def test_tma_variants_match_copy_out_variant(variant, lmax, n):
    """phased-hybrid-tma-128 (TMA tensor stores of each staged phase) and
    phased-hybrid-tma2-128 (double-buffered, 20-column phases) write the same
    bits as phased-hybrid-128 (copy-out loop), ragged last tiles, origin and
    non-finite rows included; at an lmax without a plan they run the next
    form down (tma2 -> tma -> copy-out)."""
    assert shm.eval_variant_count() > TMA2_VARIANT
    pts = _tma_test_points(n)
    p = torch.from_numpy(pts).cuda()
    has_tma = lmax % 2 == 1 and lmax <= 9
    has_tma2 = lmax in (3, 5, 7, 9)
    expect = {TMA_VARIANT: "phased-hybrid-tma-128" if has_tma else "phased-hybrid-128" if lmax <= 9 else "phased-128",
              TMA2_VARIANT: "phased-hybrid-tma2-128" if has_tma2 else "phased-hybrid-tma-128" if has_tma else
              "phased-hybrid-128" if lmax <= 9 else "phased-128"}[variant]
    try:
        shm.set_eval_variant(lmax, torch.float64, variant)
        name = shm.eval_variant(lmax, torch.float64)
        assert name == expect, (lmax, name)
        out = torch.full((n, (lmax + 1) ** 2), 7.0, dtype=torch.float64, device="cuda")
        shm.eval_sh(p, lmax, out=out)
        shm.set_eval_variant(lmax, torch.float64, COPY_OUT_VARIANT)
        ref = shm.eval_sh(p, lmax)
        torch.cuda.synchronize()
        assert torch.equal(torch.nan_to_num(out, nan=5.0), torch.nan_to_num(ref, nan=5.0)), (lmax, n)
        assert torch.equal(torch.isnan(out), torch.isnan(ref))
    finally:
        shm.set_eval_variant(lmax, torch.float64, -1)


@pytest.mark.parametrize("variant", sorted(TMA_EMU_VARIANTS))
@pytest.mark.parametrize("lmax", [1, 2, 3, 5, 7, 9, 11])
@pytest.mark.parametrize("n", [129, 4099, 200_003])
def test_tma_integer_pipe_variants_with_declined_products(variant, lmax, n):
    """phased-hybrid-tma-emu-*-128 take the binary64 products of the hybrid
    rows' m = 0, 1 columns on the integer pipes; the integer product declines
    zero operands, so a point with xb, yb or zb exactly 0 has its row written
    again by the FP64 code after the tile's TMA stores.  Such points are put
    in many tiles (one tile made only of them, the ragged last tile, next to
    origin and non-finite rows): the rows are the bits of phased-hybrid-128."""
    pts = _tma_test_points(n)
    rng = np.random.default_rng(20510 + n)
    idx = rng.choice(n, size=max(n // 40, 3), replace=False)
    for j, i in enumerate(idx):
        pts[i, j % 3] = 0.0                        # xb, yb or zb exactly 0
    if n >= 512:
        pts[256:384, 1] = 0.0                      # a whole tile on the xz-plane
    pts[n - 2] = [0.0, 3.0, 0.0]                   # on an axis, in the last tile
    p = torch.from_numpy(pts).cuda()
    has_tma = lmax % 2 == 1 and lmax <= 9
    expect = TMA_EMU_VARIANTS[variant] if has_tma else "phased-hybrid-128" if lmax <= 9 else "phased-128"
    try:
        shm.set_eval_variant(lmax, torch.float64, variant)
        assert shm.eval_variant(lmax, torch.float64) == expect, lmax
        out = torch.full((n, (lmax + 1) ** 2), 7.0, dtype=torch.float64, device="cuda")
        shm.eval_sh(p, lmax, out=out)
        shm.set_eval_variant(lmax, torch.float64, COPY_OUT_VARIANT)
        ref = shm.eval_sh(p, lmax)
        torch.cuda.synchronize()
        assert torch.equal(torch.nan_to_num(out, nan=5.0), torch.nan_to_num(ref, nan=5.0)), (lmax, n)
        assert torch.equal(torch.isnan(out), torch.isnan(ref))
    finally:
        shm.set_eval_variant(lmax, torch.float64, -1)


@pytest.mark.parametrize("variant", [TMA_VARIANT, TMA2_VARIANT, *sorted(TMA_EMU_VARIANTS)])
def test_tma_variant_next_to_other_allocations(variant):
    """The TMA stores of the last (ragged) tile stop at row n: the bytes
    after the output, inside the same allocation, are left untouched."""
    n = 1000
    pts = inputs.random_sphere_points(n, stream="tests", with_axes=False)
    p = torch.from_numpy(pts).cuda()
    buf = torch.full((n + 300, 100), -3.0, dtype=torch.float64, device="cuda")
    try:
        shm.set_eval_variant(9, torch.float64, variant)
        shm.eval_sh(p, 9, out=buf[:n])
        torch.cuda.synchronize()
        assert torch.all(buf[n:] == -3.0)
        shm.set_eval_variant(9, torch.float64, COPY_OUT_VARIANT)
        assert torch.equal(buf[:n], shm.eval_sh(p, 9))
    finally:
        shm.set_eval_variant(9, torch.float64, -1)


def test_bad_arguments_launch_nothing():
    from cuda.bindings import runtime as rt
    L = shm.lib()
    p = torch.zeros((20, 3), dtype=torch.float64, device="cuda")
    # an exact 10-row output allocation (not a slice of a larger pool block)
    err, raw = rt.cudaMalloc(10 * 100 * 8)
    assert err == rt.cudaError_t.cudaSuccess
    try:
        out = torch.full((10, 100), 7.0, dtype=torch.float64, device="cuda")
        rt.cudaMemcpy(raw, out.data_ptr(), 8000, rt.cudaMemcpyKind.cudaMemcpyDeviceToDevice)
        # n = 20 rows do not fit the 10-row allocation: rejected on the host
        assert L.shm_eval(p.data_ptr(), 20, 9, 1, int(raw), None) == 1
        assert b"past the end" in L.shm_last_error()
        # host memory passed as device memory
        host = np.zeros((10, 3))
        assert L.shm_eval(host.ctypes.data, 10, 9, 1, int(raw), None) == 1
        # overlapping input and output
        assert L.shm_eval(int(raw), 10, 9, 1, int(raw) + 64, None) == 1
        torch.cuda.synchronize()
        back = torch.empty((10, 100), dtype=torch.float64, device="cuda")
        rt.cudaMemcpy(back.data_ptr(), raw, 8000, rt.cudaMemcpyKind.cudaMemcpyDeviceToDevice)
        assert torch.all(back == 7.0)
    finally:
        rt.cudaFree(raw)


def test_host_buffer_entry_point(oracle_mod):
    pts = inputs.random_sphere_points(30_000, stream="tests")
    n = pts.shape[0]
    for pinned in (True, False):
        hin = torch.from_numpy(pts)
        hout = torch.empty((n, 100), dtype=torch.float64)
        if pinned:
            hin, hout = hin.pin_memory(), hout.pin_memory()
        ws = torch.empty(shm.eval_host_workspace_size(9, torch.float64, 7000), dtype=torch.uint8, device="cuda")
        shm.eval_host(hin, 9, hout, ws)
        torch.cuda.synchronize()
        assert_normwise(hout.numpy(), oracle_mod.real_sh(pts, 9), TOL_F64, f"host entry pinned={pinned}")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lmax", [0, 4, 9])
def test_every_launch_variant(oracle_mod, dtype, lmax):
    pts = inputs.random_sphere_points(3001, stream="tests")
    if dtype == torch.float32:
        pts = pts.astype(np.float32).astype(np.float64)
    ref = oracle_mod.real_sh(pts, lmax)
    tol = TOL_F64 if dtype == torch.float64 else TOL_F32
    try:
        for v in range(shm.eval_variant_count()):
            shm.set_eval_variant(lmax, dtype, v)
            got = gpu_eval(pts, lmax, dtype=dtype)
            assert_normwise(got, ref, tol, f"variant {shm.eval_variant(lmax, dtype)}")
    finally:
        shm.set_eval_variant(lmax, dtype, -1)


@pytest.mark.parametrize("lmax", [1, 6, 9])
def test_fp64_variants_are_bitwise_identical(lmax, oracle_mod):
    """Every native FP64 launch variant runs the same operations on the same
    operands: bitwise identical rows.  The hybrid variants share the FP64 code
    for the m = 0, 1 columns (bitwise identical there) and run m >= 2 in
    float-float (within the FP64 tolerance of the oracle)."""
    pts = np.concatenate([inputs.random_sphere_points(5001, stream="tests"), inputs.edge_points()])
    p = torch.from_numpy(pts).cuda()
    outs = {}
    try:
        for v in range(shm.eval_variant_count()):
            shm.set_eval_variant(lmax, torch.float64, v)
            outs[shm.eval_variant(lmax, torch.float64)] = shm.eval_sh(p, lmax).clone()
    finally:
        shm.set_eval_variant(lmax, torch.float64, -1)
    torch.cuda.synchronize()
    base = torch.nan_to_num(outs["staged-128"], nan=7.0)
    l = np.array([int(np.sqrt(k)) for k in range((lmax + 1) ** 2)])
    m = np.arange((lmax + 1) ** 2) - l * l - l
    low_m = torch.from_numpy(np.abs(m) <= 1).cuda()
    finite = np.all(np.isfinite(pts), axis=1) & np.all(np.abs(pts) < 1e300, axis=1)
    ref = oracle_mod.real_sh(pts[finite], lmax)
    hyb = torch.nan_to_num(outs["hybrid-64"], nan=7.0)
    for name, o in outs.items():
        o = torch.nan_to_num(o, nan=7.0)
        if "hybrid" in name:
            assert torch.equal(o, hyb), name          # every hybrid variant: the same operations
            assert torch.equal(o[:, low_m], base[:, low_m]), name
            assert_normwise(o.cpu().numpy()[finite], ref, TOL_F64, name)
        else:
            assert torch.equal(o, base), name


def test_autotune_keeps_results_correct(oracle_mod):
    ms = shm.autotune(9, torch.float64, 1 << 16)
    assert ms > 0 and shm.eval_variant(9, torch.float64)
    pts = inputs.random_sphere_points(2000, stream="tests")
    assert_normwise(gpu_eval(pts, 9), oracle_mod.real_sh(pts, 9), TOL_F64, "after autotune")
    shm.set_eval_variant(9, torch.float64, -1)


def test_dft_grid_fp64_full_size_sampled(oracle_mod, capsys):
    """192^3 grid (7.08M points, 5.7 GB out) in every launch configuration the
    tuner may pick for bench.py: sampled rows against the oracle; the addition
    theorem on every row."""
    pts = inputs.dft_grid_points(192)
    p = torch.from_numpy(pts).cuda()
    g = inputs.rng("tests", 77)
    n = pts.shape[0]
    rows = np.unique(np.concatenate([np.arange(256), np.arange(n - 300, n), g.integers(0, n, 20000)]))
    ref = oracle_mod.real_sh(pts[rows], 9)
    rows_t = torch.from_numpy(rows).cuda()
    try:
        for v in range(shm.eval_variant_count()):
            shm.set_eval_variant(9, torch.float64, v)
            out = shm.eval_sh(p, 9)
            torch.cuda.synchronize()
            got = out[rows_t].cpu().numpy()
            if shm.eval_variant(9, torch.float64) == "phased-hybrid-tma-128":  # the variant bench.py times
                with capsys.disabled():
                    print("\nFP64 192^3 grid sample (phased-hybrid-tma-128), normwise error per l (max/mean):",
                          per_l_report(normwise_err(got, ref)))
            assert_normwise(got, ref, TOL_F64, f"192^3 grid sample, variant {v}")
            for l in range(10):
                s = (out[:, l * l:(l + 1) ** 2] ** 2).sum(dim=1)
                dev = (s - (2 * l + 1) / (4 * np.pi)).abs().max().item()
                assert dev <= 4 * TOL_F64 * (2 * l + 1) / (4 * np.pi), (v, l, dev)
            del out
    finally:
        shm.set_eval_variant(9, torch.float64, -1)


def test_fp32_grid_and_sphere_per_l_report(oracle_mod, capsys):
    """The FP32 workload: the 192^3 grid (sampled) and 1M random-sphere points
    (all rows) against the oracle at the upcast FP32 inputs, error per l."""
    sph = inputs.random_sphere_points(1 << 20, stream="sphere32", with_axes=False).astype(np.float32)
    got = gpu_eval(sph, 9, dtype=torch.float32)
    err = normwise_err(got, oracle_mod.real_sh(sph.astype(np.float64), 9))
    with capsys.disabled():
        print("\nFP32 1M sphere, normwise error per l (max/mean):", per_l_report(err))
    assert float(err.max()) <= TOL_F32
    grid = inputs.dft_grid_points(192).astype(np.float32)
    p = torch.from_numpy(grid).cuda()
    out = shm.eval_sh(p, 9)
    torch.cuda.synchronize()
    rows = np.unique(inputs.rng("tests", 78).integers(0, grid.shape[0], 20000))
    got = out[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert_normwise(got, oracle_mod.real_sh(grid[rows].astype(np.float64), 9), TOL_F32, "FP32 grid sample")


# ---------------------------------------------------------------- beyond l = 9

def tol_high_l(lmax, base):
    """Tolerance above the paper's l <= 9: rounding in the l-steps of the
    recurrence grows about linearly with l, so the l <= 9 bound is scaled by
    l / 9."""
    return base * max(1.0, lmax / 9.0)


@pytest.mark.parametrize("lmax", [10, 12, 16])
def test_high_l_every_variant(oracle_mod, lmax, capsys):
    pts = np.concatenate([inputs.random_sphere_points(3001, stream="tests"), inputs.edge_points()[:14]])
    ref = oracle_mod.real_sh(pts, lmax)
    worst = {}
    try:
        for dtype, base in ((torch.float64, TOL_F64), (torch.float32, TOL_F32)):
            ref_d = ref if dtype == torch.float64 else oracle_mod.real_sh(pts.astype(np.float32).astype(np.float64), lmax)
            for v in range(shm.eval_variant_count()):
                shm.set_eval_variant(lmax, dtype, v)
                got = gpu_eval(pts, lmax, dtype=dtype)
                err = normwise_err(got, ref_d)
                worst[(str(dtype), shm.eval_variant(lmax, dtype))] = float(err.max())
                assert_normwise(got, ref_d, tol_high_l(lmax, base), f"l={lmax} {dtype} {shm.eval_variant(lmax, dtype)}")
    finally:
        shm.set_eval_variant(lmax, torch.float64, -1)
        shm.set_eval_variant(lmax, torch.float32, -1)
    with capsys.disabled():
        print(f"\nlmax={lmax} worst normwise errors:", {k: f"{v:.2e}" for k, v in worst.items()})
