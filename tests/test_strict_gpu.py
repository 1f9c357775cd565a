"""SHM_STRICT_FP64: every FP64 value computed in binary64 arithmetic (no
float-float), on the real, complex, spinor and angular paths and the host
entry point.  The strict rows are the all-binary64 rows of sh_row: bitwise
equal to the staged-128 variant (the plain copy-out kernel of the same
operations) and within 1e-13 of the l-shell norm of the oracle (Sec. II
Eq. 5-6; the paper works at machine precision in double, Sec. IV)."""
import math

import numpy as np
import pytest

from helpers import TOL_F64, assert_normwise, normwise_err, per_l_max, per_l_report

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2510_05282_b300 as shm  # noqa: E402
from paper_2510_05282_b300 import inputs  # noqa: E402

STAGED_128 = 0
STRICT_VARIANTS = ("staged-128", "staged-64", "staged-256", "direct-128", "direct-256", "phased-64", "phased-128",
                   "rows-tma-64", "rows-tma-32", "rows-tma-emu-o-32", "rows-tma-emu-os-32")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_05282_b300 import build
    build.build()
    shm.lib()


def _points(n):
    """Random-sphere points with the origin (both zero signs), poles, a tiny
    and a huge radius and a NaN row placed in the first, a middle and the
    ragged last tile where n allows."""
    pts = inputs.random_sphere_points(n, stream="tests", with_axes=False)
    special = {0: [0.0, 0.0, 0.0], 3: [0.0, 0.0, -2.5], 7: [1e-30, 0.0, 0.0], n // 2: [-0.0, 0.0, -0.0],
               n - 2: [3e29, -1e29, 2e29], n - 1: [np.nan, 1.0, 0.0]}
    if n > 16:
        for i, v in special.items():
            pts[i] = v
    return pts


def _staged128(p, lmax):
    try:
        shm.set_eval_variant(lmax, torch.float64, STAGED_128)
        return shm.eval_sh(p, lmax)
    finally:
        shm.set_eval_variant(lmax, torch.float64, -1)


def _same(a, b):
    return torch.equal(torch.nan_to_num(a, nan=7.0), torch.nan_to_num(b, nan=7.0)) and \
        torch.equal(torch.isnan(a), torch.isnan(b))


@pytest.mark.parametrize("lmax", list(range(10)) + [11, 16])
@pytest.mark.parametrize("n", [1, 63, 64, 65, 4099])
def test_strict_rows_bitwise_equal_staged128_and_oracle(oracle_mod, lmax, n):
    pts = _points(n)
    p = torch.from_numpy(pts).cuda()
    got = shm.eval_sh(p, lmax, strict=True)
    ref = _staged128(p, lmax)
    torch.cuda.synchronize()
    assert _same(got, ref), (lmax, n, shm.eval_variant(lmax, torch.float64, strict=True))
    fin = np.all(np.isfinite(pts), axis=1)
    tol = TOL_F64 * max(1.0, lmax / 9.0)
    assert_normwise(got.cpu().numpy()[fin], oracle_mod.real_sh(pts[fin], lmax), tol, f"strict lmax={lmax} n={n}")


@pytest.mark.parametrize("lmax", [1, 4, 9])
def test_every_strict_variant_is_bitwise_the_same(lmax):
    pts = _points(3001)
    p = torch.from_numpy(pts).cuda()
    ref = _staged128(p, lmax)
    seen = set()
    try:
        for v in range(shm.eval_variant_count()):
            try:
                shm.set_eval_variant(lmax, torch.float64, v, strict=True)
            except shm.ShmError as e:          # a hybrid variant: refused for strict calls
                assert e.status == 1
                continue
            name = shm.eval_variant(lmax, torch.float64, strict=True)
            seen.add(name)
            assert name in STRICT_VARIANTS, name
            out = torch.full_like(ref, 3.0)
            shm.eval_sh(p, lmax, out=out, strict=True)
            torch.cuda.synchronize()
            assert _same(out, ref), name
    finally:
        shm.set_eval_variant(lmax, torch.float64, -1, strict=True)
    assert "staged-64" in seen and len(seen) >= (9 if lmax % 2 else 7)


def test_strict_flag_does_not_change_the_default_rows():
    """The default (hybrid) rows and the strict rows are separate choices: a
    strict call leaves the default variant alone, and FP32 ignores the flag."""
    pts = _points(2000)
    p = torch.from_numpy(pts).cuda()
    default = shm.eval_sh(p, 9)
    strict = shm.eval_sh(p, 9, strict=True)
    again = shm.eval_sh(p, 9)
    torch.cuda.synchronize()
    assert _same(default, again)
    assert "hybrid" in shm.eval_variant(9, torch.float64)
    assert "hybrid" not in shm.eval_variant(9, torch.float64, strict=True)
    # the m = 0, 1 columns of the hybrid rows are the binary64 ones
    l = np.array([int(math.isqrt(k)) for k in range(100)])
    m = np.arange(100) - l * l - l
    low = torch.from_numpy(np.abs(m) <= 1).cuda()
    assert _same(default[:, low], strict[:, low])
    p32 = p.float()
    assert _same(shm.eval_sh(p32, 9), shm.eval_sh(p32, 9, strict=True))


def test_strict_rows_tma_next_to_other_allocations():
    """The TMA stores of the last (ragged) tile stop at row n."""
    n = 1000
    p = torch.from_numpy(_points(n)).cuda()
    buf = torch.full((n + 300, 100), -3.0, dtype=torch.float64, device="cuda")
    shm.eval_sh(p, 9, out=buf[:n], strict=True)
    torch.cuda.synchronize()
    assert torch.all(buf[n:] == -3.0)
    assert _same(buf[:n], _staged128(p, 9))


def test_strict_full_grid_sampled(oracle_mod, capsys):
    """The 192^3 grid in the launch configuration bench.py times for its
    headline (strict rows, default variant): sampled rows against the oracle,
    the addition theorem on every row."""
    pts = inputs.dft_grid_points(192)
    p = torch.from_numpy(pts).cuda()
    out = shm.eval_sh(p, 9, strict=True)
    torch.cuda.synchronize()
    n = pts.shape[0]
    rows = np.unique(np.concatenate([np.arange(256), np.arange(n - 300, n),
                                     inputs.rng("tests", 77).integers(0, n, 20000)]))
    got = out[torch.from_numpy(rows).cuda()].cpu().numpy()
    ref = oracle_mod.real_sh(pts[rows], 9)
    err = normwise_err(got, ref)
    with capsys.disabled():
        print(f"\nFP64 strict ({shm.eval_variant(9, torch.float64, strict=True)}) 192^3 grid sample, "
              "normwise error per l (max/mean):", per_l_report(err))
    assert_normwise(got, ref, TOL_F64, "strict 192^3 sample")
    for l in range(10):
        s = (out[:, l * l:(l + 1) ** 2] ** 2).sum(dim=1)
        dev = (s - (2 * l + 1) / (4 * np.pi)).abs().max().item()
        assert dev <= 4 * TOL_F64 * (2 * l + 1) / (4 * np.pi), (l, dev)


def test_strict_random_sphere_error_report(oracle_mod, capsys):
    pts = inputs.random_sphere_points(65_536)
    got = shm.eval_sh(torch.from_numpy(pts).cuda(), 9, strict=True).cpu().numpy()
    err = normwise_err(got, oracle_mod.real_sh(pts, 9))
    with capsys.disabled():
        print("\nFP64 strict random sphere 65,600, normwise error per l (max/mean):", per_l_report(err))
    # all-binary64 rows: within a few 1e-14 of the shell norm at every l
    assert max(per_l_max(err)) <= 3e-14


def test_strict_host_entry_point():
    pts = _points(30_000)
    n = pts.shape[0]
    hin = torch.from_numpy(pts).pin_memory()
    hout = torch.empty((n, 100), dtype=torch.float64).pin_memory()
    ws = torch.empty(shm.eval_host_workspace_size(9, torch.float64, 7000), dtype=torch.uint8, device="cuda")
    shm.eval_host(hin, 9, hout, ws, strict=True)
    torch.cuda.synchronize()
    ref = shm.eval_sh(torch.from_numpy(pts).cuda(), 9, strict=True).cpu()
    assert _same(hout, ref)


def test_strict_autotune():
    ms = shm.autotune(9, torch.float64, 1 << 16, strict=True)
    try:
        assert ms > 0
        assert shm.eval_variant(9, torch.float64, strict=True) in STRICT_VARIANTS
        p = torch.from_numpy(_points(2000)).cuda()
        assert _same(shm.eval_sh(p, 9, strict=True), _staged128(p, 9))
    finally:
        shm.set_eval_variant(9, torch.float64, -1, strict=True)


# ------------------------------------------------------------------ complex

def _cx_check(got, ref, tol, what):
    l = np.array([int(math.isqrt(k)) for k in range(ref.shape[1])])
    nb = np.sqrt((2 * l + 1) / (4 * np.pi))
    err = np.abs(got.astype(np.complex128) - ref) / nb
    assert not np.isnan(err).any(), what
    assert float(err.max()) <= tol, f"{what}: {float(err.max()):.3e}"


@pytest.mark.parametrize("lmax", [0, 1, 4, 9])
@pytest.mark.parametrize("n", [1, 63, 65, 5003])
def test_strict_complex(oracle_mod, lmax, n):
    pts = np.concatenate([inputs.random_sphere_points(n, stream="tests", with_axes=False), inputs.edge_points()])
    p = torch.from_numpy(pts).cuda()
    Y = shm.eval_complex(p, lmax, strict=True).cpu().numpy()
    fin = np.all(np.isfinite(pts), axis=1)
    _cx_check(Y[fin], oracle_mod.complex_sh(pts[fin], lmax), TOL_F64, f"strict complex lmax={lmax}")
    # Y_l^0 = R_l^0 bitwise (the same binary64 operations), imaginary part exactly 0
    R = shm.eval_sh(p, lmax, strict=True).cpu().numpy()
    for l in range(lmax + 1):
        k = l * l + l
        assert np.array_equal(Y[fin, k].real, R[fin, k]) and np.all(Y[fin, k].imag == 0)
    assert np.all(np.isnan(Y[~fin, 1:].real))


# ------------------------------------------------------------------- spinor

@pytest.mark.parametrize("lmax", [0, 1, 4, 9])
@pytest.mark.parametrize("n", [1, 63, 65, 5003])
def test_strict_spinor(oracle_mod, lmax, n):
    pts = np.concatenate([inputs.random_sphere_points(n, stream="tests", with_axes=False), inputs.edge_points()])
    pts = pts[np.all(np.isfinite(pts), axis=1)]
    got = shm.eval_spinor(torch.from_numpy(pts).cuda(), lmax, strict=True).cpu().numpy()
    ref = oracle_mod.spinor_sh(pts, lmax)
    ls = np.array([l for l in range(lmax + 1) for _ in range(4 * l + 2)])
    err = np.abs(got.astype(np.complex128) - ref) / np.sqrt((2 * ls + 1) / (4 * np.pi))[None, :, None]
    assert float(err.max()) <= TOL_F64, float(err.max())


# ------------------------------------------------------------------- angles

@pytest.mark.parametrize("lmax", [0, 5, 9])
def test_strict_angles(oracle_mod, lmax):
    g = inputs.rng("tests", 31)
    n = 20000
    theta = np.arccos(g.uniform(-1, 1, n))
    phi = g.uniform(-np.pi, np.pi, n)
    theta[:4] = [0.0, np.pi, np.pi / 2, 1e-9]
    ang = np.stack([theta, phi], axis=1)
    got = shm.eval_angles(torch.from_numpy(ang).cuda(), lmax, strict=True).cpu().numpy()
    assert_normwise(got, oracle_mod.real_sh_angles(theta, phi, lmax), TOL_F64, "strict angles")
    # unaligned output: the copy-out kernel, the same rows bitwise
    buf = torch.empty(n * (lmax + 1) ** 2 + 1, dtype=torch.float64, device="cuda")
    out = buf[1:].view(n, (lmax + 1) ** 2)
    shm.eval_angles(torch.from_numpy(ang).cuda(), lmax, out=out, strict=True)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), got)


def test_integer_pipe_multiply_is_bitwise_dmul():
    """dmul_int, the binary64 product on the integer pipes, against the DMUL
    instruction on 2^26 generated pairs (ties, all-ones significands, the
    edges of the normal range, zeros and subnormals among them): every
    product it returns is DMUL's bit for bit, and it declines the operands
    outside its range (which the rows then compute with DMUL)."""
    mismatches, declined = shm.probe_dmul(1 << 26, seed=2025)
    assert mismatches == 0
    assert 0 < declined < (1 << 26) // 4


@pytest.mark.parametrize("lmax", [1, 3, 5, 7, 9, 11, 15])
def test_emulated_product_variants_on_awkward_points(oracle_mod, lmax):
    """The rows-tma-emu variants on points whose rows contain exact zeros
    (axes, x = y diagonals), tiny and huge radii and powers of x + iy that
    underflow (y ~ 1e-200): bitwise the all-FP64 rows, through the per-point
    fallback where the integer multiply declines."""
    pts = np.concatenate([_points(5000), inputs.edge_points(),
                          np.array([[1.0, 1.0, 0.3], [2.0, -2.0, 1.0], [1.0, 1e-200, 0.5], [1e-160, 1.0, 1e-170],
                                    [3.0, 0.0, 0.0], [0.0, 0.0, 7.0], [1e-300, 1e-300, 1e-300]])])
    p = torch.from_numpy(pts).cuda()
    ref = _staged128(p, lmax)
    try:
        for name in ("rows-tma-emu-o-32", "rows-tma-emu-os-32"):
            for i in range(shm.eval_variant_count()):
                try:
                    shm.set_eval_variant(lmax, torch.float64, i, strict=True)
                except shm.ShmError:
                    continue
                if shm.eval_variant(lmax, torch.float64, strict=True) == name:
                    break
            assert shm.eval_variant(lmax, torch.float64, strict=True) == name
            out = torch.full_like(ref, 3.0)
            shm.eval_sh(p, lmax, out=out, strict=True)
            torch.cuda.synchronize()
            assert _same(out, ref), name
    finally:
        shm.set_eval_variant(lmax, torch.float64, -1, strict=True)


def _spinor_terms(lmax):
    """(ka, kb, cre, cim, im_zero) of every output component q = 2 spinor + c
    of Eq. 7, with the coefficients formed by the same binary64 operations
    (a correctly rounded quotient and square root, exact sign changes, one
    product by 1/sqrt2)."""
    rs2 = 0.70710678118654752440
    terms = []
    for l in range(lmax + 1):
        for s, tj in ((-1, 2 * l - 1), (1, 2 * l + 1)):
            if tj < 0:
                continue
            for t in range(tj + 1):
                tmj = 2 * t - tj
                for c in (0, 1):
                    m = (tmj - 1) // 2 if c == 0 else (tmj + 1) // 2
                    num = 2 * l + s * tmj + 1 if c == 0 else 2 * l - s * tmj + 1
                    a = math.sqrt(float(num) / float(2 * (2 * l + 1)))
                    if c == 0 and s < 0:
                        a = -a
                    mu = abs(m)
                    if mu > l:
                        a, mu = 0.0, 0
                    if mu == 0:
                        cre, cim = a, 0.0
                    elif m > 0:
                        cre = cim = (-a if m & 1 else a) * rs2
                    else:
                        cre = a * rs2
                        cim = -cre
                    terms.append((l * l + l + mu, l * l + l - mu, cre, cim, mu == 0))
    return terms


@pytest.mark.parametrize("lmax", [1, 4, 9])
def test_strict_spinor_is_coefficient_times_strict_row_bitwise(lmax):
    """Every strict spinor component is one binary64 product coefficient x
    real harmonic of the strict row (Eq. 7 with Y from R): the GPU values
    equal numpy's IEEE products of the same operands bit for bit, whichever
    pipe computes the product; points on the axes and poles (zero harmonics)
    included."""
    pts = np.concatenate([inputs.random_sphere_points(3001, stream="tests", with_axes=False), inputs.edge_points()])
    pts = pts[np.all(np.isfinite(pts), axis=1) & (np.linalg.norm(pts, axis=1) > 0)]
    p = torch.from_numpy(pts).cuda()
    got = shm.eval_spinor(p, lmax, strict=True).cpu().numpy()       # [n, 2 L2, 2] complex
    R = shm.eval_sh(p, lmax, strict=True).cpu().numpy()
    terms = _spinor_terms(lmax)
    assert len(terms) == 4 * (lmax + 1) ** 2
    flat = got.reshape(got.shape[0], -1)                            # component q = 2 spinor + c
    for q, (ka, kb, cre, cim, imz) in enumerate(terms):
        re = cre * R[:, ka]
        im = np.zeros_like(re) if imz else cim * R[:, kb]
        assert np.array_equal(flat[:, q].real.view(np.int64), re.view(np.int64)), (lmax, q)
        assert np.array_equal(flat[:, q].imag.view(np.int64), im.view(np.int64)), (lmax, q)
