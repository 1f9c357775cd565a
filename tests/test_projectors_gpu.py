"""GPU parity of shm_projectors against the oracle's fused projectors.

Tolerance per value: |P_gpu - P_oracle| <= tol * F_sl * sqrt((2l+1)/4pi) with
F_sl = max |f_{s,l}| over the table, i.e. normwise against the size of the
product's l-shell.  FP64: tol = 1e-13.  FP32: tol = 2e-6, the FP32 bound
of the plain evaluator (see PROJ_TOL_F32 below).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2510_05282_b300 as shm  # noqa: E402
from paper_2510_05282_b300 import inputs  # noqa: E402

PROJ_TOL_F64 = 1e-13
# FP32: table values rounded to float (0.5 ulp), Lagrange weights and the
# 4-term sum in FP32 (a few ulps of the local table magnitude), the log-grid
# index to ~1e-5 (which moves f by ~1e-5 * dlog * |d ln f / d ln r| ~ 1e-7
# relative), and the FP32 harmonics (<= 1e-6 of the l-shell norm at l = 9):
# measured worst 8.7e-7 on the 512-atom problem, within the 2e-6 FP32 bound
# of the plain evaluator.
PROJ_TOL_F32 = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_05282_b300 import build
    build.build()
    shm.lib()


def small_problem(extra=0, **kw):
    args = dict(n_atoms=6, box=6.0, h=0.25, rc_range=(1.0, 2.0), n_species=3,
                lmax_choices=(2, 3, 4), n_rad=200, r_min=1e-3, r_max=3.0, extra=extra)
    args.update(kw)
    return inputs.projector_problem(**args)


def value_scale(prob):
    """Per-value scale F_sl * sqrt((2l+1)/4pi)."""
    F = np.abs(prob.radial).max(axis=2)            # [S, lstride]
    out = np.empty(prob.n_values)
    for a in range(prob.n_atoms):
        s = prob.atom_species[a]
        L = int(prob.species_lmax[s])
        n = int(prob.point_offsets[a + 1] - prob.point_offsets[a])
        ls = np.array([int(math.isqrt(k)) for k in range((L + 1) ** 2)])
        row = F[s, ls] * np.sqrt((2 * ls + 1) / (4 * np.pi))
        out[prob.out_offsets[a]:prob.out_offsets[a + 1]] = np.tile(row, n)
    return out


def check(prob, got, ref, tol, what):
    scale = value_scale(prob)
    err = np.abs(got.astype(np.float64) - ref) / scale
    worst = float(err.max()) if err.size else 0.0
    assert not np.isnan(err).any(), what
    assert worst <= tol, f"{what}: max scaled error {worst:.3e} > {tol:.1e}"
    return worst


def run(prob, dtype):
    d = shm.DeviceProjectors(prob)
    ws = d.workspace(dtype)
    out = shm.projectors(d, dtype, workspace=ws)
    torch.cuda.synchronize()
    assert shm.projectors_check(ws) == 0
    return out.cpu().numpy()


@pytest.mark.parametrize("extra", [0, 1, 2])
def test_small_fp64(oracle_mod, extra):
    prob = small_problem(extra)
    check(prob, run(prob, torch.float64), oracle_mod.projectors(prob), PROJ_TOL_F64, "FP64 small")


@pytest.mark.parametrize("extra", [0, 1])
def test_small_fp32(oracle_mod, extra):
    prob = small_problem(extra)
    check(prob, run(prob, torch.float32), oracle_mod.projectors(prob), PROJ_TOL_F32, "FP32 small")


@pytest.mark.parametrize("dtype,tol", [(torch.float64, PROJ_TOL_F64), (torch.float32, PROJ_TOL_F32)])
def test_every_lmax_up_to_9(oracle_mod, dtype, tol):
    prob = small_problem(5, n_atoms=10, n_species=10, lmax_choices=tuple(range(10)))
    check(prob, run(prob, dtype), oracle_mod.projectors(prob), tol, f"lmax 0..9 {dtype}")


@pytest.mark.parametrize("n_rad", [4, 5])
@pytest.mark.parametrize("dtype,tol", [(torch.float64, PROJ_TOL_F64), (torch.float32, PROJ_TOL_F32)])
def test_shortest_radial_tables(oracle_mod, n_rad, dtype, tol):
    """Tables of 4 and 5 nodes: every interval's stencil is clamped at an end
    (the stencil start i0 is 0 or n_rad - 4 throughout), so each offset of
    the interval within its stencil, 0 to 3, occurs."""
    prob = small_problem(11, n_rad=n_rad, r_min=0.05, r_max=2.5)
    check(prob, run(prob, dtype), oracle_mod.projectors(prob), tol, f"n_rad {n_rad} {dtype}")


def relist(prob):
    """Rebuild the sphere lists and output offsets after moving atoms."""
    off, idx = inputs.sphere_lists(prob.atom_pos, prob.atom_rc, prob.ng, prob.h, prob.box)
    prob.point_offsets, prob.point_index = off, idx
    nh = (prob.atom_lmax().astype(np.int64) + 1) ** 2
    prob.out_offsets = np.concatenate([[0], np.cumsum(np.diff(off) * nh)]).astype(np.int64)
    return off, nh


@pytest.mark.parametrize("dtype,tol", [(torch.float64, PROJ_TOL_F64), (torch.float32, PROJ_TOL_F32)])
def test_atoms_outside_the_primary_box(oracle_mod, dtype, tol):
    """Atom coordinates shifted by whole boxes: raw displacements up to ~5
    boxes, so the minimum image subtracts several boxes (and one box where
    |d| is between half a box and 1.5 boxes)."""
    prob = small_problem(4)
    shifts = np.array([[2, 0, -1], [-3, 1, 0], [0, 0, 5], [1, -1, 1], [0, 0, 0], [-1, -2, 3]], dtype=np.float64)
    prob.atom_pos = prob.atom_pos + shifts[:prob.n_atoms] * prob.box
    relist(prob)
    check(prob, run(prob, dtype), oracle_mod.projectors(prob), tol, f"shifted atoms {dtype}")


def test_atom_on_a_grid_point_uses_origin_rule(oracle_mod):
    prob = small_problem(3)
    # move atom 0 exactly onto grid point (8, 9, 10): its own row is at r = 0
    prob.atom_pos[0] = np.array([8, 9, 10], dtype=np.float64) * prob.h
    off, nh = relist(prob)
    for dtype, tol in ((torch.float64, PROJ_TOL_F64), (torch.float32, PROJ_TOL_F32)):
        got = run(prob, dtype)
        ref = oracle_mod.projectors(prob)
        check(prob, got, ref, tol, f"origin {dtype}")
        g0 = (8 * prob.ng + 9) * prob.ng + 10
        p = int(np.nonzero(prob.point_index[:off[1]] == g0)[0][0])
        L2 = int(nh[0])
        row = got[p * L2:(p + 1) * L2]
        assert np.all(row[1:] == 0.0)


def test_empty_atoms_and_no_points():
    prob = small_problem(4)
    # atom 2 keeps no points
    a = 2
    cut = prob.point_offsets[a + 1] - prob.point_offsets[a]
    idx = np.concatenate([prob.point_index[:prob.point_offsets[a]], prob.point_index[prob.point_offsets[a + 1]:]])
    off = prob.point_offsets.copy()
    off[a + 1:] -= cut
    prob.point_index, prob.point_offsets = idx, off
    nh = (prob.atom_lmax().astype(np.int64) + 1) ** 2
    prob.out_offsets = np.concatenate([[0], np.cumsum(np.diff(off) * nh)]).astype(np.int64)
    import oracle
    check(prob, run(prob, torch.float64), oracle.projectors(prob), PROJ_TOL_F64, "empty atom")


def test_inconsistent_problem_sets_error_bits_without_faulting():
    prob = small_problem(6)
    d = shm.DeviceProjectors(prob)
    ws = d.workspace(torch.float64)
    # (a) a grid index out of range: flagged, the row is zeroed
    d.point_index[5] = prob.ng ** 3 + 7
    out = shm.projectors(d, torch.float64, workspace=ws)
    assert shm.projectors_check(ws) & 4
    # (b) output offsets inconsistent with the row widths: that atom is skipped
    d.point_index[5] = int(prob.point_index[5])
    d.out_offsets[2] += 1
    out = shm.projectors(d, torch.float64, workspace=ws)
    assert shm.projectors_check(ws) & 8
    # (c) a species index out of range
    d.out_offsets[2] -= 1
    d.atom_species[1] = 99
    out = shm.projectors(d, torch.float64, workspace=ws)
    assert shm.projectors_check(ws) & 2
    # (d) point offsets running past n_points
    d.atom_species[1] = int(prob.atom_species[1])
    d.point_offsets[3] = prob.n_points + 1000
    out = shm.projectors(d, torch.float64, workspace=ws)
    assert shm.projectors_check(ws) & 1
    # and a clean problem again reports nothing
    d.point_offsets[3] = int(prob.point_offsets[3])
    out = shm.projectors(d, torch.float64, workspace=ws)
    assert shm.projectors_check(ws) == 0
    del out


def test_host_side_validation():
    prob = small_problem(7)
    d = shm.DeviceProjectors(prob)
    ws = d.workspace(torch.float64)
    L = shm.lib()
    import ctypes
    bad = shm._binding._ProjProblem.from_buffer_copy(d.c)
    bad.radial_lstride = 1                      # smaller than 1 + max lmax
    out = torch.empty(d.n_values, dtype=torch.float64, device="cuda")
    assert L.shm_projectors(ctypes.byref(bad), 1, out.data_ptr(), ws.data_ptr(), ws.numel(), None) == 1
    bad = shm._binding._ProjProblem.from_buffer_copy(d.c)
    bad.box = 7.0                               # != ng * h
    assert L.shm_projectors(ctypes.byref(bad), 1, out.data_ptr(), ws.data_ptr(), ws.numel(), None) == 1
    assert L.shm_projectors(ctypes.byref(d.c), 1, out.data_ptr(), ws.data_ptr(), 16, None) == 1   # workspace


@pytest.mark.parametrize("dtype,tol", [(torch.float64, PROJ_TOL_F64), (torch.float32, PROJ_TOL_F32)])
def test_full_projector_workload(oracle_mod, dtype, tol, capsys):
    """512 atoms in a 40 bohr box, h = 0.2 bohr, spheres of 2-5 bohr, lmax in
    {2, 3, 4}: every value against the oracle, in bench.py's launch set-up."""
    prob = inputs.projector_problem()
    got = run(prob, dtype)
    ref = oracle_mod.projectors(prob)
    worst = check(prob, got, ref, tol, f"full workload {dtype}")
    with capsys.disabled():
        print(f"\nprojectors {dtype}: {prob.n_atoms} atoms, {prob.n_points} points, {prob.n_values} values, "
              f"max scaled error {worst:.2e}")


# ------------------------------------------------- prepare / run, variants, graphs

def _prob_all_lmax():
    return small_problem(12, n_atoms=10, n_species=10, lmax_choices=tuple(range(10)))


@pytest.mark.parametrize("dtype,tol", [(torch.float64, PROJ_TOL_F64), (torch.float32, PROJ_TOL_F32)])
def test_prepare_once_run_many(oracle_mod, dtype, tol):
    """One set-up launch, then several single-launch runs: each run gives the
    same bits (a run writes nothing in the workspace but the error word)."""
    prob = _prob_all_lmax()
    d = shm.DeviceProjectors(prob)
    ws = d.workspace(dtype)
    shm.projectors_prepare(d, dtype, ws)
    outs = []
    for _ in range(3):
        out = torch.full((d.n_values,), float("nan"), dtype=dtype, device="cuda")
        shm.projectors_run(d, dtype, out, ws)
        outs.append(out)
    torch.cuda.synchronize()
    assert shm.projectors_check(ws) == 0
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    check(prob, outs[0].cpu().numpy(), oracle_mod.projectors(prob), tol, f"prepared runs {dtype}")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_every_projector_variant_is_bitwise_the_same(dtype):
    """Tile size, points per thread, register cap and store path change the
    launch, not the arithmetic of a row."""
    prob = _prob_all_lmax()
    d = shm.DeviceProjectors(prob)
    names = set()
    ref = None
    try:
        for v in range(shm.projectors_variant_count()):
            shm.set_projectors_variant(dtype, v)
            names.add(shm.projectors_variant(dtype))
            ws = d.workspace(dtype)
            out = shm.projectors(d, dtype, workspace=ws)
            torch.cuda.synchronize()
            assert shm.projectors_check(ws) == 0
            if ref is None:
                ref = out
            assert torch.equal(out, ref), shm.projectors_variant(dtype)
    finally:
        shm.set_projectors_variant(dtype, -1)
    assert len(names) == shm.projectors_variant_count()


def _reshape(prob, species_lmax, atom_species, counts, radial=None):
    """The problem with its species, and each atom's sphere list cut to its
    first counts[a] points (every listed point stays inside its sphere), with
    the offsets rebuilt."""
    import dataclasses
    poff = np.asarray(prob.point_offsets)
    lists = [np.asarray(prob.point_index)[poff[a]:poff[a] + c] for a, c in enumerate(counts)]
    n = np.array([len(x) for x in lists], dtype=np.int64)
    lm = np.asarray(species_lmax)[np.asarray(atom_species)].astype(np.int64)
    return dataclasses.replace(
        prob, species_lmax=np.asarray(species_lmax, dtype=np.int32),
        atom_species=np.asarray(atom_species, dtype=np.int32),
        radial=prob.radial if radial is None else radial,
        point_offsets=np.concatenate([[0], np.cumsum(n)]).astype(np.int64),
        point_index=np.concatenate(lists).astype(np.int32),
        out_offsets=np.concatenate([[0], np.cumsum(n * (lm + 1) ** 2)]).astype(np.int64))


@pytest.mark.parametrize("dtype,tol", [(torch.float64, PROJ_TOL_F64), (torch.float32, PROJ_TOL_F32)])
def test_lmax3_rows_at_every_output_phase(oracle_mod, dtype, tol):
    """Rows of 16 values (lmax 3) go out by 16-byte staging and one bulk copy
    (FP32), the straddled 16-byte chunks completed from the lane before: atoms
    of lmax 0 (one value per point) in front of each lmax-3 atom shift its
    block to every 16-byte phase of the output, with ragged last tiles; the
    values match the oracle and, bit for bit, the copy-out variant."""
    base = small_problem(21, n_atoms=8, lmax_choices=(0, 3), n_species=2)
    n = np.diff(np.asarray(base.point_offsets))
    counts, total = [], 0
    for a in range(8):
        if a % 2 == 0:  # lmax 0, sized so that the next block starts at phase (a // 2) of 4 values
            c = int(n[a]) - ((total + int(n[a]) - a // 2) % 4)
            assert c > 0
        else:
            c = int(n[a]) - (int(n[a]) % 128 == 0)  # a ragged last tile
        counts.append(c)
        total += c * (1 if a % 2 == 0 else 16)
    prob = _reshape(base, [0, 3], [a % 2 for a in range(8)], counts)
    ooff = np.asarray(prob.out_offsets)
    assert sorted(int(ooff[a]) % 4 for a in (1, 3, 5, 7)) == [0, 1, 2, 3]
    d = shm.DeviceProjectors(prob)
    got = run(prob, dtype)
    check(prob, got, oracle_mod.projectors(prob), tol, f"lmax-3 phases {dtype}")
    try:
        shm.set_projectors_variant(dtype, 1)        # tile512-4rounds-copyout
        ws = d.workspace(dtype)
        ref = shm.projectors(d, dtype, workspace=ws)
        torch.cuda.synchronize()
        assert shm.projectors_check(ws) == 0
    finally:
        shm.set_projectors_variant(dtype, -1)
    assert np.array_equal(got, ref.cpu().numpy())


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_rows_up_to_lmax4_and_up_to_lmax9_agree(dtype):
    """A problem whose species all have lmax <= 4 runs the row code built up
    to lmax 4; the same atoms with one more (unused) species of lmax 9 run
    the code built up to lmax 9: the same bits."""
    prob = small_problem(4, n_atoms=8)
    S, Ls, nr = prob.radial.shape
    radial9 = np.zeros((S + 1, 10, nr))
    radial9[:S, :Ls] = prob.radial
    radial9[S] = prob.radial[0, 0]
    n = np.diff(np.asarray(prob.point_offsets))
    wide = _reshape(prob, list(prob.species_lmax) + [9], prob.atom_species, n, radial=radial9)
    assert int(np.max(prob.species_lmax)) <= 4
    a = run(prob, dtype)
    b = run(wide, dtype)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_run_captured_in_a_cuda_graph(dtype):
    """shm_projectors_run is one launch that allocates nothing: captured into
    a CUDA graph once and replayed, it gives the bits of a plain run."""
    prob = small_problem(13)
    d = shm.DeviceProjectors(prob)
    ws = d.workspace(dtype)
    plain = shm.projectors(d, dtype, workspace=ws)
    shm.projectors_prepare(d, dtype, ws)
    out = torch.zeros(d.n_values, dtype=dtype, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        shm.projectors_run(d, dtype, out, ws, stream=s)
    for _ in range(3):
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, plain)
    assert shm.projectors_check(ws) == 0


def test_projector_autotune():
    prob = small_problem(14)
    d = shm.DeviceProjectors(prob)
    for dtype in (torch.float64, torch.float32):
        ws = d.workspace(dtype)
        out = torch.empty(d.n_values, dtype=dtype, device="cuda")
        ref = shm.projectors(d, dtype, workspace=d.workspace(dtype)).clone()
        try:
            ms = shm.projectors_autotune(d, dtype, out, ws)
            assert ms > 0
            assert shm.projectors_variant(dtype)
            # the workspace is left prepared for the chosen variant
            out.zero_()
            shm.projectors_run(d, dtype, out, ws)
            torch.cuda.synchronize()
            assert torch.equal(out, ref)
        finally:
            shm.set_projectors_variant(dtype, -1)


def test_run_needs_a_prepared_workspace():
    prob = small_problem(15)
    d = shm.DeviceProjectors(prob)
    ws = d.workspace(torch.float64)
    out = torch.empty(d.n_values, dtype=torch.float64, device="cuda")
    with pytest.raises(shm.ShmError) as ei:
        shm.projectors_run(d, torch.float64, out, ws)
    assert ei.value.status == 1 and "prepare" in str(ei.value)
    shm.projectors_prepare(d, torch.float64, ws)
    with pytest.raises(shm.ShmError):          # prepared for FP64, run as FP32
        shm.projectors_run(d, torch.float32, out.view(torch.float32)[:d.n_values], ws)


def test_run_on_a_corrupted_workspace_stays_in_bounds():
    """Garbage in the tile table, the atom order and the tile descriptors of
    a prepared workspace, and a tile count above the problem's: the run
    checks every descriptor and index it follows against the problem, flags
    the tiles that do not fit it and writes only inside the output; a new
    prepare restores the correct values."""
    prob = small_problem(16)
    d = shm.DeviceProjectors(prob)
    ws = d.workspace(torch.float64)
    ref = shm.projectors(d, torch.float64, workspace=ws).clone()
    shm.projectors_prepare(d, torch.float64, ws)
    torch.cuda.synchronize()
    n_atoms = prob.n_atoms
    g = torch.Generator().manual_seed(5)
    tiles = ws[256:256 + 8 * (n_atoms + 1)].view(torch.int64)
    n_tiles = int(tiles[-1].item())
    assert n_tiles > 0
    tiles.copy_(torch.randint(-50, 400, (n_atoms + 1,), generator=g))
    tiles[-1] = n_tiles + 50
    order_off = 256 + ((8 * (n_atoms + 1) + 255) // 256) * 256
    order = ws[order_off:order_off + 4 * n_atoms].view(torch.int32)
    order.copy_(torch.randint(-3, n_atoms + 3, (n_atoms,), generator=g, dtype=torch.int32))
    desc_off = order_off + ((4 * n_atoms + 255) // 256) * 256
    desc = ws[desc_off:desc_off + 32 * n_tiles].view(torch.int32)
    desc.copy_(torch.randint(-(1 << 31), (1 << 31) - 1, (8 * n_tiles,), generator=g, dtype=torch.int32))
    guard = torch.full((d.n_values + 64,), -7.0, dtype=torch.float64, device="cuda")
    shm.projectors_run(d, torch.float64, guard[:d.n_values], ws)
    torch.cuda.synchronize()
    assert torch.all(guard[d.n_values:] == -7.0)
    assert shm.projectors_check(ws) & 8
    shm.projectors_prepare(d, torch.float64, ws)
    out = torch.empty(d.n_values, dtype=torch.float64, device="cuda")
    shm.projectors_run(d, torch.float64, out, ws)
    torch.cuda.synchronize()
    assert torch.equal(out, ref) and shm.projectors_check(ws) == 0


def test_overlapping_atom_ranges_stay_in_bounds():
    """Point offsets whose valid atoms overlap (each even atom claims every
    point; the odd atoms between them have reversed offsets and are
    rejected) claim more tiles than the workspace has descriptors for: the
    set-up writes none past them and flags the offsets, and the run writes
    only inside the output."""
    import dataclasses
    base = small_problem(7)
    n, A = base.n_points, base.n_atoms
    assert A == 6
    poff = np.array([0, n, 0, n, 0, n, 0], dtype=np.int64)
    lm = np.asarray(base.species_lmax)[np.asarray(base.atom_species)].astype(np.int64)
    ooff = [0]
    for a in range(A):
        ooff.append(ooff[-1] + (n * (lm[a] + 1) ** 2 if a % 2 == 0 else 0))
    prob = dataclasses.replace(base, point_offsets=poff, out_offsets=np.array(ooff, dtype=np.int64))
    d = shm.DeviceProjectors(prob)
    assert d.n_values == ooff[-1]
    assert 3 * -(-n // 128) > n // 128 + A + 1     # 128-point tiles: more than the descriptors
    for dtype in (torch.float64, torch.float32):
        try:
            shm.set_projectors_variant(dtype, 5)    # tile128
            ws = d.workspace(dtype)
            guard = torch.full((d.n_values + 64,), -7.0, dtype=dtype, device="cuda")
            shm.projectors(d, dtype, out=guard[:d.n_values], workspace=ws)
            torch.cuda.synchronize()
        finally:
            shm.set_projectors_variant(dtype, -1)
        assert torch.all(guard[d.n_values:] == -7.0)
        assert shm.projectors_check(ws) & 1


# ------------------------------------------------- all-binary64 projectors (SHM_STRICT_FP64)

def run_strict(prob):
    d = shm.DeviceProjectors(prob)
    ws = d.workspace(torch.float64)
    out = shm.projectors(d, torch.float64, workspace=ws, strict=True)
    torch.cuda.synchronize()
    assert shm.projectors_check(ws) == 0
    return out.cpu().numpy()


@pytest.mark.parametrize("prob_kw", [dict(extra=20), dict(extra=21, n_atoms=10, n_species=10,
                                                          lmax_choices=tuple(range(10))),
                                     dict(extra=22, n_rad=5, r_min=0.05, r_max=2.5)])
def test_strict_fp64_projectors(oracle_mod, prob_kw):
    """Binary64 tables, log-grid index and rows: within the FP64 tolerance of
    the oracle, tighter than the default FP64 form."""
    prob = small_problem(**prob_kw)
    got = run_strict(prob)
    worst = check(prob, got, oracle_mod.projectors(prob), PROJ_TOL_F64, "strict FP64 projectors")
    assert worst <= 2e-14


def test_strict_fp64_projectors_full_workload(oracle_mod, capsys):
    prob = inputs.projector_problem()
    got = run_strict(prob)
    worst = check(prob, got, oracle_mod.projectors(prob), PROJ_TOL_F64, "strict full workload")
    with capsys.disabled():
        print(f"\nstrict FP64 projectors, 512 atoms: max scaled error {worst:.2e}")


def test_strict_prepared_runs_and_graph():
    prob = small_problem(23)
    d = shm.DeviceProjectors(prob)
    ws = d.workspace(torch.float64)
    ref = shm.projectors(d, torch.float64, workspace=ws, strict=True).clone()
    shm.projectors_prepare(d, torch.float64, ws, strict=True)
    out = torch.zeros(d.n_values, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        shm.projectors_run(d, torch.float64, out, ws, stream=s)
    for _ in range(2):
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    # the default form differs (float-float), within tolerance
    dflt = shm.projectors(d, torch.float64, workspace=d.workspace(torch.float64))
    torch.cuda.synchronize()
    assert not torch.equal(dflt, ref)


def _strict_run_form(prob, form):
    d = shm.DeviceProjectors(prob)
    ws = d.workspace(torch.float64)
    try:
        shm.set_projectors_strict_form(form)
        out = shm.projectors(d, torch.float64, workspace=ws, strict=True)
        torch.cuda.synchronize()
    finally:
        shm.set_projectors_strict_form(3)
    assert shm.projectors_check(ws) == 0
    return out


def _strict_form_problems():
    on_grid = small_problem(24)
    on_grid.atom_pos[0] = np.array([8, 9, 10], dtype=np.float64) * on_grid.h  # origin and axis points
    zero_f = small_problem(25)
    zero_f.radial[1, 2] = 0.0                                                  # f_l = 0 for one (species, l)
    return {"on_grid": on_grid, "zero_f": zero_f,
            "all_lmax": small_problem(26, n_atoms=10, n_species=10, lmax_choices=tuple(range(10))),
            "full": inputs.projector_problem()}


@pytest.mark.parametrize("which", ["on_grid", "zero_f", "all_lmax", "full"])
def test_strict_forms_are_bitwise_the_same(oracle_mod, which):
    """SHM_STRICT_FP64 rows with every product on the FP64 pipe (form 1),
    with the output products (form 2) or every product of the row (form 3,
    the default) on the integer pipes by dmul_int: the same bits, including
    rows that dmul_int declines (a zero f_l, points on the atom's axes, the
    atom's own grid point) and fall back to the FP64 instructions."""
    assert shm.projectors_strict_form() == 3
    prob = _strict_form_problems()[which]
    f1 = _strict_run_form(prob, 1)
    for form in (2, 3):
        f = _strict_run_form(prob, form)
        assert torch.equal(f1, f), f"form {form}"
        if which != "full":
            check(prob, f.cpu().numpy(), oracle_mod.projectors(prob), PROJ_TOL_F64, f"strict form {form} {which}")
    with pytest.raises(shm.ShmError):
        shm.set_projectors_strict_form(4)
