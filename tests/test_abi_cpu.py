"""libshm loads without a GPU, exports every entry point include/shm.h
declares, and rejects bad arguments on the host (no compute calls here)."""
import ctypes
import os
import re

import pytest

import paper_2510_05282_b300 as shm
from paper_2510_05282_b300 import _binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = set()
    inc = os.path.join(ROOT, "include")
    for name in os.listdir(inc):
        if not name.endswith(".h"):
            continue
        text = open(os.path.join(inc, name)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(shm_\w+)\s*\(", text, flags=re.M):
            syms.add(m.group(1))
    return syms


@pytest.fixture(scope="module")
def L():
    from paper_2510_05282_b300 import build
    build.build()
    return shm.lib()


def test_exports_every_declared_symbol(L):
    syms = declared_symbols()
    assert {"shm_eval", "shm_eval_ex", "shm_last_error"} <= syms
    for s in sorted(syms):
        assert hasattr(L, s), f"libshm does not export {s}"


def test_num_harmonics_and_status_strings(L):
    assert [L.shm_num_harmonics(l) for l in range(17)] == [(l + 1) ** 2 for l in range(17)]
    assert L.shm_num_harmonics(17) == 0 and L.shm_num_harmonics(-1) == 0
    assert [L.shm_num_spinors(l) for l in range(10)] == [2 * (l + 1) ** 2 for l in range(10)]
    assert L.shm_num_spinors(10) == -1 and L.shm_num_spinors(-1) == -1
    assert L.shm_status_string(0) == b"SHM_OK"
    assert L.shm_status_string(5) == b"SHM_ETIMEOUT"


@pytest.mark.parametrize("args,msg", [
    ((1, 10, 17, 1, 1, None), "lmax"),
    ((1, 10, -1, 1, 1, None), "lmax"),
    ((1, 10, 3, 7, 1, None), "dtype"),
    ((1, -5, 3, 1, 1, None), "n must"),
    ((None, 10, 3, 1, 1, None), "non-null"),
    ((8, 10, 3, 1, 12, None), "aligned"),
])
def test_argument_errors_are_synchronous(L, args, msg):
    st = L.shm_eval(*args)
    assert st == 1
    assert msg in L.shm_last_error().decode()


def test_n_zero_is_a_no_op(L):
    assert L.shm_eval(None, 0, 9, 1, None, None) == 0


def test_unknown_flags_rejected(L):
    assert L.shm_eval_ex(8, 1, 3, 1, 0x10, 64, None) == 1
    assert "flag" in L.shm_last_error().decode()


def test_host_entry_validation(L):
    assert L.shm_eval_host(None, 5, 3, 1, None, None, 0, None) == 1
    assert L.shm_eval_host_workspace_size(9, 1, 0) == 0
    ws = L.shm_eval_host_workspace_size(9, 1, 1000)
    assert ws >= 2 * 1000 * 8 * 103


def test_binding_errors_carry_text(L):
    with pytest.raises(shm.ShmError) as ei:
        shm.check(L.shm_eval(None, 3, 17, 1, None, None))
    assert ei.value.status == 1 and "lmax" in str(ei.value)


def test_projector_sizes_rejected_on_the_host(L):
    """Atom counts the projector tables cannot index (the tile order holds
    atoms as int32) and negative sizes fail before any device call."""
    p = _binding._ProjProblem()
    p.n_species = 1
    for n_atoms, msg in ((1 << 31, "2^31"), (-1, "negative")):
        p.n_atoms = n_atoms
        assert L.shm_projectors(ctypes.byref(p), 1, None, None, 0, None) == 1
        assert msg in L.shm_last_error().decode()


def _proj_problem_scalars(**kw):
    """A projector problem struct with valid host scalars and null device
    pointers: every check below fails on the host before any CUDA call."""
    import numpy as np
    p = _binding._ProjProblem()
    p.n_atoms, p.n_species, p.radial_lstride, p.n_rad = 1, 1, 5, 2000
    p.r_min, p.dlog, p.ng, p.h = 1e-4, 0.005, 10, 0.2
    p.box = p.ng * p.h
    lm = np.array([4] * 64, dtype=np.int32)
    p.species_lmax = lm.ctypes.data
    for k, v in kw.items():
        setattr(p, k, v)
    return p, lm


@pytest.mark.parametrize("field,value,msg", [
    ("radial_lstride", 1 << 30, "radial_lstride"),   # n_species x lstride x n_rad x 32 bytes would wrap
    ("n_rad", (1 << 26) + 1, "n_rad"),
    ("n_rad", 3, "n_rad"),
    ("n_points", (1 << 40) + 1, "n_points"),
    ("n_values", (1 << 44) + 1, "n_values"),
    ("radial_lstride", 4, "radial_lstride"),          # below 1 + lmax
])
def test_projector_size_products_cannot_overflow(L, field, value, msg):
    """Sizes whose byte products would wrap round 2^64 (the example of a
    64-species problem with lstride 2^30 and n_rad 2^25) are rejected on the
    host, by shm_projectors, shm_projectors_noalloc and the workspace-size
    query alike, before anything touches the device."""
    kw = {field: value}
    if field == "radial_lstride" and value == 1 << 30:
        kw.update(n_species=64, n_rad=1 << 25)
    p, keep = _proj_problem_scalars(**kw)
    assert L.shm_projectors(ctypes.byref(p), 1, None, None, 0, None) == 1
    assert msg in L.shm_last_error().decode()
    assert L.shm_projectors_noalloc(ctypes.byref(p), 0, None, None) == 1
    assert msg in L.shm_last_error().decode()
    assert L.shm_projectors_workspace_size(ctypes.byref(p), 1) == 0


def test_projector_noalloc_reports_the_bad_field_first(L):
    """A bad field is named as such, not as a scratch shortfall."""
    p, keep = _proj_problem_scalars(ng=-5)
    assert L.shm_projectors_noalloc(ctypes.byref(p), 1, None, None) == 1
    err = L.shm_last_error().decode()
    assert "ng must" in err and "scratch" not in err


def test_strict_flag_host_side(L):
    """SHM_STRICT_FP64 selects a separate choice of launch variant: only the
    all-binary64 ones may be pinned for it; unknown flag bits are refused."""
    assert L.shm_eval_variant_ex(9, 1, 2).decode() == "rows-tma-emu-o-32"
    assert L.shm_eval_variant_ex(8, 1, 2).decode() == "staged-64"       # even lmax: no TMA row pitch
    assert "hybrid" in L.shm_eval_variant_ex(9, 1, 0).decode()
    assert L.shm_eval_variant_ex(9, 0, 2).decode() == "staged-64"       # FP32 ignores the flag
    for v in range(L.shm_eval_variant_count()):
        st = L.shm_eval_set_variant_ex(9, 1, 2, v)
        assert st in (0, 1)
        if st == 1:
            assert "float-float" in L.shm_last_error().decode()
    assert L.shm_eval_set_variant_ex(9, 1, 2, 12) == 1                  # phased-hybrid-tma-128
    assert L.shm_eval_set_variant_ex(9, 1, 2, 14) == 0
    assert L.shm_eval_variant_ex(9, 1, 2).decode() == "rows-tma-64"
    assert L.shm_eval_set_variant_ex(9, 1, 2, -1) == 0
    assert L.shm_eval_set_variant_ex(9, 1, 4, 0) == 1                   # unknown bit
    assert L.shm_eval_ex(8, 1, 3, 1, 0x4, 64, None) == 1
    assert L.shm_eval_angles_ex(8, 1, 3, 1, 0x1, 64, None) == 1         # angles take no normalised flag


def test_strict_projector_form_is_validated_on_the_host(L):
    assert L.shm_projectors_strict_form() == 3
    for bad in (0, 4, -1):
        assert L.shm_projectors_set_strict_form(bad) == 1
        assert b"form" in L.shm_last_error()
    for form in (1, 2, 3):
        assert L.shm_projectors_set_strict_form(form) == 0 and L.shm_projectors_strict_form() == form
