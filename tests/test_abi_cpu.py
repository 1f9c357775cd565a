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
