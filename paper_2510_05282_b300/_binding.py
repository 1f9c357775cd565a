"""Thin ctypes binding over libshm.so (argument marshalling only).

Every step of the computation runs in the library's CUDA kernels; PyTorch is
used here only to hold device memory and to name the current CUDA stream.
The library is loaded on first use; if it is missing or fails to load, the
call raises -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libshm.so")

SHM_F32, SHM_F64 = 0, 1
SHM_NORMALIZED_INPUT = 0x1
SHM_STRICT_FP64 = 0x2
LMAX_CAP = 9

STATUS = {0: "SHM_OK", 1: "SHM_EINVAL", 2: "SHM_ENOMEM", 3: "SHM_ECUDA", 4: "SHM_EBUSY",
          5: "SHM_ETIMEOUT", 6: "SHM_EUNSUPPORTED", 7: "SHM_ENOTFOUND"}


class ShmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    """The loaded libshm (raises if it has not been built)."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise RuntimeError(f"libshm.so is not built ({LIB_PATH}); run "
                                       "`python -m paper_2510_05282_b300.build`")
                L = ctypes.CDLL(LIB_PATH)
                _declare(L)
                _lib = L
    return _lib


def _declare(L):
    vp, i64, i32, u32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint, ctypes.c_size_t
    L.shm_eval.argtypes = [vp, i64, i32, i32, vp, vp]
    L.shm_eval.restype = i32
    L.shm_eval_ex.argtypes = [vp, i64, i32, i32, u32, vp, vp]
    L.shm_eval_ex.restype = i32
    L.shm_eval_host.argtypes = [vp, i64, i32, i32, vp, vp, sz, vp]
    L.shm_eval_host.restype = i32
    L.shm_eval_host_workspace_size.argtypes = [i32, i32, i64]
    L.shm_eval_host_workspace_size.restype = sz
    L.shm_autotune.argtypes = [i32, i32, i64, ctypes.POINTER(ctypes.c_double)]
    L.shm_autotune.restype = i32
    L.shm_eval_variant.argtypes = [i32, i32]
    L.shm_eval_variant.restype = ctypes.c_char_p
    L.shm_eval_variant_count.argtypes = []
    L.shm_eval_variant_count.restype = i32
    L.shm_eval_set_variant.argtypes = [i32, i32, i32]
    L.shm_eval_set_variant.restype = i32
    L.shm_eval_complex.argtypes = [vp, i64, i32, i32, u32, vp, vp]
    L.shm_eval_complex.restype = i32
    L.shm_eval_angles.argtypes = [vp, i64, i32, i32, vp, vp]
    L.shm_eval_angles.restype = i32
    L.shm_eval_angles_ex.argtypes = [vp, i64, i32, i32, u32, vp, vp]
    L.shm_eval_angles_ex.restype = i32
    L.shm_eval_host_ex.argtypes = [vp, i64, i32, i32, u32, vp, vp, sz, vp]
    L.shm_eval_host_ex.restype = i32
    L.shm_autotune_ex.argtypes = [i32, i32, u32, i64, ctypes.POINTER(ctypes.c_double)]
    L.shm_autotune_ex.restype = i32
    L.shm_eval_variant_ex.argtypes = [i32, i32, u32]
    L.shm_eval_variant_ex.restype = ctypes.c_char_p
    L.shm_eval_set_variant_ex.argtypes = [i32, i32, u32, i32]
    L.shm_eval_set_variant_ex.restype = i32
    L.shm_probe_fp64_rate.argtypes = [i64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.shm_probe_fp64_rate.restype = i32
    L.shm_probe_dmul.argtypes = [i64, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    L.shm_probe_dmul.restype = i32
    L.shm_eval_spinor.argtypes = [vp, i64, i32, i32, u32, vp, vp]
    L.shm_eval_spinor.restype = i32
    L.shm_num_spinors.argtypes = [i32]
    L.shm_num_spinors.restype = i32
    L.shm_num_harmonics.argtypes = [i32]
    L.shm_num_harmonics.restype = i32
    L.shm_last_error.argtypes = []
    L.shm_last_error.restype = ctypes.c_char_p
    L.shm_status_string.argtypes = [i32]
    L.shm_status_string.restype = ctypes.c_char_p
    for name, decl in _EXTRA_DECLS:
        fn = getattr(L, name, None)
        if fn is not None:
            fn.argtypes, fn.restype = decl


# further entry points register (name, (argtypes, restype)) here
_EXTRA_DECLS: list = []


def check(status: int) -> None:
    if status != 0:
        raise ShmError(status, lib().shm_last_error().decode(errors="replace"))


def num_harmonics(lmax: int) -> int:
    return (lmax + 1) * (lmax + 1)


def _dtype_code(dtype) -> int:
    import torch
    if dtype in (torch.float64, "f64", np.float64):
        return SHM_F64
    if dtype in (torch.float32, "f32", np.float32):
        return SHM_F32
    raise ValueError(f"unsupported dtype {dtype}")


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _flags(normalized: bool = False, strict: bool = False) -> int:
    return (SHM_NORMALIZED_INPUT if normalized else 0) | (SHM_STRICT_FP64 if strict else 0)


def eval_sh(points, lmax: int, out=None, normalized: bool = False, stream=None, strict: bool = False):
    """All R_l^m, l <= lmax, at device points [n, 3] (float32 or float64 CUDA
    tensor) -> [n, (lmax+1)^2] of the same dtype, column k = l*l + l + m.
    strict: all-binary64 rows for float64 (SHM_STRICT_FP64)."""
    import torch
    if not (isinstance(points, torch.Tensor) and points.is_cuda):
        raise TypeError("points must be a CUDA tensor")
    if points.dim() != 2 or points.shape[1] != 3 or not points.is_contiguous():
        raise ValueError("points must be a contiguous [n, 3] tensor")
    code = _dtype_code(points.dtype)
    n = points.shape[0]
    if out is None:
        out = torch.empty((n, num_harmonics(lmax)), dtype=points.dtype, device=points.device)
    elif out.dtype != points.dtype or not out.is_contiguous() or out.numel() != n * num_harmonics(lmax):
        raise ValueError("out must be contiguous, of the points dtype and [n, (lmax+1)^2]")
    check(lib().shm_eval_ex(points.data_ptr(), n, int(lmax), code, _flags(normalized, strict), out.data_ptr(),
                            _stream_ptr(stream)))
    return out


def eval_complex(points, lmax: int, out=None, normalized: bool = False, stream=None, strict: bool = False):
    """Complex Y_l^m, l <= lmax, at device points [n, 3] -> complex CUDA tensor
    [n, (lmax+1)^2] (complex128 for float64 points, complex64 for float32)."""
    import torch
    if not (isinstance(points, torch.Tensor) and points.is_cuda):
        raise TypeError("points must be a CUDA tensor")
    if points.dim() != 2 or points.shape[1] != 3 or not points.is_contiguous():
        raise ValueError("points must be a contiguous [n, 3] tensor")
    code = _dtype_code(points.dtype)
    n = points.shape[0]
    if out is None:
        out = torch.empty((n, num_harmonics(lmax), 2), dtype=points.dtype, device=points.device)
    elif out.dtype != points.dtype or not out.is_contiguous() or out.numel() != 2 * n * num_harmonics(lmax):
        raise ValueError("out must be a contiguous [n, (lmax+1)^2, 2] tensor of the points dtype")
    check(lib().shm_eval_complex(points.data_ptr(), n, int(lmax), code, _flags(normalized, strict), out.data_ptr(),
                                 _stream_ptr(stream)))
    return torch.view_as_complex(out.view(n, num_harmonics(lmax), 2))


def num_spinors(lmax: int) -> int:
    """Spinor harmonics per point: 2 (lmax+1)^2."""
    n = lib().shm_num_spinors(int(lmax))
    if n < 0:
        raise ShmError(1, "lmax must be in 0..9")
    return n


def eval_spinor(points, lmax: int, out=None, normalized: bool = False, stream=None, strict: bool = False):
    """Spin-1/2 spinor harmonics (Eq. 7) for l <= lmax at device points [n, 3]
    -> complex CUDA tensor [n, 2 (lmax+1)^2, 2]: spinor q (l ascending, j = l - 1/2
    before j = l + 1/2, m_j ascending), component (upper, lower)."""
    import torch
    if not (isinstance(points, torch.Tensor) and points.is_cuda):
        raise TypeError("points must be a CUDA tensor")
    if points.dim() != 2 or points.shape[1] != 3 or not points.is_contiguous():
        raise ValueError("points must be a contiguous [n, 3] tensor")
    code = _dtype_code(points.dtype)
    n = points.shape[0]
    ns = num_spinors(lmax)
    if out is None:
        out = torch.empty((n, ns, 2, 2), dtype=points.dtype, device=points.device)
    elif out.dtype != points.dtype or not out.is_contiguous() or out.numel() != 4 * n * ns:
        raise ValueError("out must be a contiguous [n, 2 (lmax+1)^2, 2, 2] tensor of the points dtype")
    check(lib().shm_eval_spinor(points.data_ptr(), n, int(lmax), code, _flags(normalized, strict), out.data_ptr(),
                                _stream_ptr(stream)))
    return torch.view_as_complex(out.view(n, ns, 2, 2))


def eval_angles(angles, lmax: int, out=None, stream=None, strict: bool = False):
    """All R_l^m, l <= lmax, at directions given as a device tensor [n, 2] of
    (theta, phi) -> [n, (lmax+1)^2] of the same dtype."""
    import torch
    if not (isinstance(angles, torch.Tensor) and angles.is_cuda):
        raise TypeError("angles must be a CUDA tensor")
    if angles.dim() != 2 or angles.shape[1] != 2 or not angles.is_contiguous():
        raise ValueError("angles must be a contiguous [n, 2] tensor")
    n = angles.shape[0]
    if out is None:
        out = torch.empty((n, num_harmonics(lmax)), dtype=angles.dtype, device=angles.device)
    check(lib().shm_eval_angles_ex(angles.data_ptr(), n, int(lmax), _dtype_code(angles.dtype),
                                   _flags(False, strict), out.data_ptr(), _stream_ptr(stream)))
    return out


def autotune(lmax: int, dtype, n_probe: int = 1 << 20, strict: bool = False) -> float:
    """Time every launch variant for (lmax, dtype) (the all-binary64 ones only
    with strict); keep the fastest. Returns its ms."""
    best = ctypes.c_double(0.0)
    check(lib().shm_autotune_ex(int(lmax), _dtype_code(dtype), _flags(False, strict), int(n_probe),
                                ctypes.byref(best)))
    return best.value


def eval_variant(lmax: int, dtype, strict: bool = False) -> str:
    return lib().shm_eval_variant_ex(int(lmax), _dtype_code(dtype), _flags(False, strict)).decode()


def set_eval_variant(lmax: int, dtype, variant: int, strict: bool = False) -> None:
    check(lib().shm_eval_set_variant_ex(int(lmax), _dtype_code(dtype), _flags(False, strict), int(variant)))


def probe_dmul(n: int, seed: int = 1):
    """(mismatches, declined) of the integer-pipe binary64 multiply against
    the DMUL instruction on n generated operand pairs."""
    mm, dec = ctypes.c_int64(-1), ctypes.c_int64(-1)
    check(lib().shm_probe_dmul(int(n), int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(mm), ctypes.byref(dec)))
    return mm.value, dec.value


def probe_fp64_rate(iters: int = 1 << 14):
    """Measured FP64 pipe rate of the current device: (DFMA instructions per
    second, ms of the timed launch)."""
    rate, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    check(lib().shm_probe_fp64_rate(int(iters), ctypes.byref(rate), ctypes.byref(ms)))
    return rate.value, ms.value


def eval_variant_count() -> int:
    return int(lib().shm_eval_variant_count())


def eval_host_workspace_size(lmax: int, dtype, chunk_points: int) -> int:
    return int(lib().shm_eval_host_workspace_size(int(lmax), _dtype_code(dtype), int(chunk_points)))


def eval_host(points_host, lmax: int, out_host, workspace, stream=None, strict: bool = False) -> None:
    """shm_eval_host: host (ideally pinned) points -> host rows, through a device
    workspace.  Enqueued on `stream`; synchronise it before reading out_host.
    points_host / out_host are CPU torch tensors or numpy arrays."""
    import torch

    def ptr(a):
        return a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data

    dt = points_host.dtype
    code = _dtype_code(dt)
    n = points_host.shape[0]
    check(lib().shm_eval_host_ex(ptr(points_host), n, int(lmax), code, _flags(False, strict), ptr(out_host),
                                 workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                 _stream_ptr(stream)))


# --------------------------------------------------------------------------- projectors

class _ProjProblem(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int64), ("atom_pos", ctypes.c_void_p), ("atom_species", ctypes.c_void_p),
                ("n_species", ctypes.c_int32), ("species_lmax", ctypes.c_void_p), ("radial", ctypes.c_void_p),
                ("radial_lstride", ctypes.c_int32), ("n_rad", ctypes.c_int32), ("r_min", ctypes.c_double),
                ("dlog", ctypes.c_double), ("box", ctypes.c_double), ("ng", ctypes.c_int32), ("h", ctypes.c_double),
                ("point_offsets", ctypes.c_void_p), ("point_index", ctypes.c_void_p),
                ("out_offsets", ctypes.c_void_p), ("n_points", ctypes.c_int64), ("n_values", ctypes.c_int64)]


_EXTRA_DECLS.extend([
    ("shm_projectors_workspace_size", ([ctypes.POINTER(_ProjProblem), ctypes.c_int], ctypes.c_size_t)),
    ("shm_projectors", ([ctypes.POINTER(_ProjProblem), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                         ctypes.c_size_t, ctypes.c_void_p], ctypes.c_int)),
    ("shm_projectors_check", ([ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int)),
    ("shm_projectors_noalloc", ([ctypes.POINTER(_ProjProblem), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p],
                                ctypes.c_int)),
    ("shm_projectors_prepare", ([ctypes.POINTER(_ProjProblem), ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                 ctypes.c_void_p], ctypes.c_int)),
    ("shm_projectors_prepare_ex", ([ctypes.POINTER(_ProjProblem), ctypes.c_int, ctypes.c_uint, ctypes.c_void_p,
                                    ctypes.c_size_t, ctypes.c_void_p], ctypes.c_int)),
    ("shm_projectors_ex", ([ctypes.POINTER(_ProjProblem), ctypes.c_int, ctypes.c_uint, ctypes.c_void_p,
                            ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p], ctypes.c_int)),
    ("shm_projectors_run", ([ctypes.POINTER(_ProjProblem), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_size_t, ctypes.c_void_p], ctypes.c_int)),
    ("shm_projectors_autotune", ([ctypes.POINTER(_ProjProblem), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)], ctypes.c_int)),
    ("shm_projectors_variant_count", ([], ctypes.c_int)),
    ("shm_projectors_variant", ([ctypes.c_int], ctypes.c_char_p)),
    ("shm_projectors_set_variant", ([ctypes.c_int, ctypes.c_int], ctypes.c_int)),
    ("shm_projectors_set_strict_form", ([ctypes.c_int], ctypes.c_int)),
    ("shm_projectors_strict_form", ([], ctypes.c_int)),
])

PROJ_NOALLOC_SCRATCH_BYTES = 1 << 25


class DeviceProjectors:
    """A projector problem uploaded to the GPU (device tensors kept alive here),
    with the C struct the library reads.  `prob` is an
    ``inputs.ProjectorProblem``-like object with numpy fields."""

    def __init__(self, prob, device="cuda"):
        import torch
        t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(device)  # noqa: E731
        self.atom_pos = t(prob.atom_pos, np.float64)
        self.atom_species = t(prob.atom_species, np.int32)
        self.radial = t(prob.radial, np.float64)
        self.point_offsets = t(prob.point_offsets, np.int64)
        self.point_index = t(prob.point_index, np.int32)
        self.out_offsets = t(prob.out_offsets, np.int64)
        self.species_lmax = np.ascontiguousarray(prob.species_lmax, dtype=np.int32)   # host
        self.n_values = int(prob.out_offsets[-1])
        self.n_points = int(prob.point_offsets[-1])
        self.c = _ProjProblem(
            n_atoms=int(prob.atom_pos.shape[0]), atom_pos=self.atom_pos.data_ptr(),
            atom_species=self.atom_species.data_ptr(), n_species=int(self.species_lmax.shape[0]),
            species_lmax=self.species_lmax.ctypes.data, radial=self.radial.data_ptr(),
            radial_lstride=int(prob.radial.shape[1]), n_rad=int(prob.radial.shape[2]),
            r_min=float(prob.r_min), dlog=float(prob.dlog), box=float(prob.box), ng=int(prob.ng), h=float(prob.h),
            point_offsets=self.point_offsets.data_ptr(), point_index=self.point_index.data_ptr(),
            out_offsets=self.out_offsets.data_ptr(), n_points=self.n_points, n_values=self.n_values)

    def workspace_size(self, dtype) -> int:
        return int(lib().shm_projectors_workspace_size(ctypes.byref(self.c), _dtype_code(dtype)))

    def workspace(self, dtype):
        import torch
        return torch.empty(max(self.workspace_size(dtype), 256), dtype=torch.uint8, device=self.atom_pos.device)


def projectors(dprob: DeviceProjectors, dtype, out=None, workspace=None, stream=None, strict: bool = False):
    """Fused projector values (flat CSR, [n_values]) of a DeviceProjectors problem
    (strict: all-binary64 for float64)."""
    import torch
    tdt = torch.float64 if _dtype_code(dtype) == SHM_F64 else torch.float32
    if out is None:
        out = torch.empty(dprob.n_values, dtype=tdt, device=dprob.atom_pos.device)
    if workspace is None:
        workspace = dprob.workspace(dtype)
    check(lib().shm_projectors_ex(ctypes.byref(dprob.c), _dtype_code(dtype), _flags(False, strict), out.data_ptr(),
                                  workspace.data_ptr(), workspace.numel(), _stream_ptr(stream)))
    return out


def projectors_prepare(dprob: DeviceProjectors, dtype, workspace, stream=None, strict: bool = False) -> None:
    """shm_projectors_prepare_ex: the per-problem set-up launch into `workspace`."""
    check(lib().shm_projectors_prepare_ex(ctypes.byref(dprob.c), _dtype_code(dtype), _flags(False, strict),
                                          workspace.data_ptr(), workspace.numel(), _stream_ptr(stream)))


def projectors_run(dprob: DeviceProjectors, dtype, out, workspace, stream=None):
    """shm_projectors_run: one persistent launch on a prepared workspace."""
    check(lib().shm_projectors_run(ctypes.byref(dprob.c), _dtype_code(dtype), out.data_ptr(), workspace.data_ptr(),
                                   workspace.numel(), _stream_ptr(stream)))
    return out


def projectors_autotune(dprob: DeviceProjectors, dtype, out, workspace) -> float:
    """Time every projector launch variant on this problem; keep the fastest
    (the workspace is left prepared for it).  Returns its ms per run."""
    best = ctypes.c_double(0.0)
    check(lib().shm_projectors_autotune(ctypes.byref(dprob.c), _dtype_code(dtype), out.data_ptr(),
                                        workspace.data_ptr(), workspace.numel(), ctypes.byref(best)))
    return best.value


def projectors_variant(dtype) -> str:
    return lib().shm_projectors_variant(_dtype_code(dtype)).decode()


def projectors_variant_count() -> int:
    return int(lib().shm_projectors_variant_count())


def set_projectors_variant(dtype, variant: int) -> None:
    check(lib().shm_projectors_set_variant(_dtype_code(dtype), int(variant)))


def set_projectors_strict_form(form: int) -> None:
    """Row form of later SHM_STRICT_FP64 projector prepares: 1 every product
    on the FP64 pipe, 2 the output products, 3 (default) every product of the
    row on the integer pipes (the same bits)."""
    check(lib().shm_projectors_set_strict_form(int(form)))


def projectors_strict_form() -> int:
    return int(lib().shm_projectors_strict_form())


def projectors_check(workspace, stream=None) -> int:
    bits = ctypes.c_uint32(0)
    check(lib().shm_projectors_check(workspace.data_ptr(), _stream_ptr(stream), ctypes.byref(bits)))
    return int(bits.value)


def projectors_noalloc(dprob: DeviceProjectors, dtype, out, stream=None):
    """shm_projectors_noalloc: the projector values into the caller's `out`
    ([n_values] CUDA tensor of dtype) with no device allocation by the library
    (its scratch is a static device array of PROJ_NOALLOC_SCRATCH_BYTES)."""
    check(lib().shm_projectors_noalloc(ctypes.byref(dprob.c), _dtype_code(dtype), out.data_ptr(),
                                       _stream_ptr(stream)))
    return out


# --------------------------------------------------------------------------- serving

SHM_REQ_DISCARD = 0x1
SHM_REQ_STRICT_FP64 = 0x2


class ServeConfig(ctypes.Structure):
    _fields_ = [("pool_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int32), ("queue_capacity", ctypes.c_int32),
                ("batch_points", ctypes.c_int64), ("chunk_points", ctypes.c_int64),
                ("inflight_batches", ctypes.c_int32), ("device", ctypes.c_int32)]


class _Request(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("n", ctypes.c_int64), ("lmax", ctypes.c_int32),
                ("dtype", ctypes.c_int), ("seed", ctypes.c_uint64), ("flags", ctypes.c_uint32)]


class ServeResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("out", ctypes.c_void_p), ("n", ctypes.c_int64), ("lmax", ctypes.c_int32),
                ("dtype", ctypes.c_int), ("t_submit_ms", ctypes.c_double), ("t_admit_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("rejected", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("batches", ctypes.c_uint64), ("queued_now", ctypes.c_uint64),
                ("active_now", ctypes.c_uint64), ("harmonics_done", ctypes.c_double), ("busy_ms", ctypes.c_double),
                ("lat_p50_ms", ctypes.c_double), ("lat_p99_ms", ctypes.c_double), ("lat_max_ms", ctypes.c_double),
                ("pool_bytes", ctypes.c_size_t), ("pool_in_use", ctypes.c_size_t), ("pool_peak", ctypes.c_size_t),
                ("collected", ctypes.c_uint64), ("client_lat_p50_ms", ctypes.c_double),
                ("client_lat_p99_ms", ctypes.c_double), ("client_lat_max_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp = ctypes.c_void_p
_EXTRA_DECLS.extend([
    ("shm_serve_create", ([ctypes.POINTER(ServeConfig), ctypes.POINTER(_vp)], ctypes.c_int)),
    ("shm_serve_submit", ([_vp, ctypes.POINTER(_Request), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int)),
    ("shm_serve_wait", ([_vp, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ServeResult)], ctypes.c_int)),
    ("shm_serve_wait_any", ([_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ServeResult)],
                            ctypes.c_int)),
    ("shm_serve_release", ([_vp, ctypes.c_uint64], ctypes.c_int)),
    ("shm_serve_stats_get", ([_vp, ctypes.POINTER(ServeStats)], ctypes.c_int)),
    ("shm_serve_stats_reset", ([_vp], ctypes.c_int)),
    ("shm_serve_destroy", ([_vp], ctypes.c_int)),
    ("shm_serve_generated_point", ([ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)], None)),
])


def serve_generated_point(seed: int, i: int):
    xyz = (ctypes.c_double * 3)()
    lib().shm_serve_generated_point(int(seed), int(i), xyz)
    return [xyz[0], xyz[1], xyz[2]]


class Server:
    """Continuous-batching evaluation server (shm_serve_*)."""

    def __init__(self, pool_bytes=8 << 30, max_slots=64, queue_capacity=1024, batch_points=4 << 20,
                 chunk_points=1 << 19, inflight_batches=3, device=None):
        import torch
        if device is None:
            device = torch.cuda.current_device()
        self.cfg = ServeConfig(pool_bytes=int(pool_bytes), max_slots=int(max_slots),
                               queue_capacity=int(queue_capacity), batch_points=int(batch_points),
                               chunk_points=int(chunk_points), inflight_batches=int(inflight_batches),
                               device=int(device))
        h = ctypes.c_void_p()
        check(lib().shm_serve_create(ctypes.byref(self.cfg), ctypes.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, n: int, lmax: int, dtype, seed: int = 0, points=None, discard: bool = False,
               strict: bool = False):
        """Returns a ticket, or None when the server answered SHM_EBUSY.
        strict: all-binary64 rows for a float64 request."""
        req = _Request(points=points.data_ptr() if points is not None else None, n=int(n), lmax=int(lmax),
                       dtype=_dtype_code(dtype), seed=int(seed) & 0xFFFFFFFFFFFFFFFF,
                       flags=(SHM_REQ_DISCARD if discard else 0) | (SHM_REQ_STRICT_FP64 if strict else 0))
        t = ctypes.c_uint64(0)
        st = lib().shm_serve_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        if st == 4:
            return None
        check(st)
        if points is not None:
            self._keep[t.value] = points
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1) -> ServeResult:
        r = ServeResult()
        check(lib().shm_serve_wait(self.h, int(ticket), int(timeout_ms), ctypes.byref(r)))
        return r

    def wait_any(self, timeout_ms: int = -1):
        """(status, ticket, result) of the oldest completed request no wait has
        returned yet; status SHM_ETIMEOUT (5) when none completed in time."""
        r = ServeResult()
        t = ctypes.c_uint64(0)
        st = lib().shm_serve_wait_any(self.h, int(timeout_ms), ctypes.byref(t), ctypes.byref(r))
        return st, t.value, r

    def wait_status(self, ticket: int, timeout_ms: int = 0):
        r = ServeResult()
        st = lib().shm_serve_wait(self.h, int(ticket), int(timeout_ms), ctypes.byref(r))
        return st, r

    def result_tensor(self, r: ServeResult):
        """A copy of a completed request's rows as a CUDA tensor [n, (lmax+1)^2]."""
        import torch
        dt = torch.float64 if r.dtype == SHM_F64 else torch.float32
        nh = num_harmonics(r.lmax)
        out = torch.empty((r.n, nh), dtype=dt, device="cuda")
        from cuda.bindings import runtime as rt
        err, = rt.cudaMemcpy(out.data_ptr(), r.out, r.n * nh * out.element_size(),
                             rt.cudaMemcpyKind.cudaMemcpyDeviceToDevice)
        if err != rt.cudaError_t.cudaSuccess:
            raise RuntimeError(f"cudaMemcpy failed: {err}")
        return out

    def release(self, ticket: int) -> None:
        check(lib().shm_serve_release(self.h, int(ticket)))
        self._keep.pop(ticket, None)

    def stats(self) -> dict:
        s = ServeStats()
        check(lib().shm_serve_stats_get(self.h, ctypes.byref(s)))
        return s.as_dict()

    def reset_stats(self) -> None:
        check(lib().shm_serve_stats_reset(self.h))

    def close(self) -> None:
        if self.h:
            check(lib().shm_serve_destroy(self.h))
            self.h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
