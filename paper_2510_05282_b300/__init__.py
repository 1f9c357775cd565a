"""B300-native real spherical harmonics R_l^m (l <= 9) after arXiv 2510.05282.

The computation lives in libshm.so (hand-written CUDA for sm_103a behind a C
ABI, include/shm.h); this package is its thin Python binding plus the seeded
input generators used by tests and benchmarks.
"""
from ._binding import (LMAX_CAP, SHM_F32, SHM_F64, ShmError, autotune, check, eval_angles,  # noqa: F401
                       eval_complex, eval_spinor, num_spinors, eval_host,
                       eval_host_workspace_size, eval_sh, eval_variant, eval_variant_count, lib,
                       num_harmonics, set_eval_variant, DeviceProjectors, projectors, projectors_check,
                       projectors_noalloc, Server, serve_generated_point, probe_fp64_rate, probe_dmul,
                       SHM_STRICT_FP64, projectors_prepare, projectors_run, projectors_autotune,
                       projectors_variant, projectors_variant_count, set_projectors_variant,
                       set_projectors_strict_form, projectors_strict_form)
from . import inputs  # noqa: F401
