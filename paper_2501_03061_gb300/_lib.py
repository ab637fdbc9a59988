"""ctypes declarations of the C ABI in include/ptim.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libptim.so")

PT_OK, PT_INVALID_ARG, PT_OOM, PT_NOT_PD, PT_NOT_CONVERGED, PT_NONFINITE, PT_TIMEOUT, PT_CUDA, PT_UNSUPPORTED = range(9)
STATUS_NAMES = {0: "PT_OK", 1: "PT_INVALID_ARG", 2: "PT_OOM", 3: "PT_NOT_PD", 4: "PT_NOT_CONVERGED",
                5: "PT_NONFINITE", 6: "PT_TIMEOUT", 7: "PT_CUDA", 8: "PT_UNSUPPORTED"}
PRECISIONS = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}
PT_MAX_ORBITALS = 32768  # largest orbital count a call accepts


class pt_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("L", C.c_double * 3)]


class pt_kernel(C.Structure):
    _fields_ = [("type", C.c_int), ("mu", C.c_double), ("g0", C.c_double)]


class pt_exchange_item(C.Structure):
    _fields_ = [("src", C.c_void_p), ("occ", C.c_void_p), ("N", C.c_int), ("tgt", C.c_void_p), ("M", C.c_int),
                ("out", C.c_void_p), ("grid", pt_grid), ("kernel", pt_kernel)]


class pt_ptim_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("alpha", C.c_double), ("ecut", C.c_double), ("tol", C.c_double),
                ("max_outer", C.c_int), ("max_inner", C.c_int), ("anderson_depth", C.c_int),
                ("anderson_beta", C.c_double), ("use_ace", C.c_int), ("spin", C.c_double), ("hxc", C.c_int),
                ("A", C.c_double * 3)]


class pt_ptim_stats(C.Structure):
    _fields_ = [("outer", C.c_int), ("inner", C.c_int), ("residual", C.c_double), ("exch_energy", C.c_double),
                ("orth_error", C.c_double), ("converged", C.c_int), ("pair_ffts", C.c_longlong),
                ("exchange_calls", C.c_int), ("exchange_ms", C.c_double), ("phase_ms", C.c_double * 12),
                ("eig_sweeps", C.c_int), ("total_energy", C.c_double), ("pure_state", C.c_int),
                ("ace_warm", C.c_int), ("passes", C.c_int), ("pass_inner", C.c_int * 16),
                ("sinv_path", C.c_int * 4), ("sinv_mixed_fallback", C.c_int), ("s_dev_max", C.c_double),
                ("plane_waves", C.c_int)]

PHASES = ("exchange", "ace_build", "ace_apply", "apply_H", "subspace_gemm", "subspace_nxn", "sigma_eig",
          "sigma_rot", "commutator", "anderson", "loewdin", "hxc")


vp = C.c_void_p
i32 = C.c_int
PROTOTYPES = {
    "pt_create": (i32, [C.POINTER(vp), i32, C.c_size_t]),
    "pt_destroy": (None, [vp]),
    "pt_last_error": (C.c_char_p, [vp]),
    "pt_workspace_bytes": (C.c_size_t, [vp]),
    "pt_trim": (i32, [vp]),
    "pt_set_option": (i32, [vp, C.c_char_p, C.c_double]),
    "pt_apply_exchange": (i32, [vp, vp, vp, i32, vp, i32, vp, C.POINTER(pt_grid), C.POINTER(pt_kernel), i32, vp]),
    "pt_apply_exchange_mixed": (i32, [vp, vp, vp, i32, vp, i32, vp, C.POINTER(pt_grid), C.POINTER(pt_kernel), i32,
                                      C.POINTER(C.c_longlong), vp]),
    "pt_apply_exchange_noalloc": (i32, [vp, vp, i32, vp, i32, vp, C.POINTER(pt_grid), C.POINTER(pt_kernel), i32, vp]),
    "pt_apply_exchange_batched": (i32, [vp, C.POINTER(pt_exchange_item), i32, i32, C.POINTER(C.c_longlong),
                                        C.POINTER(C.c_size_t), vp]),
    "pt_build_ace": (i32, [vp, vp, vp, i32, C.POINTER(pt_grid), C.POINTER(pt_kernel), i32, C.POINTER(vp), vp]),
    "pt_build_ace_from": (i32, [vp, vp, vp, i32, C.POINTER(pt_grid), i32, C.POINTER(vp), vp]),
    "pt_apply_ace": (i32, [vp, vp, vp, i32, vp, vp]),
    "pt_ace_get_xi": (i32, [vp, vp, vp]),
    "pt_ace_destroy": (None, [vp]),
    "pt_overlap": (i32, [vp, vp, i32, vp, i32, C.POINTER(pt_grid), i32, vp, vp]),
    "pt_rotate": (i32, [vp, vp, i32, vp, i32, C.POINTER(pt_grid), i32, vp, vp]),
    "pt_apply_H": (i32, [vp, vp, i32, vp, vp, vp, C.c_double, C.c_double, C.POINTER(C.c_double),
                         C.POINTER(pt_grid), i32, vp]),
    "pt_current": (i32, [vp, vp, vp, i32, C.POINTER(pt_grid), i32, C.POINTER(C.c_double), C.c_double,
                         C.POINTER(C.c_double), vp]),
    "pt_diag_occupations": (i32, [vp, vp, i32, vp, vp, vp]),
    "pt_density": (i32, [vp, vp, vp, i32, C.POINTER(pt_grid), i32, C.c_double, vp, vp]),
    "pt_hxc_potential": (i32, [vp, vp, vp, C.POINTER(pt_grid), vp, C.POINTER(C.c_double), vp]),
    "pt_ptim_step": (i32, [vp, vp, vp, i32, vp, C.POINTER(pt_grid), C.POINTER(pt_kernel),
                           C.POINTER(pt_ptim_params), i32, C.POINTER(pt_ptim_stats), vp]),
    "pt_ptim_footprint": (C.c_size_t, [i32, C.POINTER(pt_grid), i32, i32]),
    "pt_version": (C.c_char_p, []),
    "pt_kernel_launches": (C.c_longlong, []),
    "pt_selftest_wait": (i32, [vp, i32, C.c_double, vp]),
    "pt_alu_peaks": (i32, [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]),
}

_lib = None


def load(path: str | None = None):
    """Load libptim.so and declare every prototype.  Raises if the library is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(p)
    for name, (res, args) in PROTOTYPES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib
