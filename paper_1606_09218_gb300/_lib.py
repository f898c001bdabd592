"""ctypes binding of ``librs_gb300.so`` (the C ABI declared in ``include/rs.h``).

Argument marshalling only: every step of the method runs in the CUDA library.  If the
library is missing or fails to load, importing the functions raises; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librs_gb300.so")

# status codes (rs_status)
RS_OK = 0
RS_RANK_CAPPED = 1
RS_ERR_INVALID_ARG = -1
RS_ERR_OUTSIDE_BOX = -2
RS_ERR_SEPARATION = -3
RS_ERR_OOM = -4
RS_ERR_CUDA = -5
RS_ERR_TIMEOUT = -6
RS_ERR_NOT_READY = -7
RS_ERR_CAPACITY = -8
STATUS_NAMES = {0: "RS_OK", 1: "RS_RANK_CAPPED", -1: "RS_ERR_INVALID_ARG", -2: "RS_ERR_OUTSIDE_BOX",
                -3: "RS_ERR_SEPARATION", -4: "RS_ERR_OOM", -5: "RS_ERR_CUDA", -6: "RS_ERR_TIMEOUT",
                -7: "RS_ERR_NOT_READY", -8: "RS_ERR_CAPACITY"}

# precisions
RS_FP64, RS_FP32_SPLIT, RS_FP32 = 0, 1, 2
# solve flags
RS_INPUT_HOST, RS_POTENTIAL, RS_ENERGY, RS_FORCES, RS_VALIDATE_SEPARATION, RS_FORCES_PAIR = 1, 2, 4, 8, 16, 32

#: every symbol ``include/rs.h`` declares
EXPORTED = ["rs_create", "rs_destroy", "rs_workspace_bytes", "rs_solve", "rs_energy", "rs_forces", "rs_report",
            "rs_get_tucker", "rs_get_windows", "rs_eval_points", "rs_canonical", "rs_canonical_eval_points", "rs_get_canonical",
            "rs_tucker_als",
            "rs_profile_enable", "rs_profile_read", "rs_stage_name",
            "rs_debug_buffer", "rs_gram_noalloc", "rs_plain_direct", "rs_plain_canonical",
            "rs_pair_energy_forces", "rs_matvec", "rs_energy_matvec",
            "rs_server_create", "rs_submit", "rs_wait", "rs_server_info", "rs_server_destroy",
            "rs_last_error", "rs_version"]
RS_NSTAGE = 9
# rs_matvec flags
RS_MATVEC_LONG, RS_MATVEC_SHORT, RS_MATVEC_OFFDIAG = 1, 2, 4


class RSConfigC(C.Structure):
    _fields_ = [("b", C.c_double), ("n", C.c_int), ("R", C.c_int), ("R_s", C.c_int),
                ("h_q", C.c_double), ("u0", C.c_double), ("eps", C.c_double),
                ("rank_cap", C.c_int), ("max_rank", C.c_int), ("delta_rel", C.c_double),
                ("precision", C.c_int), ("snap", C.c_int), ("max_particles", C.c_int)]


class RSRequestC(C.Structure):
    _fields_ = [("cfg", RSConfigC), ("N", C.c_int), ("xyz", C.c_void_p), ("Z", C.c_void_p),
                ("flags", C.c_int), ("potential_out", C.c_void_p)]


class RSResultC(C.Structure):
    _fields_ = [("status", C.c_int), ("energy", C.c_double), ("latency_ms", C.c_double),
                ("queue_ms", C.c_double), ("ranks", C.c_int * 3), ("slot", C.c_int),
                ("message", C.c_char * 128)]


class RSStatsC(C.Structure):
    _fields_ = [("N", C.c_int), ("N_nonzero", C.c_int), ("ranks", C.c_int * 3),
                ("subspace", C.c_int * 3), ("gamma", C.c_int), ("tail_rel", C.c_double * 3),
                ("eps_bound", C.c_double), ("P_R0", C.c_double), ("P_Rl0", C.c_double),
                ("energy", C.c_double), ("status", C.c_int), ("kernel_launches", C.c_int)]


class RSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load the library once and declare the prototypes of ``include/rs.h``."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RSError(RS_ERR_CUDA, f"{path} is missing; build it with paper_1606_09218_gb300.build")
    lib = C.CDLL(path)
    vp = C.c_void_p
    lib.rs_create.argtypes = [C.POINTER(RSConfigC), vp, C.POINTER(vp)]
    lib.rs_create.restype = C.c_int
    lib.rs_destroy.argtypes = [vp]
    lib.rs_destroy.restype = None
    lib.rs_workspace_bytes.argtypes = [C.POINTER(RSConfigC)]
    lib.rs_workspace_bytes.restype = C.c_size_t
    lib.rs_solve.argtypes = [vp, C.c_int, vp, vp, C.c_int, C.c_double, vp]
    lib.rs_solve.restype = C.c_int
    lib.rs_energy.argtypes = [vp, C.POINTER(C.c_double)]
    lib.rs_energy.restype = C.c_int
    lib.rs_forces.argtypes = [vp, vp, C.c_int]
    lib.rs_forces.restype = C.c_int
    lib.rs_pair_energy_forces.argtypes = [vp, C.c_int, vp, vp, vp, vp]
    lib.rs_pair_energy_forces.restype = C.c_int
    lib.rs_matvec.argtypes = [vp, vp, vp, C.c_int]
    lib.rs_matvec.restype = C.c_int
    lib.rs_energy_matvec.argtypes = [vp, C.POINTER(C.c_double)]
    lib.rs_energy_matvec.restype = C.c_int
    for nm in ("rs_plain_direct", "rs_plain_canonical"):
        getattr(lib, nm).argtypes = [vp, vp]
        getattr(lib, nm).restype = C.c_int
    lib.rs_server_create.argtypes = [C.c_size_t, C.c_int, C.POINTER(vp)]
    lib.rs_server_create.restype = C.c_int
    lib.rs_submit.argtypes = [vp, C.POINTER(RSRequestC), C.POINTER(C.c_ulonglong)]
    lib.rs_submit.restype = C.c_int
    lib.rs_wait.argtypes = [vp, C.c_ulonglong, C.c_int, C.POINTER(RSResultC)]
    lib.rs_wait.restype = C.c_int
    lib.rs_server_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_size_t), C.POINTER(C.c_int)]
    lib.rs_server_info.restype = C.c_int
    lib.rs_server_destroy.argtypes = [vp]
    lib.rs_server_destroy.restype = None
    lib.rs_report.argtypes = [vp, C.POINTER(RSStatsC)]
    lib.rs_report.restype = C.c_int
    lib.rs_get_tucker.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(vp), C.POINTER(vp)]
    lib.rs_get_tucker.restype = C.c_int
    ip = C.POINTER(C.c_int)
    lib.rs_get_windows.argtypes = [vp, ip, ip, ip, C.POINTER(vp), ip, C.POINTER(vp), C.POINTER(vp)]
    lib.rs_get_windows.restype = C.c_int
    lib.rs_eval_points.argtypes = [vp, C.c_int, vp, vp]
    lib.rs_eval_points.restype = C.c_int
    lib.rs_canonical.argtypes = [vp, C.c_double, C.POINTER(C.c_int)]
    lib.rs_canonical.restype = C.c_int
    lib.rs_canonical_eval_points.argtypes = [vp, C.c_int, vp, vp]
    lib.rs_canonical_eval_points.restype = C.c_int
    lib.rs_get_canonical.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(vp), C.POINTER(vp), C.POINTER(C.c_int)]
    lib.rs_get_canonical.restype = C.c_int
    lib.rs_tucker_als.argtypes = [vp, C.c_int, C.c_int, vp]
    lib.rs_tucker_als.restype = C.c_int
    lib.rs_profile_enable.argtypes = [vp, C.c_int]
    lib.rs_profile_enable.restype = C.c_int
    lib.rs_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    lib.rs_profile_read.restype = C.c_int
    lib.rs_stage_name.argtypes = [C.c_int]
    lib.rs_stage_name.restype = C.c_char_p
    lib.rs_debug_buffer.argtypes = [vp, C.c_char_p, C.POINTER(vp), C.POINTER(C.c_size_t)]
    lib.rs_debug_buffer.restype = C.c_int
    lib.rs_gram_noalloc.argtypes = [C.POINTER(RSConfigC), C.c_int, vp, vp, vp, vp]
    lib.rs_gram_noalloc.restype = C.c_int
    lib.rs_last_error.argtypes = [vp]
    lib.rs_last_error.restype = C.c_char_p
    lib.rs_version.argtypes = []
    lib.rs_version.restype = C.c_char_p
    _lib = lib
    return lib


def check(status: int, ctx=None) -> int:
    if status < 0:
        lib = load()
        msg = lib.rs_last_error(ctx).decode() if lib.rs_last_error(ctx) else ""
        raise RSError(status, msg)
    return status
