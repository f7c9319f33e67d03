"""ctypes declarations of the C ABI in include/mrlbm.h (argument marshalling only).

The shared library is built in-tree by ``_build.build()``; loading fails loudly
if it is missing, so no computation can silently run anywhere else.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

MR_OK, MR_ERR_ARG, MR_ERR_CUDA, MR_ERR_CAPACITY, MR_ERR_NONFINITE, MR_ERR_TIMEOUT, MR_ERR_STATE = 0, -1, -2, -3, -4, -5, -6
MR_FP64, MR_FP32_MIXED = 0, 1
MR_BC_PERIODIC, MR_BC_COPY = 0, 1
MR_EQ_ADVECTION, MR_EQ_BURGERS, MR_EQ_SW_VEC, MR_EQ_EULER_VEC = 0, 1, 2, 3
MR_EQ_SW_D1Q3, MR_EQ_SW_D1Q5 = 4, 5
MR_COLLIDE_LEAVES, MR_COLLIDE_RECONSTRUCTED = 0, 1

STATUS_NAMES = {0: "MR_OK", -1: "MR_ERR_ARG", -2: "MR_ERR_CUDA", -3: "MR_ERR_CAPACITY",
                -4: "MR_ERR_NONFINITE", -5: "MR_ERR_TIMEOUT", -6: "MR_ERR_STATE"}


class mr_instance_desc(ctypes.Structure):
    _fields_ = [
        ("Jmin", ctypes.c_int), ("Jmax", ctypes.c_int), ("gamma", ctypes.c_int), ("mu_bar", ctypes.c_int),
        ("bc", ctypes.c_int), ("eq", ctypes.c_int), ("eps", ctypes.c_double), ("a", ctypes.c_double),
        ("b", ctypes.c_double), ("lambda_", ctypes.c_double), ("s", ctypes.c_double * 3),
        ("eq_param", ctypes.c_double), ("collision", ctypes.c_int),
    ]


# name -> (restype, argtypes); every entry point returns mr_status
_P = ctypes.POINTER
_vp, _i, _d, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
SIGNATURES = {
    "mr_mesh_init": [_P(_vp), _i, _i, _i, _d, _d, _d, _i, _i, _i],
    "lbm_scheme": [_vp, _i, _i, _d, _P(_d), _i, _P(_d)],
    "mr_batch_create": [_P(_vp), _P(mr_instance_desc), _i, _i],
    "mr_workspace_size": [_vp, _P(_sz)],
    "mr_bind": [_vp, _vp, _sz, _vp],
    "mr_set_initial": [_vp, _vp, _sz],
    "mr_set_state": [_vp, _i, _vp, _vp],
    "mr_adapt": [_vp],
    "lbm_step": [_vp],
    "mr_advance": [_vp, _i],
    "mr_sync": [_vp],
    "mr_get_leaves": [_vp, _i, _P(_i), _P(ctypes.c_long), _P(_d), ctypes.c_long, _P(ctypes.c_long)],
    "mr_get_moments": [_vp, _i, _P(_d), ctypes.c_long, _P(ctypes.c_long)],
    "mr_get_finest": [_vp, _i, _vp],
    "mr_get_tree": [_vp, _i, _vp],
    "mr_audit": [_vp, _i, _P(_d), _P(_d)],
    "mr_get_summary": [_vp, _P(_d), _P(_i)],
    "mr_near_ties": [_vp, _i, _P(ctypes.c_longlong)],
    "mr_step_passes": [_vp, _i, _P(ctypes.c_ulonglong), _P(ctypes.c_ulonglong)],
    "mr_probe_latency": [_vp, _sz, _vp, _P(_d)],
    "mr_stats": [_vp, _P(ctypes.c_ulonglong), _P(ctypes.c_ulonglong), _P(ctypes.c_longlong)],
    "mr_set_launch": [_vp, _i, _i],
    "mr_set_order": [_vp, _i],
    "mr_set_collision": [_vp, _i],
    "mr_autotune": [_vp, _i, _vp, ctypes.c_size_t, _P(_i), _P(_i), _P(ctypes.c_float)],
    "mr_reconstruction_coefficients": [_i, _i, _P(_d)],
    "mr_phase_times": [_vp, _i, _P(ctypes.c_ulonglong), _i],
    "mr_info": [_vp, _P(_i), _P(ctypes.c_longlong)],
    "mr_last_error": [_vp, ctypes.c_char_p, _i],
    "mr_destroy": [_vp],
    "mr_run_static": [_P(mr_instance_desc), _i, _vp, _i, _vp, _P(ctypes.c_ulonglong), _vp],
}

_lib = None


PHASES = ["projection (adapt)", "details + threshold", "enlargement", "grading + marking",
          "grading (small levels)", "candidate words", "list compaction", "data transfer", "collision",
          "projection (step)", "ghosts", "reconstruction", "stream + audit"]


def load(build_if_missing: bool = True, profile: bool = False) -> ctypes.CDLL:
    """Load libmrlbm.so (or the phase-timer build with profile=True); raises if
    it cannot be built or loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.PROF_LIB if profile else _build.LIB
    if not os.path.exists(path) or not _build.up_to_date(profile):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
        _build.build(profile=profile)
    L = ctypes.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = ctypes.c_int
        fn.argtypes = args
    _lib = L
    return L


def exported_symbols() -> list[str]:
    return list(SIGNATURES)


class MRError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(ctx, code: int) -> None:
    if code != MR_OK:
        buf = ctypes.create_string_buffer(512)
        load().mr_last_error(ctx, buf, 512)
        raise MRError(code, buf.value.decode(errors="replace"))
