"""ctypes declarations of the C ABI in ``include/rvea.h``.

Argument marshalling only: every step of a generation runs in the CUDA
library.  Loading fails loudly when the library is missing; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_LATTICE, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_STATE, ERR_DEVICE = (
    0, -1, -2, -3, -4, -5, -6, -7)
DTLZ2_SPHERE, DTLZ1_LINEAR, NEURO_LINEAR, DTLZ3_SPHERE, DTLZ4_SPHERE = 0, 1, 2, 3, 4
REPRO_SBX_PM, REPRO_DE, REPRO_RANDOM, REPRO_CSO, REPRO_PSO = 0, 1, 2, 3, 4


class NeuroDynamics(C.Structure):
    _fields_ = [("ns", C.c_int), ("na", C.c_int), ("h1", C.c_int), ("h2", C.c_int),
                ("steps", C.c_int), ("sigma", C.c_double),
                ("A", C.POINTER(C.c_double)), ("B", C.POINTER(C.c_double)),
                ("gemv", C.c_int)]


class Config(C.Structure):
    _fields_ = [("m", C.c_int), ("d", C.c_int), ("N", C.c_int), ("H", C.c_int),
                ("problem", C.c_int), ("t_max", C.c_int),
                ("alpha", C.c_double), ("f_r", C.c_double), ("eta_c", C.c_double),
                ("eta_m", C.c_double), ("p_c", C.c_double), ("p_m", C.c_double),
                ("lower", C.c_double), ("upper", C.c_double), ("seed", C.c_uint64),
                ("neuro", C.POINTER(NeuroDynamics)), ("reproduction", C.c_int),
                ("de_F", C.c_double), ("de_CR", C.c_double), ("cso_phi", C.c_double),
                ("pso_w", C.c_double), ("pso_c1", C.c_double), ("pso_c2", C.c_double)]


class Plan(C.Structure):
    _fields_ = [("sel_mode", C.c_int), ("sel_per_sm", C.c_int), ("repro_staged", C.c_int),
                ("repro_us", C.c_double), ("sel_us", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("live", C.c_int), ("queued", C.c_int), ("finished", C.c_int),
                ("admitted", C.c_int), ("arena_used", C.c_size_t), ("generations", C.c_longlong)]


class RveaError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = lib().rvea_status_str(status).decode()
        if status == ERR_CUDA:
            msg += " [" + lib().rvea_last_cuda_error().decode() + "]"
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")


def check(status: int, what: str = "") -> None:
    if status != OK:
        raise RveaError(status, what)


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load (building first if needed) the in-tree librvea.so."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError("librvea.so is missing and could not be built")
        L = C.CDLL(_build.LIB)
        vp, sz, i32, u64, dbl, flt = C.c_void_p, C.c_size_t, C.c_int, C.c_uint64, C.c_double, C.c_float
        run_pp = C.POINTER(C.c_void_p)
        L.rvea_lattice_for.argtypes = [i32, i32]
        L.rvea_lattice_for.restype = i32
        L.rvea_workspace_bytes.argtypes = [i32, i32, i32]
        L.rvea_workspace_bytes.restype = sz
        L.rvea_workspace_bytes_ex.argtypes = [C.POINTER(Config)]
        L.rvea_workspace_bytes_ex.restype = sz
        L.rvea_init.argtypes = [i32, i32, i32, i32, dbl, dbl, dbl, dbl, u64, i32, i32, vp, sz, vp, run_pp]
        L.rvea_init.restype = i32
        L.rvea_init_ex.argtypes = [C.POINTER(Config), vp, sz, vp, run_pp]
        L.rvea_init_ex.restype = i32
        L.rvea_step.argtypes = [vp, i32, vp]
        L.rvea_step.restype = i32
        L.rvea_step_batch.argtypes = [C.POINTER(C.c_void_p), i32, vp]
        L.rvea_step_batch.restype = i32
        L.rvea_population.argtypes = [vp, vp, vp, vp]
        L.rvea_population.restype = i32
        L.rvea_objectives.argtypes = [vp, vp, vp, vp]
        L.rvea_igd.argtypes = [vp, vp, i32, C.POINTER(C.c_double), vp]
        L.rvea_igd.restype = i32
        L.rvea_selftest_wait.argtypes = [i32, vp]
        L.rvea_selftest_wait.restype = i32
        L.rvea_hypervolume.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
        L.rvea_hypervolume.restype = i32
        L.rvea_objectives.restype = i32
        L.rvea_sync_status.argtypes = [vp]
        L.rvea_sync_status.restype = i32
        L.rvea_free.argtypes = [vp]
        L.rvea_free.restype = None
        L.rvea_status_str.argtypes = [i32]
        L.rvea_status_str.restype = C.c_char_p
        L.rvea_last_cuda_error.argtypes = []
        L.rvea_last_cuda_error.restype = C.c_char_p
        L.rvea_generation.argtypes = [vp]
        L.rvea_generation.restype = i32
        L.rvea_launches_per_generation.argtypes = [vp, i32]
        L.rvea_launches_per_generation.restype = i32
        L.rvea_step_profiled.argtypes = [vp, i32, vp, C.POINTER(C.c_double), i32]
        L.rvea_step_profiled.restype = i32
        L.rvea_export_state.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.rvea_export_state.restype = i32
        L.rvea_import_state.argtypes = [vp, vp, vp, vp, vp, vp, i32, vp]
        L.rvea_import_state.restype = i32
        L.rvea_offspring.argtypes = [vp, vp, vp, vp]
        L.rvea_offspring.restype = i32
        L.rvea_export_swarm.argtypes = [vp, vp, vp, vp, vp, vp]
        L.rvea_export_swarm.restype = i32
        L.rvea_import_swarm.argtypes = [vp, vp, vp, vp, vp, vp]
        L.rvea_import_swarm.restype = i32
        L.rvea_last_selection.argtypes = [vp, vp, vp, vp]
        L.rvea_last_selection.restype = i32
        L.rvea_record_draws.argtypes = [vp, i32, vp]
        L.rvea_record_draws.restype = i32
        L.rvea_last_draws.argtypes = [vp, vp, vp, vp]
        L.rvea_last_draws.restype = i32
        L.rvea_select_scratch_bytes.argtypes = [i32, i32, i32]
        L.rvea_select_scratch_bytes.restype = sz
        L.rvea_select.argtypes = [i32, i32, vp, vp, i32, vp, vp, i32, i32, flt, vp, vp, vp, sz, vp]
        L.rvea_select.restype = i32
        L.rvea_select_noalloc.argtypes = [i32, i32, vp, vp, i32, vp, vp, i32, i32, flt, vp, vp, vp]
        L.rvea_select_noalloc.restype = i32
        L.rvea_gamma.argtypes = [i32, i32, vp, vp, vp]
        L.rvea_gamma.restype = i32
        L.rvea_get_plan.argtypes = [vp, C.POINTER(Plan)]
        L.rvea_get_plan.restype = i32
        L.rvea_set_plan.argtypes = [vp, C.POINTER(Plan), vp]
        L.rvea_set_plan.restype = i32
        L.rvea_autotune.argtypes = [vp, vp, i32, C.POINTER(Plan)]
        L.rvea_autotune.restype = i32
        L.rvea_batch_create.argtypes = [C.POINTER(C.c_void_p), i32, C.POINTER(C.c_void_p)]
        L.rvea_batch_create.restype = i32
        L.rvea_batch_step.argtypes = [vp, i32, vp]
        L.rvea_batch_step.restype = i32
        L.rvea_batch_launches_per_step.argtypes = [vp]
        L.rvea_batch_launches_per_step.restype = i32
        L.rvea_batch_step_profiled.argtypes = [vp, i32, vp, C.POINTER(C.c_double), i32]
        L.rvea_batch_step_profiled.restype = i32
        L.rvea_batch_free.argtypes = [vp]
        L.rvea_batch_free.restype = None
        L.rvea_server_create.argtypes = [vp, sz, i32, i32, C.POINTER(C.c_void_p)]
        L.rvea_server_create.restype = i32
        L.rvea_server_submit.argtypes = [vp, C.POINTER(Config), i32, C.POINTER(C.c_int64)]
        L.rvea_server_submit.restype = i32
        L.rvea_server_step.argtypes = [vp, vp, C.POINTER(ServerStats)]
        L.rvea_server_step.restype = i32
        L.rvea_server_poll.argtypes = [vp, C.POINTER(C.c_int64), i32, C.POINTER(C.c_int)]
        L.rvea_server_poll.restype = i32
        L.rvea_server_fetch.argtypes = [vp, C.c_int64, vp, vp, vp, vp]
        L.rvea_server_fetch.restype = i32
        L.rvea_server_free.argtypes = [vp]
        L.rvea_server_free.restype = None
        _lib = L
    return _lib
