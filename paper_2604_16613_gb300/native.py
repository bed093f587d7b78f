"""ctypes declarations of the C ABI in include/gpdem.h and include/gpserve.h
(argument marshalling only).

Loading fails loudly when ``_lib/libgpdem.so`` has not been built: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libgpdem.so")

GP_OK, GP_ERR_INVALID, GP_ERR_NONDETERMINISTIC, GP_ERR_CAPACITY, GP_ERR_CUDA, GP_ERR_TIMEOUT, GP_ERR_HORIZON = range(7)
STATUS_NAMES = {0: "GP_OK", 1: "GP_ERR_INVALID", 2: "GP_ERR_NONDETERMINISTIC", 3: "GP_ERR_CAPACITY",
                4: "GP_ERR_CUDA", 5: "GP_ERR_TIMEOUT", 6: "GP_ERR_HORIZON"}
LEVELS = {"L0": 0, "L1": 1, "L2": 2, 0: 0, 1: 1, 2: 2}

# every symbol include/gpdem.h declares
EXPORTED = [
    "gp_workspace_size", "gp_driver_create", "gp_driver_destroy", "gp_compile_batch", "gp_compile",
    "gp_backward", "gp_result_view", "gp_result_to_host", "gp_set_tuning", "gp_get_tuning", "gp_enable_timing",
    "gp_last_timing", "gp_last_launch_count", "gp_last_error", "gp_set_debug", "gp_pmerge_noalloc",
    "gp_server_create", "gp_server_destroy", "gp_server_open_patch", "gp_server_close_patch",
    "gp_server_submit", "gp_server_step", "gp_server_completed", "gp_server_result", "gp_server_release",
    "gp_server_register_cycle", "gp_server_submit_registered", "gp_server_submit_registered_many",
    "gp_server_drain", "gp_server_last_timing", "gp_server_set_tuning", "gp_set_host_output",
]


class GpBounds(ctypes.Structure):
    _fields_ = [("max_circuits", ctypes.c_uint32), ("max_qubits", ctypes.c_uint32),
                ("max_ops", ctypes.c_uint64), ("max_recs", ctypes.c_uint64),
                ("max_layers", ctypes.c_uint32), ("max_measurements", ctypes.c_uint32),
                ("max_detectors", ctypes.c_uint32), ("max_locations", ctypes.c_uint32),
                ("max_mechanisms", ctypes.c_uint32), ("max_mask_words", ctypes.c_uint32),
                ("max_det_entries", ctypes.c_uint64)]


class GpCircuit(ctypes.Structure):
    _fields_ = [("ops", ctypes.c_void_p), ("n_ops", ctypes.c_uint64),
                ("recs", ctypes.c_void_p), ("n_recs", ctypes.c_uint64),
                ("n_qubits", ctypes.c_uint32), ("n_detectors", ctypes.c_uint32),
                ("n_observables", ctypes.c_uint32), ("n_locations", ctypes.c_uint32)]


class GpDemView(ctypes.Structure):
    _fields_ = [("n_circuits", ctypes.c_uint32), ("n_edges", ctypes.c_uint32),
                ("n_det_entries", ctypes.c_uint64), ("n_mechanisms", ctypes.c_uint32),
                ("pad", ctypes.c_uint32),
                ("det_offsets", ctypes.c_void_p), ("det_idx", ctypes.c_void_p),
                ("obs_mask", ctypes.c_void_p), ("prob", ctypes.c_void_p),
                ("logodds", ctypes.c_void_p), ("edge_circuit", ctypes.c_void_p),
                ("mech_class", ctypes.c_void_p), ("edge_offsets", ctypes.POINTER(ctypes.c_uint32))]


class GpTuning(ctypes.Structure):
    _fields_ = [("stage1_threads", ctypes.c_uint32), ("stage1_blocks_per_sm", ctypes.c_uint32),
                ("stage2_threads", ctypes.c_uint32), ("stage2_blocks_per_sm", ctypes.c_uint32),
                ("obs_words", ctypes.c_uint32), ("obs_segments", ctypes.c_uint32),
                ("stage1_wide_emit", ctypes.c_uint32)]


class GpHostOutput(ctypes.Structure):
    _fields_ = [("det_offsets", ctypes.c_void_p), ("det_idx", ctypes.c_void_p), ("obs_mask", ctypes.c_void_p),
                ("prob", ctypes.c_void_p), ("logodds", ctypes.c_void_p), ("edges_cap", ctypes.c_uint64),
                ("det_cap", ctypes.c_uint64)]


class GpDebug(ctypes.Structure):
    _fields_ = [("weak_hash", ctypes.c_uint32), ("wait_limit", ctypes.c_uint32),
                ("stall_windows", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class GpServerConfig(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in (
        "max_patches", "max_batch", "max_cycles_per_step", "max_horizon", "max_pending", "max_qubits",
        "max_cycle_ops", "max_cycle_recs", "max_cycle_locations", "max_cycle_measurements",
        "max_cycle_detectors", "max_cycle_mechanisms", "max_cycle_layers", "max_logical_qubits")]


class GpPatchSpec(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_uint32), ("horizon", ctypes.c_uint32), ("n_observables", ctypes.c_uint32),
                ("logical_qubits", ctypes.POINTER(ctypes.c_uint32)),
                ("logical_offsets", ctypes.POINTER(ctypes.c_uint32))]


class GpSealedView(ctypes.Structure):
    _fields_ = [("request", ctypes.c_uint64), ("patch", ctypes.c_uint32), ("cycle", ctypes.c_uint32),
                ("status", ctypes.c_int), ("n_edges", ctypes.c_uint32), ("n_det_entries", ctypes.c_uint64),
                ("det_offsets", ctypes.POINTER(ctypes.c_uint32)), ("det_idx", ctypes.POINTER(ctypes.c_uint32)),
                ("obs_mask", ctypes.POINTER(ctypes.c_uint64)), ("prob", ctypes.POINTER(ctypes.c_float)),
                ("logodds", ctypes.POINTER(ctypes.c_float)), ("t_arrival_ns", ctypes.c_uint64),
                ("t_done_ns", ctypes.c_uint64)]


class GpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load libgpdem.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2604_16613_gb300.build.build() "
                               "(nvcc, sm_103a); there is no CPU fallback")
        lib = ctypes.CDLL(path)
        vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        lib.gp_workspace_size.argtypes = [ctypes.POINTER(GpBounds), ctypes.POINTER(u64)]
        lib.gp_driver_create.argtypes = [ctypes.POINTER(GpBounds), vp, u64, ctypes.POINTER(vp)]
        lib.gp_driver_destroy.argtypes = [vp]
        lib.gp_driver_destroy.restype = None
        lib.gp_compile_batch.argtypes = [vp, ctypes.POINTER(GpCircuit), u32, vp, i32, i32, vp,
                                         ctypes.POINTER(GpDemView)]
        lib.gp_compile.argtypes = [vp, ctypes.POINTER(GpCircuit), vp, i32, i32, vp, ctypes.POINTER(GpDemView)]
        lib.gp_backward.argtypes = [vp, vp, vp, vp, vp]
        lib.gp_result_view.argtypes = [vp, ctypes.POINTER(GpDemView)]
        lib.gp_result_to_host.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.gp_set_tuning.argtypes = [vp, ctypes.POINTER(GpTuning)]
        lib.gp_set_host_output.argtypes = [vp, ctypes.POINTER(GpHostOutput)]
        lib.gp_get_tuning.argtypes = [vp, ctypes.POINTER(GpTuning)]
        lib.gp_enable_timing.argtypes = [vp, i32]
        lib.gp_last_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
        lib.gp_last_launch_count.argtypes = [vp]
        lib.gp_last_launch_count.restype = u32
        lib.gp_set_debug.argtypes = [vp, ctypes.POINTER(GpDebug)]
        lib.gp_pmerge_noalloc.argtypes = [vp, vp, u32, u32, vp, vp, vp]
        lib.gp_pmerge_noalloc.restype = i32
        lib.gp_server_create.argtypes = [ctypes.POINTER(GpServerConfig), ctypes.POINTER(vp)]
        lib.gp_server_destroy.argtypes = [vp]
        lib.gp_server_destroy.restype = None
        lib.gp_server_open_patch.argtypes = [vp, ctypes.POINTER(GpPatchSpec), ctypes.POINTER(u32)]
        lib.gp_server_close_patch.argtypes = [vp, u32]
        lib.gp_server_submit.argtypes = [vp, u32, ctypes.POINTER(GpCircuit), vp, i32, u64,
                                         ctypes.POINTER(u64)]
        lib.gp_server_step.argtypes = [vp, i32, vp, ctypes.POINTER(u32)]
        lib.gp_server_completed.argtypes = [vp, ctypes.POINTER(u64), u32, ctypes.POINTER(u32)]
        lib.gp_server_result.argtypes = [vp, u64, ctypes.POINTER(GpSealedView)]
        lib.gp_server_release.argtypes = [vp, u64]
        lib.gp_server_register_cycle.argtypes = [vp, u32, ctypes.POINTER(GpCircuit), vp, ctypes.POINTER(u32)]
        lib.gp_server_submit_registered.argtypes = [vp, u32, u32, i32, u64, ctypes.POINTER(u64)]
        lib.gp_server_submit_registered_many.argtypes = [vp, u32, vp, vp, vp, vp, vp, ctypes.POINTER(u32)]
        lib.gp_server_drain.argtypes = [vp, u32, vp, vp, vp, vp, vp, ctypes.POINTER(u32)]
        lib.gp_server_last_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
        lib.gp_server_set_tuning.argtypes = [vp, ctypes.POINTER(GpTuning)]
        for name in ("gp_server_create", "gp_server_open_patch", "gp_server_close_patch", "gp_server_submit",
                     "gp_server_step", "gp_server_completed", "gp_server_result", "gp_server_release",
                     "gp_server_register_cycle", "gp_server_submit_registered",
                     "gp_server_submit_registered_many", "gp_server_drain", "gp_server_last_timing",
                     "gp_server_set_tuning"):
            getattr(lib, name).restype = i32
        lib.gp_last_error.argtypes = []
        lib.gp_last_error.restype = ctypes.c_char_p
        for name in ("gp_workspace_size", "gp_driver_create", "gp_compile_batch", "gp_compile",
                     "gp_backward", "gp_result_view", "gp_result_to_host", "gp_set_tuning",
                     "gp_get_tuning", "gp_enable_timing", "gp_last_timing", "gp_set_debug", "gp_set_host_output"):
            getattr(lib, name).restype = i32
        _lib = lib
        return lib


def check(code: int) -> None:
    if code != GP_OK:
        msg = load().gp_last_error()
        raise GpError(code, msg.decode() if msg else "")
