"""ctypes binding of lib/libtvolap.so (argument marshalling only).

The C declarations and their contracts are in include/tvolap.h. Loading
fails loudly when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_int, c_int64, c_float, c_void_p = ctypes.c_int, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p
P_int32 = ctypes.POINTER(ctypes.c_int32)
P_int = ctypes.POINTER(ctypes.c_int)
P_int64 = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes); mirrors include/tvolap.h
SIGNATURES = {
    "tvolap_strerror": (ctypes.c_char_p, [c_int]),
    "tvolap_version": (c_int, []),
    "tvolap_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int, c_int, c_int, c_int,
                              P_int32, c_int, c_void_p]),
    "tvolap_destroy": (c_int, [c_void_p]),
    "tvolap_get_dims": (c_int, [c_void_p, P_int, P_int, P_int, P_int, P_int, P_int]),
    "tvolap_slot_count": (c_int, [c_void_p]),
    "tvolap_reset": (c_int, [c_void_p]),
    "tvolap_load_bank": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_int64]),
    "tvolap_set_filter": (c_int, [c_void_p, c_int, c_void_p, c_int]),
    "tvolap_select": (c_int, [c_void_p, c_int, c_int, c_int, c_float]),
    "tvolap_process_block": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "tvolap_process_signal": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_void_p, c_void_p,
                                      c_void_p, c_int64, c_void_p, c_int64, c_int64]),
    "tvolap_signal_workspace_bytes": (c_int64, [c_void_p, c_int64]),
    "tvolap_process_ragged": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p,
                                      c_int64, c_void_p, c_void_p, c_void_p, c_int64, c_void_p,
                                      c_int64]),
    "tvolap_forward_spectra": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int, c_void_p]),
    "tvolap_mac": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int64,
                           c_void_p]),
    "tvolap_inverse_ola": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_int64, c_int64]),
    "tvolap_bank_spectra": (c_int, [c_void_p, c_int, c_void_p]),
    "tvolap_check": (c_int, [c_void_p]),
    "tvolap_set_option": (c_int, [c_void_p, c_int, c_int]),
    "tvolap_stage_times": (c_int, [c_void_p, ctypes.POINTER(ctypes.c_double), P_int64]),
    "tvolap_set_mix": (c_int, [c_void_p, c_int, c_void_p]),
    "tvolap_nu_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int, c_int, c_int, c_int,
                                 c_int, c_void_p,
                                 c_int, c_void_p]),
    "tvolap_nu_destroy": (c_int, [c_void_p]),
    "tvolap_nu_reset": (c_int, [c_void_p]),
    "tvolap_nu_dims": (c_int, [c_void_p, P_int, P_int, P_int64, P_int64]),
    "tvolap_nu_load_bank": (c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_int64]),
    "tvolap_nu_process_signal": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_void_p,
                                         c_void_p, c_void_p, c_int64, c_void_p, c_int64,
                                         c_int64]),
    "tvolap_nu_process_block": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                        c_void_p]),
    "tvolap_nu_check": (c_int, [c_void_p]),
    "tvolap_nu_set_option": (c_int, [c_void_p, c_int, c_int, c_int]),
    "tvolap_state_bytes": (c_int64, [c_void_p]),
    "tvolap_get_state": (c_int, [c_void_p, c_void_p, c_int64]),
    "tvolap_set_state": (c_int, [c_void_p, c_void_p, c_int64]),
    "tvolap_mix": (c_int, [c_void_p, c_void_p, c_int, c_void_p]),
    "tvolap_process_signal_mix": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_void_p,
                                          c_void_p, c_void_p, c_int64, c_void_p, c_int64,
                                          c_int64]),
    "tvolap_process_block_mix": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                         c_void_p]),
    "tvolap_block_spectra": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int64, c_int,
                                     c_void_p]),
    "tvolap_mac_params": (c_int, [c_void_p, c_void_p, c_int64, c_int, c_void_p, c_int64, c_int64,
                                  c_int, c_void_p, c_int64]),
    "tvolap_adjoint_output": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int64, c_int,
                                      c_void_p]),
    "tvolap_adjoint_mac": (c_int, [c_void_p, c_void_p, c_int64, c_int, c_void_p, c_int64, c_int,
                                   c_void_p, c_int64, c_int64, c_int, c_void_p, c_void_p,
                                   c_int64]),
    "tvolap_adjoint_mac_x": (c_int, [c_void_p, c_void_p, c_int64, c_int, c_void_p, c_int64,
                                     c_int64, c_void_p, c_int64, c_int64, c_int, c_void_p,
                                     c_void_p, c_int64]),
    "tvolap_adjoint_input": (c_int, [c_void_p, c_void_p, c_int64, c_int, c_void_p, c_int64,
                                     c_int64]),
    "tvolap_process_signal_static": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_void_p,
                                             c_void_p, c_void_p, c_int64, c_void_p, c_int64,
                                             c_int64]),
    # batched sources
    "tvolap_batch_create": (c_int, [ctypes.POINTER(c_void_p), c_void_p, c_int, c_void_p]),
    "tvolap_batch_destroy": (c_int, [c_void_p]),
    "tvolap_batch_source_view": (c_int, [c_void_p, c_int, ctypes.POINTER(c_void_p),
                                         ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), P_int,
                                         P_int64]),
    "tvolap_batch_set_source": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "tvolap_batch_get_output": (c_int, [c_void_p, c_int, c_void_p]),
    "tvolap_batch_load_filters": (c_int, [c_void_p, c_int, c_void_p, c_int, c_int64]),
    "tvolap_batch_run": (c_int, [c_void_p]),
    "tvolap_batch_capture": (c_int, [c_void_p]),
    "tvolap_batch_autotune": (c_int, [c_void_p, c_int, P_int]),
    "tvolap_batch_set_staging": (c_int, [c_void_p, c_int, c_int]),
    "tvolap_batch_groups": (c_int, [c_void_p, P_int]),
    "tvolap_batch_group_info": (c_int, [c_void_p, c_int, P_int, P_int, P_int]),
    "tvolap_batch_group_tiling": (c_int, [c_void_p, c_int, P_int, P_int]),
    "tvolap_batch_check": (c_int, [c_void_p]),
    # streaming server
    "tvolap_server_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int, c_int, c_int, c_int64,
                                     c_void_p]),
    "tvolap_server_destroy": (c_int, [c_void_p]),
    "tvolap_server_footprint": (c_int, [c_void_p, c_int, c_int, c_int, c_int, P_int64]),
    "tvolap_server_admit": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_int, c_int64,
                                    P_int]),
    "tvolap_server_submit": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_int,
                                     c_int64, P_int64]),
    "tvolap_server_admitted": (c_int, [c_void_p, P_int64, P_int32, P_int64, c_int, P_int]),
    "tvolap_server_cancel": (c_int, [c_void_p, c_int64]),
    "tvolap_server_queue": (c_int, [c_void_p, P_int, P_int64, P_int64, P_int64]),
    "tvolap_server_retire": (c_int, [c_void_p, c_int]),
    "tvolap_server_stream_bytes": (c_int, [c_void_p, c_int, P_int64]),
    "tvolap_server_snapshot": (c_int, [c_void_p, c_int, c_void_p, c_int64]),
    "tvolap_server_restore": (c_int, [c_void_p, c_void_p, c_int64, P_int]),
    "tvolap_server_state": (c_int, [c_void_p, c_int, P_int, P_int64, P_int]),
    "tvolap_server_staging": (c_int, [c_void_p, c_int, ctypes.POINTER(c_void_p), P_int64,
                                      ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), P_int64]),
    "tvolap_server_due": (c_int, [c_void_p, P_int32, c_int, P_int, P_int]),
    "tvolap_server_tick": (c_int, [c_void_p]),
    "tvolap_server_wait": (c_int, [c_void_p]),
    "tvolap_server_post": (c_int, [c_void_p, ctypes.c_uint64]),
    "tvolap_server_set_option": (c_int, [c_void_p, c_int, c_int64]),
    "tvolap_server_stats_get": (c_int, [c_void_p, c_void_p]),
    # host scheduler alone
    "tvolap_sched_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int, c_int, c_int, c_int64]),
    "tvolap_sched_destroy": (c_int, [c_void_p]),
    "tvolap_sched_footprint": (c_int, [c_int, c_int, c_int, c_int, P_int64]),
    "tvolap_sched_admit": (c_int, [c_void_p, c_int, c_int, c_int, c_int, P_int, P_int64, P_int]),
    "tvolap_sched_fail_admits": (c_int, [c_void_p, c_int64]),
    "tvolap_sched_submit": (c_int, [c_void_p, c_int, c_int, c_int, c_int, P_int64]),
    "tvolap_sched_pump": (c_int, [c_void_p, P_int]),
    "tvolap_sched_cancel": (c_int, [c_void_p, c_int64]),
    "tvolap_sched_admitted": (c_int, [c_void_p, P_int64, P_int32, P_int64, c_int, P_int]),
    "tvolap_sched_queue": (c_int, [c_void_p, P_int, P_int64]),
    "tvolap_sched_activate": (c_int, [c_void_p, c_int]),
    "tvolap_sched_retire": (c_int, [c_void_p, c_int]),
    "tvolap_sched_due": (c_int, [c_void_p, P_int32, c_int, P_int]),
    "tvolap_sched_advance": (c_int, [c_void_p]),
    "tvolap_sched_phase_loads": (c_int, [c_void_p, P_int64, c_int, P_int]),
    "tvolap_sched_arena": (c_int, [c_void_p, P_int64, P_int64]),
}

STATUS = {0: "TVOLAP_OK", -1: "TVOLAP_ERR_ARG", -2: "TVOLAP_ERR_OOM", -3: "TVOLAP_ERR_CUDA",
          -4: "TVOLAP_ERR_STATE", -5: "TVOLAP_ERR_CAPACITY", -6: "TVOLAP_ERR_TIMEOUT"}


class TvolapError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


def header_symbols() -> list:
    """Every tvolap_* function declared in include/tvolap.h."""
    with open(_build.HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"TVOLAP_API\s+[\w\s\*]*?\b(tvolap_\w+)\s*\(", text)))


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = False):
    """Load the library (and optionally build it). Raises if it is absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(
                f"TVOLAP CUDA library not built ({path}); run "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(status: int, what: str) -> int:
    if status < 0:
        raise TvolapError(status, what)
    return status
