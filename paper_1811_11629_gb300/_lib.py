"""ctypes binding of librsaprng (include/rsaprng.h). Argument marshalling only.

Every generation step runs in the library's CUDA kernels; this module only
converts Python values and torch tensors into the pointers and sizes of the
C ABI. If the compiled library is missing, loading fails loudly: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

u64, u32, i32, dbl = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_double
vp = ctypes.c_void_p
pu64 = ctypes.POINTER(ctypes.c_uint64)
pu32 = ctypes.POINTER(ctypes.c_uint32)
pdbl = ctypes.POINTER(ctypes.c_double)
pvp = ctypes.POINTER(ctypes.c_void_p)

OK = 0
MODEXP_AUTO, MODEXP_CRT32, MODEXP_MONT64 = 0, 1, 2
DIVIDE_AUTO, DIVIDE_INT, DIVIDE_FP64, DIVIDE_HYBRID, DIVIDE_RECIP = 0, 1, 2, 3, 4
LOOKBACK_AUTO, LOOKBACK_OFF, LOOKBACK_CONFIGURED = 0, 1, 2
E_SMALLEST, E_UNIFORM, E_AT_LEAST = 0, 1, 2
HIST_HIGH, HIST_LOW = 0, 1
ROUND_DEFAULT, ROUND_PAPER, ROUND_EXACT = 0, 1, 2
Q = (1 << 63) - 25
DEFAULT_ROOT = 2307085864

ERRORS = {
    -1: "ERR_ARG", -2: "ERR_NOT_PRIME", -3: "ERR_RANGE", -4: "ERR_P_EQ_Q", -5: "ERR_E",
    -6: "ERR_ROOT", -7: "ERR_OOM", -8: "ERR_BUDGET", -9: "ERR_CUDA", -10: "ERR_TIMEOUT",
    -11: "ERR_DEVICE_FLAG", -12: "ERR_CAPACITY", -13: "ERR_CANCELLED", -14: "ERR_STATE",
    -15: "ERR_ID", -16: "ERR_BUSY",
}
CODES = {v: k for k, v in ERRORS.items()}


class Config(ctypes.Structure):
    _fields_ = [("struct_size", u32), ("modexp", i32), ("divide", i32),
                ("threads_per_block", i32), ("numbers_per_thread", i32), ("blocks_per_sm", i32),
                ("chunk", u64), ("require_safe", i32), ("rounding", i32),
                ("lookback", i32), ("spin_limit", i32), ("test_flags", i32),
                ("streams_per_block", i32), ("unroll", i32), ("pieces_per_block", i32)]


class Stats(ctypes.Structure):
    _fields_ = [("submitted", u64), ("admitted", u64), ("completed", u64), ("rejected", u64),
                ("cancelled", u64), ("queued_now", u64), ("inflight_now", u64),
                ("numbers_done", u64), ("p50_ms", dbl), ("p99_ms", dbl), ("mean_ms", dbl),
                ("max_ms", dbl), ("busy_s", dbl), ("wall_s", dbl), ("iterations", u64),
                ("max_inflight_iterations", u64), ("overlapped_iterations", u64)]


# name: (restype, argtypes) for every symbol declared in include/rsaprng.h
SIGNATURES = {
    "rsaprng_ctx_create": (i32, [pvp, i32, u64, ctypes.POINTER(Config)]),
    "rsaprng_ctx_destroy": (None, [vp]),
    "rsaprng_device_status": (i32, [vp, vp]),
    "rsaprng_ctx_configure": (i32, [vp, ctypes.POINTER(Config)]),
    "rsaprng_ctx_get_config": (i32, [vp, ctypes.POINTER(Config)]),
    "rsaprng_instance_count": (u64, [vp]),
    "rsaprng_instance_create": (i32, [vp, u64, u64, u64, u64, pu32]),
    "rsaprng_instance_create_ex": (i32, [vp, u64, u64, u64, u64, u64, u64, pu32]),
    "rsaprng_instances_create_bulk": (i32, [vp, u64, pu64, pu64, pu64, pu64, pu32]),
    "rsaprng_instances_create_seeded": (i32, [vp, u64, pu64, i32, u64, u64, pu32]),
    "rsaprng_split": (i32, [vp, u32, u32, pu32]),
    "rsaprng_get_state": (i32, [vp, u32, pu64, pu64]),
    "rsaprng_set_state": (i32, [vp, u32, u64, u64]),
    "rsaprng_get_params": (i32, [vp, u32, pu64, pu64, pu64, pu64]),
    "rsaprng_generate_u64": (i32, [vp, u32, u64, vp, vp]),
    "rsaprng_generate_f64": (i32, [vp, u32, u64, vp, vp]),
    "rsaprng_generate_both": (i32, [vp, u32, u64, vp, vp, vp]),
    "rsaprng_generate_f64_noalloc": (i32, [vp, u32, u64, vp, vp]),
    "rsaprng_latency_shape": (i32, [u64, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]),
    "rsaprng_generate_batch": (i32, [vp, u64, pu32, pu64, pu64, vp, vp, vp]),
    "rsaprng_generate_batch_host": (i32, [vp, u64, pu32, pu64, pu64, vp, vp, vp]),
    "rsaprng_histogram": (i32, [vp, u64, pu32, pu64, u32, u32, i32, vp, vp]),
    "rsaprng_generate_interleaved": (i32, [vp, u64, u32, pu32, u64, vp, vp, vp]),
    "rsaprng_instance_create_crt": (i32, [vp, u64, u64, u64, u64, u64, u64, u64, pu32]),
    "rsaprng_get_exponents": (i32, [vp, u32, pu64, pu64]),
    "rsaprng_chi2_uniform": (i32, [pu64, u64, pdbl, pu64]),
    "rsaprng_plan_create": (i32, [vp, u64, pu32, pu64, pu64, pvp]),
    "rsaprng_plan_launch": (i32, [vp, vp, vp, vp]),
    "rsaprng_plan_launch_timed": (i32, [vp, vp, vp, vp, vp, vp]),
    "rsaprng_plan_capture": (i32, [vp, vp, vp, vp]),
    "rsaprng_plan_replay": (i32, [vp, vp]),
    "rsaprng_plan_info": (i32, [vp, pu64, pu64, pu64]),
    "rsaprng_plan_shape": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                 ctypes.POINTER(i32), ctypes.POINTER(i32)]),
    "rsaprng_plan_destroy": (None, [vp]),
    "rsaprng_autotune": (i32, [vp, u64, pu32, pu64, i32, ctypes.POINTER(Config)]),
    "rsaprng_autotune_cached": (i32, [vp, u64, pu32, pu64, i32, ctypes.POINTER(Config),
                                      ctypes.POINTER(i32)]),
    "rsaprng_autotune_cache_size": (u64, []),
    "rsaprng_autotune_cache_clear": (None, []),
    "rsaprng_autotune_cache_save": (i32, [ctypes.c_char_p]),
    "rsaprng_autotune_cache_load": (i32, [ctypes.c_char_p]),
    "rsaprng_server_create": (i32, [vp, u64, i32, pvp]),
    "rsaprng_server_submit": (i32, [vp, u32, u64, pu64]),
    "rsaprng_server_poll": (i32, [vp, u64, ctypes.POINTER(i32)]),
    "rsaprng_server_wait": (i32, [vp, u64, u64]),
    "rsaprng_server_result": (i32, [vp, u64, pvp, pu64]),
    "rsaprng_server_copy": (i32, [vp, u64, vp, vp]),
    "rsaprng_server_release": (i32, [vp, u64]),
    "rsaprng_server_cancel": (i32, [vp, u64]),
    "rsaprng_server_stats": (i32, [vp, ctypes.POINTER(Stats)]),
    "rsaprng_server_replay": (i32, [vp, u64, pu32, pu64, pu64, u64, pdbl]),
    "rsaprng_server_replay_keep": (i32, [vp, u64, pu32, pu64, pu64, u64, pu64]),
    "rsaprng_server_destroy": (None, [vp]),
    "rsaprng_is_prime": (i32, [u64]),
    "rsaprng_root_allowed": (i32, [u64]),
    "rsaprng_validate_params": (i32, [u64, u64, u64, i32]),
    "rsaprng_params_from_seed": (i32, [u64, i32, u64, u64, pu64, pu64, pu64, pu64]),
    "rsaprng_launch_count": (u64, [vp]),
    "rsaprng_transfer_bytes": (i32, [vp, pu64, pu64]),
    "rsaprng_microbench": (i32, [vp, i32, u64, pdbl]),
    "rsaprng_unit_f64": (i32, [vp, u32, u64, vp, vp, i32, vp]),
    "rsaprng_strerror": (ctypes.c_char_p, [i32]),
    "rsaprng_last_error_detail": (ctypes.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads librsaprng (building it with nvcc if needed). Raises if unavailable."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not _build.up_to_date():
                if not build_if_missing:
                    raise RuntimeError(f"librsaprng is not built ({path})")
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"librsaprng missing at {path}")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class RsaPrngError(RuntimeError):
    def __init__(self, code: int, where: str):
        L = load()
        detail = L.rsaprng_last_error_detail().decode(errors="replace")
        name = ERRORS.get(code, str(code))
        super().__init__(f"{where}: {name} ({L.rsaprng_strerror(code).decode()}): {detail}")
        self.code = code
        self.name = name


def check(code: int, where: str):
    if code != OK:
        raise RsaPrngError(code, where)
    return code
