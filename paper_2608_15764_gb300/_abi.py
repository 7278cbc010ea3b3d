"""ctypes mirror of include/streamload.h (structures, enums, prototypes).

Argument marshalling only: every step of the streaming-load path runs in the
CUDA library; nothing here computes a checksum or a sum.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstreamload.so")

# status codes
SL_OK = 0
SL_ERR_ARG = -1
SL_ERR_ALIGN = -2
SL_ERR_INFEASIBLE = -3
SL_ERR_TIMEOUT = -4
SL_ERR_CUDA = -5
SL_ERR_OOM = -6
SL_ERR_NODEV = -7
STATUS_NAMES = {0: "SL_OK", -1: "SL_ERR_ARG", -2: "SL_ERR_ALIGN", -3: "SL_ERR_INFEASIBLE",
                -4: "SL_ERR_TIMEOUT", -5: "SL_ERR_CUDA", -6: "SL_ERR_OOM", -7: "SL_ERR_NODEV"}

# enums
SL_U32, SL_F32, SL_BF16, SL_FP8_E4M3 = 0, 1, 2, 3
SL_LDG, SL_CPASYNC, SL_TMA, SL_LDSTS, SL_LDG4, SL_LDG32 = 0, 1, 2, 3, 4, 5
SL_ASC, SL_DESC, SL_DYN = 0, 1, 2
SL_COP_CG, SL_COP_CG_L2_256, SL_COP_NC_NA_L2_256 = 0, 1, 2
SL_MAX_K, SL_MAX_D, SL_MIN_STAGES, SL_MAX_STAGES = 16, 16, 2, 8
SL_RING_CTA, SL_RING_WARP = 0, 1
SL_DEBUG_TMA_SKIP_STAGE = 1
SL_DEBUG_SMEM_SKEW_SHIFT = 8


def SL_DEBUG_SMEM_SKEW(n: int) -> int:
    return (int(n) & 7) << SL_DEBUG_SMEM_SKEW_SHIFT


class sl_config(ctypes.Structure):
    _fields_ = [
        ("mech", ctypes.c_int32),
        ("k", ctypes.c_int32),
        ("stage_bytes", ctypes.c_int32),
        ("stages", ctypes.c_int32),
        ("cta", ctypes.c_int32),
        ("grid", ctypes.c_int32),
        ("order", ctypes.c_int32),
        ("flush_l2", ctypes.c_int32),
        ("passes", ctypes.c_int32),
        ("cop", ctypes.c_int32),
        ("debug_flags", ctypes.c_int32),
        ("host_direct", ctypes.c_int32),
        ("tma_ring", ctypes.c_int32),
        ("copies", ctypes.c_int32),
        ("target_loads", ctypes.c_uint64),
        ("stream", ctypes.c_void_p),
    ]


class sl_result(ctypes.Structure):
    _fields_ = [
        ("xor_u64", ctypes.c_uint64),
        ("issued_loads", ctypes.c_uint64),
        ("device_ns", ctypes.c_uint64),
        ("window_ns", ctypes.c_uint64),
        ("fsum", ctypes.c_double),
        ("fsum_hi", ctypes.c_float),
        ("fsum_lo", ctypes.c_float),
        ("sum_u32", ctypes.c_uint32),
        ("status", ctypes.c_int32),
        ("grid", ctypes.c_int32),
        ("cta", ctypes.c_int32),
        ("resident_per_sm", ctypes.c_int32),
        ("smem_bytes", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class sl_devinfo(ctypes.Structure):
    _fields_ = [
        ("device", ctypes.c_int32),
        ("sm_count", ctypes.c_int32),
        ("cc_major", ctypes.c_int32),
        ("cc_minor", ctypes.c_int32),
        ("l2_bytes", ctypes.c_int64),
        ("smem_per_block_optin", ctypes.c_int64),
        ("smem_per_sm", ctypes.c_int64),
        ("global_mem_bytes", ctypes.c_int64),
        ("max_threads_per_sm", ctypes.c_int32),
        ("regs_per_sm", ctypes.c_int32),
        ("clock_khz", ctypes.c_int32),
        ("mem_clock_khz", ctypes.c_int32),
        ("mem_bus_bits", ctypes.c_int32),
        ("driver_version", ctypes.c_int32),
        ("runtime_version", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("name", ctypes.c_char * 256),
    ]

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}
        d["name"] = self.name.decode(errors="replace")
        return d


class sl_chase_result(ctypes.Structure):
    _fields_ = [("final_index", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("hops", ctypes.c_uint64),
                ("ns", ctypes.c_uint64), ("cycles", ctypes.c_uint64), ("ns_per_hop", ctypes.c_double),
                ("cycles_per_hop", ctypes.c_double)]


class sl_twostream_result(ctypes.Structure):
    _fields_ = [("xor_u64", ctypes.c_uint64 * 2), ("issued_loads", ctypes.c_uint64 * 2),
                ("window_ns", ctypes.c_uint64 * 2), ("b_first_end_ns", ctypes.c_uint64),
                ("device_ns", ctypes.c_uint64), ("sum_u32", ctypes.c_uint32 * 2), ("grid", ctypes.c_int32),
                ("cta", ctypes.c_int32), ("b_covers_a", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class sl_batch_desc(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("bytes", ctypes.c_uint64), ("dtype", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class sl_tune_entry(ctypes.Structure):
    _fields_ = [("min_bytes", ctypes.c_uint64), ("max_bytes", ctypes.c_uint64), ("dtype", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("cfg", sl_config)]


assert ctypes.sizeof(sl_batch_desc) == 24
assert ctypes.sizeof(sl_tune_entry) == 96
assert ctypes.sizeof(sl_config) == 72
assert ctypes.sizeof(sl_result) == 72
RESULT_BYTES = ctypes.sizeof(sl_result)

_P = ctypes.c_void_p
_U64 = ctypes.c_uint64
_I32 = ctypes.c_int32
PROTOTYPES = {
    "sl_device_info": (_I32, [ctypes.POINTER(sl_devinfo)]),
    "sl_last_error": (ctypes.c_char_p, []),
    "sl_fill_splitmix64": (_I32, [_P, _U64, _U64, _P]),
    "sl_flush_l2": (_I32, [_P]),
    "sl_plan": (_I32, [_U64, _I32, ctypes.POINTER(sl_config), ctypes.POINTER(sl_result)]),
    "sl_run": (_I32, [_P, _U64, _I32, ctypes.POINTER(sl_config), ctypes.POINTER(sl_result)]),
    "sl_enqueue": (_I32, [_P, _U64, _I32, ctypes.POINTER(sl_config), _P]),
    "sl_sweep": (_I32, [_P, _U64, _I32, ctypes.POINTER(sl_config), _I32, _I32, _I32, _I32,
                        ctypes.POINTER(sl_result)]),
    "sl_run_host": (_I32, [_P, _U64, _I32, ctypes.POINTER(sl_config), ctypes.POINTER(sl_result)]),
    "sl_run_noalloc": (_I32, [_P, _U64, _I32, ctypes.POINTER(sl_config), _P]),
    "sl_chase": (_I32, [_P, _U64, ctypes.c_uint32, _U64, _U64, _I32, _P, ctypes.POINTER(sl_chase_result)]),
    "sl_coverage": (_I32, [_P, _U64, ctypes.POINTER(sl_config), _P, ctypes.POINTER(sl_result)]),
    "sl_enqueue_steps": (_I32, [ctypes.POINTER(ctypes.c_void_p), _I32, _U64, _I32, ctypes.POINTER(sl_config), _I32,
                                _P]),
    "sl_twostream": (_I32, [_P, _U64, _P, _U64, _I32, _I32, _I32, _I32, _I32, _P,
                            ctypes.POINTER(sl_twostream_result)]),
    "sl_batch_create": (_I32, [ctypes.POINTER(sl_batch_desc), _I32, ctypes.POINTER(sl_tune_entry), _I32,
                               ctypes.POINTER(ctypes.c_void_p)]),
    "sl_batch_run": (_I32, [_P, ctypes.POINTER(sl_result), ctypes.POINTER(ctypes.c_uint64)]),
    "sl_batch_info": (_I32, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "sl_batch_destroy": (None, [_P]),
}
SL_NOALLOC_MAX_CTAS = 4096

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libstreamload.so.  Fails loudly if it has not been built: there is
    no fallback implementation."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(
                    f"{path} is missing: build it with `python -m paper_2608_15764_gb300.build` "
                    "(the streaming-load path has no CPU fallback)")
            lib = ctypes.CDLL(path)
            for name, (res, args) in PROTOTYPES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib
