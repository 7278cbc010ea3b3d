"""CPU oracle for the streaming global-load checksum path.

TEST INFRASTRUCTURE ONLY.  The product package never imports this module; only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference arm may.  It shares no code with the CUDA path.

``oracle.c`` holds the plain definitions (paper §3 "Instruments", §3
"Fixed-work control", §4.2 "Exact-work accounting"); this module builds it with
gcc and exposes it over numpy arrays.  ``brute.py`` is a second, pure-Python
statement of the same definitions for tiny inputs.

Every function here is pinned by ``tests/test_oracle.py`` against something
other than itself: pure-Python brute force, closed forms, ``math.fsum`` (the
correctly rounded sum), torch CPU casts for the decoders, and the paper's
printed fixed-work mismatch (0.024576%, §4.2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

U32, F32, BF16, FP8_E4M3 = 0, 1, 2, 3
ELEM_BYTES = {U32: 4, F32: 4, BF16: 2, FP8_E4M3: 1}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (plain -O2, no FMA
    contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
             "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.oracle_sum_u32.restype = ctypes.c_uint32
            lib.oracle_sum_u32.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
            lib.oracle_xor_u64.restype = ctypes.c_uint64
            lib.oracle_xor_u64.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
            lib.oracle_checksum.restype = None
            lib.oracle_checksum.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                            u32p, ctypes.POINTER(ctypes.c_uint64)]
            lib.oracle_wrapped_checksum.restype = None
            lib.oracle_wrapped_checksum.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                                    u32p, ctypes.POINTER(ctypes.c_uint64)]
            lib.oracle_issued_loads.restype = ctypes.c_uint64
            lib.oracle_issued_loads.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.oracle_fixed_iteration.restype = ctypes.c_double
            lib.oracle_fixed_iteration.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                                                   ctypes.c_int32, ctypes.c_void_p]
            lib.oracle_elem_bytes.restype = ctypes.c_int32
            lib.oracle_elem_bytes.argtypes = [ctypes.c_int32]
            lib.oracle_decode.restype = ctypes.c_int32
            lib.oracle_decode.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
            lib.oracle_chase.restype = ctypes.c_uint32
            lib.oracle_chase.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64]
            lib.oracle_fsum.restype = ctypes.c_int32
            lib.oracle_fsum.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
            _lib = lib
    return _lib


def _words(buf) -> np.ndarray:
    a = np.ascontiguousarray(buf)
    if a.dtype != np.uint32:
        a = a.view(np.uint8).reshape(-1)
        if a.size % 4:
            raise ValueError("byte length must be a multiple of 4")
        a = a.view(np.uint32)
    return a.reshape(-1)


def checksum(buf, passes: int = 1) -> tuple[int, int]:
    """(sum_u32, xor_u64) of a host buffer read ``passes`` times (§3
    Instruments: every loaded word is folded into the sink)."""
    w = _words(buf)
    if w.size % 2:
        raise ValueError("word count must be even (bytes a multiple of 8)")
    lib = _load()
    s = ctypes.c_uint32()
    x = ctypes.c_uint64()
    lib.oracle_checksum(w.ctypes.data, w.size, passes, ctypes.byref(s), ctypes.byref(x))
    return int(s.value), int(x.value)


def wrapped_checksum(buf, nloads: int) -> tuple[int, int]:
    """(sum_u32, xor_u64) of ``nloads`` 16-byte loads j = 0, 1, ... reading
    vector j mod (vectors in the buffer): the paper's fixed-iteration reads,
    which wrap around the allocation (§3 Fixed-work control)."""
    w = _words(buf)
    if w.size % 4:
        raise ValueError("buffer must be a whole number of 16-byte vectors")
    s = ctypes.c_uint32()
    x = ctypes.c_uint64()
    _load().oracle_wrapped_checksum(w.ctypes.data, w.size, int(nloads), ctypes.byref(s), ctypes.byref(x))
    return int(s.value), int(x.value)


def combine(parts) -> tuple[int, int]:
    """Exact combination of (sum_u32, xor_u64) checksums of disjoint pieces of
    one buffer: mod-2^32 addition and XOR are associative and commutative."""
    s, x = 0, 0
    for ps, px in parts:
        s = (s + ps) & 0xFFFFFFFF
        x ^= px
    return s, x


def issued_loads(nbytes: int, passes: int = 1) -> int:
    """Issued 16-byte logical loads under the library's fixed-work control."""
    return int(_load().oracle_issued_loads(nbytes, passes))


def fixed_iteration(target_loads: int, threads: int, ks) -> tuple[list[int], float]:
    """The paper's fixed-work arithmetic (§3 Fixed-work control): per K, issued
    = floor(L/(threads*K)) * threads * K; returns (issued per K, max relative
    mismatch against the largest)."""
    karr = np.ascontiguousarray(np.asarray(ks, dtype=np.int32))
    out = np.zeros(karr.size, dtype=np.uint64)
    mm = _load().oracle_fixed_iteration(target_loads, threads, karr.ctypes.data, karr.size, out.ctypes.data)
    return [int(v) for v in out], float(mm)


def decode(dtype: int, payload) -> np.ndarray:
    """Decode a float payload (bytes/array) into float64 values."""
    if dtype not in (F32, BF16, FP8_E4M3):
        raise ValueError(f"bad dtype {dtype}")
    b = np.ascontiguousarray(payload).view(np.uint8).reshape(-1)
    eb = ELEM_BYTES[dtype]
    n = b.size // eb
    out = np.empty(n, dtype=np.float64)
    rc = _load().oracle_decode(dtype, b.ctypes.data, n, out.ctypes.data)
    if rc != 0:
        raise ValueError(f"bad dtype {dtype}")
    return out


def fsum(dtype: int, payload) -> tuple[float, float]:
    """(sum, sum of |x|) of a float payload: FP64 Neumaier in element order."""
    if dtype not in (F32, BF16, FP8_E4M3):
        raise ValueError(f"bad dtype {dtype}")
    b = np.ascontiguousarray(payload).view(np.uint8).reshape(-1)
    eb = ELEM_BYTES[dtype]
    n = b.size // eb
    s = ctypes.c_double()
    a = ctypes.c_double()
    rc = _load().oracle_fsum(dtype, b.ctypes.data, n, ctypes.byref(s), ctypes.byref(a))
    if rc != 0:
        raise ValueError(f"bad dtype {dtype}")
    return float(s.value), float(a.value)


def chase(chain, start: int, steps: int) -> int:
    """Final word index after following the chain `steps` times from `start`
    (paper §4.1 pointer chase); 0xFFFFFFFF if an index leaves the buffer."""
    w = _words(chain)
    return int(_load().oracle_chase(w.ctypes.data, w.size, start, steps))
