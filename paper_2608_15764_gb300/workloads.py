"""Seeded synthetic inputs (host side) for the streaming-load path.

The input generator only: no checksum or summation arithmetic lives here, so
both the CUDA path and the CPU oracle can be fed the same bytes from it.

* ``splitmix_u32(seed, nwords)`` -- the uint32 buffer: word 2m / 2m+1 are the
  low / high halves of splitmix64 output m (counter form, seed 1 for the
  streaming workloads).
* ``payload(dtype, seed, n)`` -- N(0,1) float payloads by Box-Muller (single
  precision, one pair of normals per two splitmix64 outputs):
  float32 (seed 2), bfloat16 = RNE of the float32 (seed 3), FP8 E4M3 = RNE,
  saturating, of 8 x the float32 (seed 4).
* ``batch_sizes(...)`` -- the 1,024 log-uniform buffer sizes (seed 5) scaled so
  they add up to a fixed total.
* Adversarial float payloads, built from bit patterns: ``bf16_cancel`` (large
  values that cancel inside each vector next to small ones),
  ``bf16_wide`` (magnitudes spread over ~36 binades with cancelling pairs),
  ``bf16_code_groups`` (every finite bfloat16 code, grouped so that no sum
  can overflow FP32) and ``fp8_finite_codes`` (every finite E4M3 code).

The heavy lifting is in ``csrc/workloads.c``; large requests are split into
chunks generated on host threads (the generator is counter-based, so a chunk
depends only on its first index).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "workloads.c")
_LIB = os.path.join(_HERE, "libslworkloads.so")
_lock = threading.Lock()
_lib = None

U32, F32, BF16, FP8_E4M3 = 0, 1, 2, 3
ELEM_BYTES = {U32: 4, F32: 4, BF16: 2, FP8_E4M3: 1}
NP_DTYPE = {U32: np.uint32, F32: np.float32, BF16: np.uint16, FP8_E4M3: np.uint8}
DEFAULT_SEED = {U32: 1, F32: 2, BF16: 3, FP8_E4M3: 4}
FP8_SCALE = 8.0
SIZES_SEED = 5
_CHUNK = 1 << 22  # elements per generator call (even: chunks start on pair boundaries)


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u64 = ctypes.c_uint64
            lib.wl_splitmix64_at.restype = u64
            lib.wl_splitmix64_at.argtypes = [u64, u64]
            lib.wl_splitmix_u64.restype = None
            lib.wl_splitmix_u64.argtypes = [u64, u64, u64, ctypes.c_void_p]
            lib.wl_splitmix_u32.restype = None
            lib.wl_splitmix_u32.argtypes = [u64, u64, u64, ctypes.c_void_p]
            lib.wl_normal_f32.restype = None
            lib.wl_normal_f32.argtypes = [u64, u64, u64, ctypes.c_void_p]
            lib.wl_f32_to_bf16.restype = None
            lib.wl_f32_to_bf16.argtypes = [ctypes.c_void_p, u64, ctypes.c_void_p]
            lib.wl_f32_to_fp8_e4m3.restype = None
            lib.wl_f32_to_fp8_e4m3.argtypes = [ctypes.c_void_p, u64, ctypes.c_float, ctypes.c_void_p]
            lib.wl_chase_chain.restype = ctypes.c_int32
            lib.wl_chase_chain.argtypes = [u64, u64, u64, ctypes.c_void_p, ctypes.c_void_p]
            lib.wl_payload.restype = ctypes.c_int32
            lib.wl_payload.argtypes = [ctypes.c_int32, u64, u64, u64, ctypes.c_float, ctypes.c_void_p]
            _lib = lib
    return _lib


def _threads() -> int:
    return max(1, os.cpu_count() or 1)


def _chunked(n: int, fn, threads: int | None = None):
    """Run fn(first, count) over [0, n) in chunks on a thread pool (ctypes
    releases the GIL during each call)."""
    starts = list(range(0, n, _CHUNK))
    if len(starts) <= 1:
        if n:
            fn(0, n)
        return
    with ThreadPoolExecutor(max_workers=threads or _threads()) as ex:
        list(ex.map(lambda s: fn(s, min(_CHUNK, n - s)), starts))


def splitmix64(seed: int, first: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    _load().wl_splitmix_u64(seed, first, n, out.ctypes.data)
    return out


def splitmix_u32(seed: int, nwords: int, first_word: int = 0, out: np.ndarray | None = None) -> np.ndarray:
    """uint32 words [first_word, first_word + nwords) of the splitmix64 buffer."""
    if out is None:
        out = np.empty(nwords, dtype=np.uint32)
    assert out.dtype == np.uint32 and out.size == nwords and out.flags.c_contiguous
    lib = _load()
    base = out.ctypes.data
    _chunked(nwords, lambda s, c: lib.wl_splitmix_u32(seed, first_word + s, c, base + 4 * s))
    return out


def payload(dtype: int, n: int, seed: int | None = None, first: int = 0,
            out: np.ndarray | None = None) -> np.ndarray:
    """n elements of a N(0,1) payload in the given float dtype (numpy dtype
    float32 / uint16 for bfloat16 bits / uint8 for FP8 E4M3 bits)."""
    if dtype not in (F32, BF16, FP8_E4M3):
        raise ValueError(f"not a float payload dtype: {dtype}")
    seed = DEFAULT_SEED[dtype] if seed is None else seed
    if out is None:
        out = np.empty(n, dtype=NP_DTYPE[dtype])
    assert out.size == n and out.flags.c_contiguous
    lib = _load()
    eb = ELEM_BYTES[dtype]
    base = out.ctypes.data
    scale = FP8_SCALE if dtype == FP8_E4M3 else 1.0

    def gen(s, c):
        rc = lib.wl_payload(dtype, seed, first + s, c, scale, base + eb * s)
        if rc != 0:
            raise RuntimeError("wl_payload failed")

    _chunked(n, gen)
    return out


def normal_f32(seed: int, n: int, first: int = 0) -> np.ndarray:
    out = np.empty(n, dtype=np.float32)
    _load().wl_normal_f32(seed, first, n, out.ctypes.data)
    return out


def f32_to_bf16(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.size, dtype=np.uint16)
    _load().wl_f32_to_bf16(x.ctypes.data, x.size, out.ctypes.data)
    return out


def f32_to_fp8_e4m3(x: np.ndarray, scale: float = 1.0) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.size, dtype=np.uint8)
    _load().wl_f32_to_fp8_e4m3(x.ctypes.data, x.size, scale, out.ctypes.data)
    return out


def batch_sizes(n: int = 1024, total: int = 16 << 30, lo: int = 64 << 10, hi: int = 256 << 20,
                seed: int = SIZES_SEED, align: int = 4096) -> list[int]:
    """Sizes of the batched workload: n log-uniform draws on [lo, hi], scaled by
    a common factor c (found by bisection) so that sum(clamp(c*s_i, lo, hi)) =
    total, floored to ``align`` bytes; the remainder goes, ``align`` bytes at a
    time, to the largest buffers that still have room below ``hi``.

    A plain log-uniform draw of 1,024 sizes on [64 KiB, 256 MiB] averages about
    32 MB per buffer (about 33 GB in all), so a fixed 16 GiB total needs this
    rescaling."""
    if n * lo > total or n * hi < total:
        raise ValueError("total not reachable with these bounds")
    raw = splitmix64(seed, 0, n)
    la, lb = math.log(lo), math.log(hi)
    s = [math.exp(la + ((int(v) >> 11) + 0.5) / float(1 << 53) * (lb - la)) for v in raw]

    def tot(c):
        return sum(min(max(c * x, lo), hi) for x in s)

    c_lo, c_hi = 1e-6, 1e6
    for _ in range(200):
        mid = math.sqrt(c_lo * c_hi)
        if tot(mid) < total:
            c_lo = mid
        else:
            c_hi = mid
    sizes = [int(min(max(c_lo * x, lo), hi)) // align * align for x in s]
    sizes = [max(lo, min(hi, v)) for v in sizes]
    rem = total - sum(sizes)
    order = sorted(range(n), key=lambda i: (-sizes[i], i))
    while rem > 0:
        progressed = False
        for i in order:
            room = hi - sizes[i]
            if room <= 0:
                continue
            add = min(room, rem)
            sizes[i] += add
            rem -= add
            progressed = True
            if rem == 0:
                break
        if not progressed:
            raise ValueError("cannot place the remainder")
    while rem < 0:  # only if flooring overshot (cannot happen with floor), kept for safety
        i = order[0]
        take = min(-rem, sizes[i] - lo)
        sizes[i] -= take
        rem += take
    assert sum(sizes) == total and all(lo <= v <= hi and v % 16 == 0 for v in sizes)
    return sizes


def chase_chain(n: int, stride_bytes: int = 64, seed: int = 6) -> np.ndarray:
    """Pointer-chase chain of n elements, one every stride_bytes (a multiple
    of 4): word i*stride/4 holds the word index of the next element, and the
    successor map is one random cycle through all n elements (Sattolo)."""
    sw = stride_bytes // 4
    out = np.empty(n * sw, dtype=np.uint32)
    perm = np.empty(n, dtype=np.uint32)
    if _load().wl_chase_chain(seed, n, sw, out.ctypes.data, perm.ctypes.data) != 0:
        raise ValueError("chain too large for 32-bit word indices")
    return out


# ---- adversarial float payloads (bit patterns only) -------------------------------

def bf16_code(e: int, m: int = 0, neg: bool = False) -> int:
    """bfloat16 code of (-1)^neg * (1 + m/128) * 2^e, for a normal exponent e
    (-126..127) and mantissa m (0..127)."""
    assert -126 <= e <= 127 and 0 <= m < 128
    return (0x8000 if neg else 0) | ((e + 127) << 7) | m


# Eight bfloat16 values whose plain left-to-right FP32 sum loses the small
# one: 2^20 + 2^-5 rounds to 2^20 in FP32, so 2^-5 disappears in some orders.
CANCEL_CODES = (bf16_code(-5), bf16_code(20, neg=True), bf16_code(0), bf16_code(20), 0, 0, 0, 0)


def bf16_cancel(nvec: int, seed: int = 7, nperm: int = 64) -> np.ndarray:
    """nvec 16-byte vectors of bfloat16 (8 codes each): vector i holds the
    codes of CANCEL_CODES in permutation i mod nperm (seeded), so the large
    pair, the small value and the zeros occupy every position.  Exact sum:
    nvec * (1 + 2^-5)."""
    rng = np.random.default_rng(seed)
    base = np.array(CANCEL_CODES, dtype=np.uint16)
    perms = np.stack([base[rng.permutation(8)] for _ in range(nperm)])
    reps = -(-nvec // nperm)
    return np.ascontiguousarray(np.tile(perms, (reps, 1))[:nvec].reshape(-1))


def bf16_wide(nvec: int, seed: int = 8) -> np.ndarray:
    """nvec 16-byte vectors of bfloat16 spanning ~36 binades: in every vector
    two random positions hold +L and -L (L = (1 + m/128) 2^e, e in 8..24) and
    the six others small positive values (e in -12..4), so the exact sum is
    the sum of the small values while every running FP32 sum is dominated by
    the large ones."""
    rng = np.random.default_rng(seed)
    e = rng.integers(-12, 5, size=(nvec, 8))
    m = rng.integers(0, 128, size=(nvec, 8))
    codes = ((e + 127) << 7) | m
    order = np.argsort(rng.random((nvec, 8)), axis=1)
    el = rng.integers(8, 25, size=nvec)
    ml = rng.integers(0, 128, size=nvec)
    big = ((el + 127) << 7) | ml
    rows = np.arange(nvec)
    codes[rows, order[:, 0]] = big
    codes[rows, order[:, 1]] = big | 0x8000
    return np.ascontiguousarray(codes.astype(np.uint16).reshape(-1))


def bf16_as_f32_bits(codes: np.ndarray) -> np.ndarray:
    """The float32 payload holding exactly the values of the given bfloat16
    codes (a bfloat16 is the top half of the float32 with its value)."""
    return (np.asarray(codes, dtype=np.uint32) << 16).view(np.float32)


def bf16_code_groups(limit_log2: int = 127) -> list[np.ndarray]:
    """Every finite bfloat16 code (both zeros, subnormals and all normal
    binades, both signs) exactly once, split into groups of one sign and one
    binade; a binade is split further, in mantissa order, where its values
    would add up to more than 2^limit_log2.  Within a group every value is an
    integer multiple of the binade's unit 2^(E-134) (2^-133 for subnormals)
    and the multiples add up to less than 2^15, so every partial sum of a
    group, in any order, is exactly representable in FP32 and below the
    FP32 maximum.  Grouping uses integer arithmetic on the code fields only.
    The two zeros join the subnormal groups."""
    groups = []
    for neg in (0, 1):
        sign = 0x8000 if neg else 0
        groups.append(np.array([sign | m for m in range(0, 128)], dtype=np.uint16))  # zero + subnormals
        for big_e in range(1, 255):
            # value of mantissa m: (128 + m) * 2^(big_e - 134)
            cur, acc = [], 0
            for m in range(128):
                mult = 128 + m
                if cur and big_e - 134 + math.log2(acc + mult) > limit_log2:
                    groups.append(np.array(cur, dtype=np.uint16))
                    cur, acc = [], 0
                cur.append(sign | (big_e << 7) | m)
                acc += mult
            groups.append(np.array(cur, dtype=np.uint16))
    return groups


def fp8_finite_codes() -> np.ndarray:
    """Every finite FP8 E4M3 code (all 256 but the two NaNs 0x7F and 0xFF):
    both zeros, the subnormals and +-448."""
    return np.array([c for c in range(256) if (c & 0x7F) != 0x7F], dtype=np.uint8)
