"""Pure-Python brute-force statement of the oracle's definitions.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Meant for tiny inputs
(a few thousand words): Python integers, ``struct`` and ``math.fsum``.  It
is written independently of ``oracle.c`` so that each pins the other.
"""
from __future__ import annotations

import math
import struct


def checksum(data: bytes, passes: int = 1) -> tuple[int, int]:
    """(sum of uint32 words mod 2^32, XOR of little-endian uint64 words),
    folded ``passes`` times (paper §3 Instruments)."""
    if len(data) % 8:
        raise ValueError("length must be a multiple of 8")
    words = struct.unpack(f"<{len(data) // 4}I", data)
    qwords = struct.unpack(f"<{len(data) // 8}Q", data)
    s = 0
    x = 0
    for _ in range(passes):
        for w in words:
            s = (s + w) % (1 << 32)
        for q in qwords:
            x ^= q
    return s, x


def wrapped_checksum(data: bytes, nloads: int) -> tuple[int, int]:
    """Checksum of nloads 16-byte loads where load j reads vector j mod
    (number of 16-byte vectors): the sink of every loaded vector, in order."""
    if len(data) % 16:
        raise ValueError("length must be a multiple of 16")
    vecs = [data[16 * i:16 * i + 16] for i in range(len(data) // 16)]
    s = 0
    x = 0
    for j in range(nloads if vecs else 0):
        a, b, c, d = struct.unpack("<4I", vecs[j % len(vecs)])
        s = (s + a + b + c + d) % (1 << 32)
        x ^= (a | (b << 32)) ^ (c | (d << 32))
    return s, x


def _fp8_e4m3(b: int) -> float:
    sign = -1.0 if b & 0x80 else 1.0
    e = (b >> 3) & 0xF
    m = b & 0x7
    if e == 0xF and m == 0x7:
        return math.nan
    if e == 0:
        return sign * (m / 8.0) * 2.0 ** -6
    return sign * (1.0 + m / 8.0) * 2.0 ** (e - 7)


def decode(dtype: int, data: bytes) -> list[float]:
    """dtype codes: 1 = float32, 2 = bfloat16, 3 = FP8 E4M3 (fn)."""
    if dtype == 1:
        return list(struct.unpack(f"<{len(data) // 4}f", data))
    if dtype == 2:
        hs = struct.unpack(f"<{len(data) // 2}H", data)
        return [struct.unpack("<f", struct.pack("<I", h << 16))[0] for h in hs]
    if dtype == 3:
        return [_fp8_e4m3(b) for b in data]
    raise ValueError(dtype)


def fsum(dtype: int, data: bytes) -> tuple[float, float]:
    """Correctly rounded sum (math.fsum) and sum of |x|."""
    vals = decode(dtype, data)
    return math.fsum(vals), math.fsum(abs(v) for v in vals)
