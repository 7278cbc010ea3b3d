"""Pins for the CPU oracle (``oracle/``) against things other than itself:
pure-Python brute force, closed forms, invariants, ``math.fsum``, torch CPU
casts and the paper's printed fixed-work figures.  CPU only."""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
from oracle import brute

RNG = np.random.default_rng(12345)


def _rand_bytes(nbytes):
    return RNG.integers(0, 256, size=nbytes, dtype=np.uint8)


# ---- integer checksum: brute force -----------------------------------------

@pytest.mark.parametrize("nwords", [0, 2, 4, 6, 8, 34, 4096])
def test_checksum_matches_brute_force(nwords):
    b = _rand_bytes(4 * nwords)
    assert oracle.checksum(b) == brute.checksum(b.tobytes())


@pytest.mark.parametrize("passes", [1, 2, 3, 4, 7])
def test_checksum_passes_matches_brute_force(passes):
    b = _rand_bytes(4 * 130)
    assert oracle.checksum(b, passes) == brute.checksum(b.tobytes(), passes)


def test_checksum_sensitive_to_every_word():
    # Changing any single word must change the sum (a dropped or doubled load
    # changes it); the xor changes too.
    b = _rand_bytes(4 * 64).view(np.uint32).copy()
    s0, x0 = oracle.checksum(b)
    for i in range(b.size):
        c = b.copy()
        c[i] ^= np.uint32(1 << (i % 32))
        s, x = oracle.checksum(c)
        assert s != s0 and x != x0


def test_word_pairing_is_little_endian_uint64():
    # q[j] = w[2j] | w[2j+1] << 32: a buffer whose only nonzero word is w[1]
    # must put it in the high half.
    w = np.zeros(4, dtype=np.uint32)
    w[1] = 0xDEADBEEF
    assert oracle.checksum(w) == (0xDEADBEEF, 0xDEADBEEF << 32)
    w = np.zeros(4, dtype=np.uint32)
    w[2] = 0x12345678
    assert oracle.checksum(w) == (0x12345678, 0x12345678)


# ---- integer checksum: closed forms ------------------------------------------

def _prefix_xor(m):
    """0 ^ 1 ^ ... ^ m (closed form by m mod 4)."""
    if m < 0:
        return 0
    return [m, 1, m + 1, 0][m % 4]


@pytest.mark.parametrize("nwords", [4, 1 << 10, (1 << 20) + 4, 1 << 24])
def test_closed_forms(nwords):
    z = np.zeros(nwords, dtype=np.uint32)
    assert oracle.checksum(z) == (0, 0)

    ones = np.full(nwords, 0xFFFFFFFF, dtype=np.uint32)
    s, x = oracle.checksum(ones)
    assert s == (-nwords) % (1 << 32)
    assert x == (0xFFFFFFFFFFFFFFFF if (nwords // 2) % 2 else 0)

    ramp = np.arange(nwords, dtype=np.uint64).astype(np.uint32)
    s, x = oracle.checksum(ramp)
    assert s == (nwords * (nwords - 1) // 2) % (1 << 32)
    half = nwords // 2
    lo = 2 * _prefix_xor(half - 1)            # XOR of 2j, j < half
    hi = lo ^ (1 if half % 2 else 0)          # XOR of 2j+1, j < half
    assert x == (lo | (hi << 32))


@pytest.mark.parametrize("passes", [1, 2, 3, 6, 9])
def test_passes_closed_form(passes):
    b = _rand_bytes(4 * 1000)
    s1, x1 = oracle.checksum(b)
    assert oracle.checksum(b, passes) == ((passes * s1) % (1 << 32), x1 if passes % 2 else 0)


def test_split_and_permutation_invariance():
    w = _rand_bytes(4 * 10000).view(np.uint32)
    full = oracle.checksum(w)
    # any split into even-length pieces combines exactly
    cuts = [0, 2, 1000, 1002, 5000, 10000]
    parts = [oracle.checksum(w[a:b]) for a, b in zip(cuts[:-1], cuts[1:])]
    assert oracle.combine(parts) == full
    # permuting the 64-bit words (any tile order, any mechanism) changes nothing
    q = w.view(np.uint64).copy()
    RNG.shuffle(q)
    assert oracle.checksum(q.view(np.uint32)) == full


# ---- issued loads and the paper's fixed-work arithmetic ----------------------

def test_issued_loads_closed_form():
    for nbytes in [0, 16, 4096, 256 << 20, 4 << 30, 20 << 30]:
        for p in [1, 2, 5]:
            assert oracle.issued_loads(nbytes, p) == p * nbytes // 16


def test_paper_fixed_work_mismatch(golden_dir):
    """§4.2 prints a maximum issued-load mismatch of 0.024576% over K=1,2,4,8
    at the primary cell (132 CTAs x 32 warps) for an issued volume of
    16,785 MiB of 16-byte loads (§3).  Rebuild it from those printed inputs."""
    g = json.load(open(os.path.join(golden_dir, "paper_fixed_work.json")))
    threads = g["ctas"] * g["warps_per_cta"] * 32
    target = g["issued_volume_mib"] * (1 << 20) // g["bytes_per_load"]
    issued, mm = oracle.fixed_iteration(target, threads, g["ks"])
    assert round(100 * mm, 6) == pytest.approx(g["max_mismatch_pct"], abs=5e-7)
    # total DRAM-side volume of the K=1 cell is the printed ~17.6 GB
    assert round(issued[0] * g["bytes_per_load"] / 1e9, 1) == g["issued_volume_gb"]
    # K=2 divides exactly; K=4 and K=8 lose the same two loads per thread
    assert issued[1] == issued[0]
    assert issued[2] == issued[3] == issued[0] - 2 * threads


@pytest.mark.parametrize("nvec,nloads", [(0, 5), (1, 0), (1, 7), (3, 10), (5, 5), (8, 37), (33, 200), (64, 64)])
def test_wrapped_checksum_brute_force(nvec, nloads):
    b = _rand_bytes(16 * nvec)
    assert oracle.wrapped_checksum(b, nloads) == brute.wrapped_checksum(b.tobytes(), nloads)


def test_wrapped_checksum_closed_forms():
    """q whole wraps are q passes; a partial wrap adds the prefix of r vectors;
    below one wrap it is the checksum of the prefix."""
    b = _rand_bytes(16 * 1000)
    w = b.view(np.uint32)
    for q, r in [(0, 1), (0, 999), (1, 0), (2, 0), (3, 17), (66, 123)]:
        got = oracle.wrapped_checksum(b, q * 1000 + r)
        want = oracle.combine([oracle.checksum(w, q) if q else (0, 0), oracle.checksum(w[:4 * r])])
        assert got == want, (q, r)
    assert oracle.wrapped_checksum(b, 0) == (0, 0)


def test_fixed_iteration_exact_when_divisible():
    issued, mm = oracle.fixed_iteration(1024 * 256 * 16, 1024 * 256, [1, 2, 4, 8, 16])
    assert mm == 0.0 and len(set(issued)) == 1


# ---- float payloads: decoders -------------------------------------------------

def test_fp8_decoder_all_codes_vs_torch():
    codes = np.arange(256, dtype=np.uint8)
    ours = oracle.decode(oracle.FP8_E4M3, codes)
    ref = torch.from_numpy(codes.copy()).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    nan = np.isnan(ref)
    assert nan.sum() == 2 and np.array_equal(np.isnan(ours), nan)
    assert np.array_equal(ours[~nan], ref[~nan])
    assert ours[0x7E] == 448.0 and ours[0x01] == 2.0 ** -9 and ours[0x08] == 2.0 ** -6
    assert brute.decode(3, codes.tobytes())[0x3F] == ours[0x3F]


def test_bf16_decoder_all_codes_vs_torch():
    codes = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    ours = oracle.decode(oracle.BF16, codes)
    ref = torch.from_numpy(codes.view(np.int16).copy()).view(torch.bfloat16).to(torch.float64).numpy()
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(ours), nan)
    assert np.array_equal(ours[~nan], ref[~nan])


def test_f32_decoder_vs_numpy():
    bits = RNG.integers(0, 1 << 32, size=100000, dtype=np.uint64).astype(np.uint32)
    ours = oracle.decode(oracle.F32, bits)
    with np.errstate(invalid="ignore"):
        ref = bits.view(np.float32).astype(np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(ours[~nan], ref[~nan])


# ---- float payloads: sums -------------------------------------------------------

@pytest.mark.parametrize("dtype", [oracle.F32, oracle.BF16, oracle.FP8_E4M3])
def test_fsum_vs_math_fsum(dtype):
    n = 200000
    x = RNG.standard_normal(n).astype(np.float32)
    if dtype == oracle.F32:
        p = x
    elif dtype == oracle.BF16:
        p = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy()
    else:
        p = torch.from_numpy(8 * x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    vals = oracle.decode(dtype, p)
    s, a = oracle.fsum(dtype, p)
    ref = math.fsum(vals.tolist())
    assert abs(s - ref) <= 1e-15 * math.fsum(np.abs(vals).tolist())
    assert a == pytest.approx(math.fsum(np.abs(vals).tolist()), rel=1e-12)


def test_fsum_brute_force_tiny():
    for dtype, n in [(oracle.F32, 37), (oracle.BF16, 74), (oracle.FP8_E4M3, 148)]:
        b = _rand_bytes(n * oracle.ELEM_BYTES[dtype])
        if dtype == oracle.F32:  # keep the float32 bit patterns finite
            b = (b.view(np.uint32) & np.uint32(0xBFFFFFFF)).view(np.uint8)
        if dtype == oracle.FP8_E4M3:
            b = np.where((b & 0x7F) == 0x7F, b ^ 1, b).astype(np.uint8)
        if dtype == oracle.BF16:
            b = (b.view(np.uint16) & np.uint16(0xBFFF)).view(np.uint8)
        s, a = oracle.fsum(dtype, b)
        bs, ba = brute.fsum(dtype, b.tobytes())
        assert abs(s - bs) <= 1e-15 * ba
        assert a == pytest.approx(ba, rel=1e-14)


def test_fsum_cancellation_is_compensated():
    # 1e8 + (1 repeated) - 1e8 in float32 values: a naive FP64 running sum is
    # exact here too, so make the cancellation exceed FP64: 2^60, 1, -2^60.
    x = np.array([2.0 ** 60, 1.0, -(2.0 ** 60), 1.0], dtype=np.float32)
    s, a = oracle.fsum(oracle.F32, x)
    assert s == 2.0
    # closed form: alternating +v, -v sums to exactly zero
    v = RNG.standard_normal(5000).astype(np.float32)
    alt = np.empty(10000, dtype=np.float32)
    alt[0::2] = v
    alt[1::2] = -v
    assert oracle.fsum(oracle.F32, alt)[0] == 0.0
    # constant payload: n * c exactly
    c = np.full(1 << 16, 0.375, dtype=np.float32)
    assert oracle.fsum(oracle.F32, c)[0] == 0.375 * (1 << 16)


def test_bad_dtype_rejected():
    with pytest.raises(ValueError):
        oracle.fsum(7, np.zeros(16, np.uint8))


# ---- pointer chase ----------------------------------------------------------

def test_chase_brute_force_and_closed_form():
    rng = np.random.default_rng(5)
    n, sw = 257, 3
    succ = rng.permutation(n)
    chain = np.zeros(n * sw, dtype=np.uint32)
    chain[np.arange(n) * sw] = succ * sw
    for steps in (0, 1, 2, 100, 1000):
        idx = 0
        for _ in range(steps):
            idx = int(chain[idx])
        assert oracle.chase(chain, 0, steps) == idx
    # successor i -> i+1 (mod n): after s steps from element a, element (a+s) mod n
    ring = np.zeros(n * sw, dtype=np.uint32)
    ring[np.arange(n) * sw] = ((np.arange(n) + 1) % n) * sw
    for a, s in [(0, 5), (17, 300), (256, 1)]:
        assert oracle.chase(ring, a * sw, s) == ((a + s) % n) * sw
    # an index outside the buffer is reported, not followed
    bad = np.array([5, 0], dtype=np.uint32)
    assert oracle.chase(bad, 0, 2) == 0xFFFFFFFF
