"""Checks of the seeded input generator (``paper_2608_15764_gb300.workloads``):
splitmix64 against an independent numpy statement and its sequential form,
the encoders against torch CPU casts, and the batch-size recipe.  CPU only."""
import math

import numpy as np
import pytest
import torch

from paper_2608_15764_gb300 import workloads as wl

M64 = (1 << 64) - 1


def _np_splitmix(seed, first, n):
    """splitmix64 restated with numpy uint64 arithmetic (wraps mod 2^64)."""
    with np.errstate(over="ignore"):
        m = np.arange(first, first + n, dtype=np.uint64)
        z = np.uint64(seed) + (m + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _seq_splitmix(seed, n):
    """The sequential generator: state += gamma, then finalise."""
    out, state = [], seed
    for _ in range(n):
        state = (state + 0x9E3779B97F4A7C15) & M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        out.append(z ^ (z >> 31))
    return out


@pytest.mark.parametrize("seed", [0, 1, 5, 0xFFFFFFFFFFFFFFFF])
def test_splitmix_counter_form(seed):
    ours = wl.splitmix64(seed, 0, 300)
    assert ours.tolist() == _seq_splitmix(seed, 300)
    assert np.array_equal(wl.splitmix64(seed, 1000, 5000), _np_splitmix(seed, 1000, 5000))


def test_u32_layout_and_offsets():
    q = wl.splitmix64(1, 0, 1000)
    w = wl.splitmix_u32(1, 2000)
    assert np.array_equal(w.view(np.uint64), q)  # word 2m = low half of output m
    # any window (odd starts included) equals the slice of the full buffer
    for a in [0, 1, 7, 512, 1999]:
        assert np.array_equal(wl.splitmix_u32(1, 2000 - a, first_word=a), w[a:])
    # chunked (threaded) generation equals one call
    big = wl.splitmix_u32(1, (1 << 24) + 40)
    assert np.array_equal(big[-2000:], wl.splitmix_u32(1, 2000, first_word=(1 << 24) + 40 - 2000))


def test_normal_moments_and_determinism():
    x = wl.payload(wl.F32, 1 << 20)
    assert abs(float(x.mean())) < 5e-3
    assert abs(float(x.var()) - 1.0) < 1e-2
    assert float(np.abs(x).max()) < 7.0
    assert np.array_equal(x[12345:12400], wl.payload(wl.F32, 55, first=12345))


def test_bf16_encoder_vs_torch():
    x = np.concatenate([wl.payload(wl.F32, 1 << 16),
                        np.array([0.0, -0.0, 1.0, 3.0e38, -1e-40, 1.00390625, 1.01171875], np.float32)])
    ours = wl.f32_to_bf16(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)
    assert np.array_equal(wl.payload(wl.BF16, 1 << 16, seed=wl.DEFAULT_SEED[wl.F32]), ours[: 1 << 16])


def test_fp8_encoder_vs_torch():
    x = wl.payload(wl.F32, 1 << 16)
    ours = wl.f32_to_fp8_e4m3(x, 8.0)
    ref = torch.from_numpy(8.0 * x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(ours, ref)
    assert np.array_equal(wl.payload(wl.FP8_E4M3, 1 << 16, seed=wl.DEFAULT_SEED[wl.F32]), ours)
    # every in-range grid point and midpoint between neighbours
    grid = torch.arange(0, 0x7F, dtype=torch.uint8).view(torch.float8_e4m3fn).float().numpy()
    mids = ((grid[:-1].astype(np.float64) + grid[1:]) / 2).astype(np.float32)
    probe = np.concatenate([grid, -grid, mids, -mids, np.array([447.0, 460.0, 1e-4], np.float32)])
    ref = torch.from_numpy(probe).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(wl.f32_to_fp8_e4m3(probe), ref)
    # saturation (torch gives NaN above 464; the encoder clamps to 448 by definition)
    assert wl.f32_to_fp8_e4m3(np.array([500.0, -1e6], np.float32)).tolist() == [0x7E, 0xFE]


def test_batch_sizes_recipe():
    s = wl.batch_sizes()
    assert len(s) == 1024 and sum(s) == 16 << 30
    assert min(s) >= 64 << 10 and max(s) <= 256 << 20
    assert all(v % 4096 == 0 for v in s)
    assert s == wl.batch_sizes()  # deterministic
    # spread over the whole log range: sizes at both bounds and a wide middle
    logs = sorted(math.log2(v) for v in s)
    assert logs[0] == 16.0 and logs[-1] <= 28.0
    assert logs[len(logs) // 2] > 20 and logs[len(logs) // 10] < logs[9 * len(logs) // 10] - 4


@pytest.mark.parametrize("n,stride", [(2, 64), (3, 16), (1000, 64), (4096, 128)])
def test_chase_chain_is_one_cycle(n, stride):
    c = wl.chase_chain(n, stride)
    sw = stride // 4
    assert c.size == n * sw
    mask = np.ones(c.size, bool)
    mask[::sw] = False
    assert not c[mask].any()                     # only element slots are used
    seen, idx = set(), 0
    for _ in range(n):
        assert idx % sw == 0 and idx not in seen
        seen.add(idx)
        idx = int(c[idx])
    assert idx == 0 and len(seen) == n           # a single cycle through every element
    assert np.array_equal(c, wl.chase_chain(n, stride))


# ---- adversarial float payloads ----------------------------------------------------

def _bf16_values(codes):
    """bfloat16 codes -> float64 values through torch's own bfloat16 type."""
    t = torch.from_numpy(np.ascontiguousarray(codes, dtype=np.uint16).view(np.int16)).view(torch.bfloat16)
    return t.to(torch.float64).numpy()


def test_bf16_code_helper_matches_torch():
    for e, m, neg in [(0, 0, False), (-5, 0, False), (20, 0, True), (127, 127, False), (-126, 1, True)]:
        v = _bf16_values([wl.bf16_code(e, m, neg)])[0]
        assert v == (-1) ** neg * (1 + m / 128) * 2.0 ** e


def test_bf16_cancel_pattern():
    n = 1000
    c = wl.bf16_cancel(n)
    v = _bf16_values(c).reshape(n, 8)
    # every vector holds the same multiset, in many different orders
    assert all(sorted(r) == sorted([2.0 ** -5, -2.0 ** 20, 1.0, 2.0 ** 20, 0, 0, 0, 0]) for r in v)
    # each of the four non-zero values appears in every one of the 8 positions
    for x in (2.0 ** -5, -2.0 ** 20, 1.0, 2.0 ** 20):
        assert set(np.nonzero(v == x)[1].tolist()) == set(range(8))
    assert math.fsum(v.reshape(-1)) == n * (1 + 2.0 ** -5)
    # a plain left-to-right FP32 sum of some vectors loses the 2^-5
    lossy = [r for r in v.astype(np.float32) if np.float32(np.cumsum(r, dtype=np.float32)[-1]) != np.float32(1 + 2.0 ** -5)]
    assert lossy


def test_bf16_wide_structure():
    n = 4096
    v = _bf16_values(wl.bf16_wide(n)).reshape(n, 8)
    big = np.abs(v) >= 2.0 ** 8
    assert (big.sum(axis=1) == 2).all()
    assert np.all(v[big].reshape(n, 2).sum(axis=1) == 0)  # +L and -L in every vector
    small = v[~big]
    assert small.min() >= 2.0 ** -12 and small.max() < 2.0 ** 5
    f32 = wl.bf16_as_f32_bits(wl.bf16_wide(n)).astype(np.float64)
    assert np.array_equal(f32, v.reshape(-1))


def test_bf16_code_groups_cover_every_finite_code_once():
    groups = wl.bf16_code_groups()
    allc = np.concatenate(groups)
    finite = [c for c in range(1 << 16) if (c >> 7) & 0xFF != 0xFF]
    assert sorted(allc.tolist()) == finite
    fmax = float(torch.finfo(torch.float32).max)
    for g in groups:
        v = _bf16_values(g)
        assert len(set(np.sign(v[v != 0]))) <= 1  # one sign per group
        # every value a multiple of one power-of-two unit, multiples adding up
        # to < 2^15: every partial sum in any order is exact in FP32
        e = (int(g[-1]) >> 7) & 0xFF
        unit = 2.0 ** (e - 134) if e else 2.0 ** -133
        mult = np.abs(v) / unit
        assert np.all(mult == np.round(mult)) and mult.sum() < 2 ** 15
        assert math.fsum(np.abs(v)) <= fmax


def test_fp8_finite_codes():
    c = wl.fp8_finite_codes()
    assert c.size == 254 and 0x7F not in c and 0xFF not in c
    v = torch.from_numpy(c).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.isfinite(v).all() and v.max() == 448 and v.min() == -448
    assert (v == 0).sum() == 2 and np.abs(v[v != 0]).min() == 2.0 ** -9
