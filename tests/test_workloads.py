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
