"""Failure detection without a GPU fault: the TMA ring's waits are bounded.

With SL_DEBUG_TMA_SKIP_STAGE the producer leaves the second stage of every
CTA unarmed, so the consumers wait on a phase that never completes.  Their
bounded wait (50 ms for debug runs, by %globaltimer, plus an iteration cap)
gives up, records a device error code and raises the CTA's abort flag; the
producer sees the flag, waits for the copies it did issue to land, and the
kernel exits normally.  The call must return SL_ERR_TIMEOUT and the CUDA
context must stay usable.  Nothing here traps, faults or hangs."""
import numpy as np
import pytest

import oracle
from paper_2608_15764_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2608_15764_gb300 as sl
    sl.load()
    return sl


@pytest.mark.parametrize("ring,stage", [("cta", 16384), ("warp", 4096)])
def test_tma_unarmed_stage_times_out_and_context_survives(sl, ring, stage):
    nbytes = 1 << 20
    host = workloads.splitmix_u32(9, nbytes // 4)
    dev = torch.from_numpy(host.view(np.uint8)).cuda()
    bad = sl.config("tma", cta=128, grid=4, stage_bytes=stage, stages=4, ring=ring,
                    debug_flags=sl.SL_DEBUG_TMA_SKIP_STAGE)
    for _ in range(2):
        with pytest.raises(sl.SLError) as e:
            sl.sl_run(dev, dtype=sl.SL_U32, cfg=bad)
        assert e.value.status == sl.SL_ERR_TIMEOUT
        assert "timed out" in sl.sl_last_error()
        # the same context still computes correct results, and the error
        # word was cleared for the next launch
        r = sl.sl_run(dev, dtype=sl.SL_U32, cfg=sl.config("tma", cta=128, grid=4, stage_bytes=stage, stages=4,
                                                          ring=ring))
        assert r.status == 0 and (r.sum_u32, r.xor_u64) == oracle.checksum(host)
    torch.cuda.synchronize()
