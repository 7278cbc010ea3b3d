"""Host-side behaviour of the C ABI that needs no GPU: every entry point
rejects malformed arguments with its documented status and a message before
it touches a device, and -- on a machine without a usable GPU -- returns
SL_ERR_NODEV (never aborts, traps or prints).  CPU only: no kernel runs."""
import ctypes

import pytest

from paper_2608_15764_gb300 import _abi, build

C = ctypes
ARG, ALIGN, NODEV = _abi.SL_ERR_ARG, _abi.SL_ERR_ALIGN, _abi.SL_ERR_NODEV


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _abi.load()


def _cfg(mech=_abi.SL_LDG, **kw):
    c = _abi.sl_config()
    c.mech, c.k, c.cta, c.stage_bytes, c.stages = mech, 2, 256, 16384, 4
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _expect(lib, status, want):
    assert status == want, (status, lib.sl_last_error())
    assert lib.sl_last_error()


def test_argument_errors_before_any_device_use(lib):
    r = _abi.sl_result()
    cfg = _cfg()
    ch = _abi.sl_chase_result()
    tw = _abi.sl_twostream_result()
    one = (C.c_void_p * 1)(16)
    cases = [
        (lib.sl_run(16, 16, 0, C.byref(cfg), None), ARG),
        (lib.sl_plan(16, 0, C.byref(cfg), None), ARG),
        (lib.sl_enqueue(16, 16, 0, C.byref(cfg), None), ARG),
        (lib.sl_enqueue(16, 16, 0, C.byref(cfg), 20), ARG),  # dev_out not 8-byte aligned
        (lib.sl_sweep(16, 16, 0, None, 1, 1, 0, 0, C.byref(r)), ARG),
        (lib.sl_sweep(16, 16, 0, C.byref(cfg), 1, 0, 0, 0, C.byref(r)), ARG),
        (lib.sl_sweep(16, 16, 0, C.byref(cfg), 1, 1, 0, 7, C.byref(r)), ARG),
        (lib.sl_fill_splitmix64(8, 16, 1, None), ALIGN),
        (lib.sl_fill_splitmix64(16, 24, 1, None), ALIGN),
        (lib.sl_fill_splitmix64(None, 32, 1, None), ARG),
        (lib.sl_run_host(None, 16, 0, C.byref(cfg), C.byref(r)), ARG),
        (lib.sl_run_host(16, 24, 0, C.byref(cfg), C.byref(r)), ALIGN),
        (lib.sl_run_host(16, 16, 0, C.byref(_cfg(target_loads=5)), C.byref(r)), ARG),
        (lib.sl_enqueue_steps(one, 1, 16, 0, None, 2, 64), ARG),
        (lib.sl_enqueue_steps(one, 1, 16, 0, C.byref(cfg), 0, 64), ARG),
        (lib.sl_enqueue_steps(one, 0, 16, 0, C.byref(cfg), 2, 64), ARG),
        (lib.sl_enqueue_steps(one, 1, 16, 0, C.byref(_cfg(flush_l2=1)), 2, 64), ARG),
        (lib.sl_coverage(16, 16, C.byref(cfg), None, C.byref(r)), ARG),
        (lib.sl_coverage(16, 16, C.byref(cfg), 64, None), ARG),
        (lib.sl_coverage(16, 16, C.byref(_cfg(_abi.SL_LDG4)), 64, C.byref(r)), ARG),
        (lib.sl_chase(16, 16, 0, 0, 1, 0, None, None), ARG),
        (lib.sl_chase(16, 18, 0, 0, 1, 0, None, C.byref(ch)), ALIGN),
        (lib.sl_chase(16, 16, 4, 0, 1, 0, None, C.byref(ch)), ARG),
        (lib.sl_twostream(16, 16, 32, 16, 1, 0, 1, 2, 0, None, C.byref(tw)), ARG),
        (lib.sl_twostream(16, 16, 32, 16, 1, 16, 17, 2, 0, None, C.byref(tw)), ARG),
        (lib.sl_twostream(16, 16, 32, 16, 1, 1, 1, 3, 0, None, C.byref(tw)), ARG),
        (lib.sl_twostream(16, 16, 32, 16, -1, 1, 1, 2, 0, None, C.byref(tw)), ARG),
        (lib.sl_twostream(None, 16, 32, 16, 1, 1, 1, 2, 0, None, C.byref(tw)), ARG),
        (lib.sl_twostream(16, 16, 32, 24, 1, 1, 1, 2, 0, None, C.byref(tw)), ALIGN),
        (lib.sl_twostream(16, 16, 32, 16, 1, 1, 1, 2, 0, None, None), ARG),
        (lib.sl_batch_create(None, 1, None, 0, C.byref(C.c_void_p())), ARG),
        (lib.sl_batch_create(None, 0, None, 1, None), ARG),
        (lib.sl_run_noalloc(16, 16, 0, None, 64), ARG),
        (lib.sl_run_noalloc(16, 16, 0, C.byref(_cfg(_abi.SL_CPASYNC)), 64), ARG),
        (lib.sl_run_noalloc(16, 16, 0, C.byref(_cfg(flush_l2=1)), 64), ARG),
        (lib.sl_run_noalloc(16, 16, 0, C.byref(_cfg(target_loads=7)), 64), ARG),
        (lib.sl_run_noalloc(16, 24, 0, C.byref(cfg), 64), ALIGN),
    ]
    for i, (status, want) in enumerate(cases):
        assert status == want, (i, status, want, lib.sl_last_error())


def test_no_device_is_reported_not_fatal(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _abi.sl_result()
    info = _abi.sl_devinfo()
    cfg = _cfg()
    _expect(lib, lib.sl_device_info(C.byref(info)), NODEV)
    _expect(lib, lib.sl_run(16, 16, 0, C.byref(cfg), C.byref(r)), NODEV)
    _expect(lib, lib.sl_plan(1 << 20, 0, C.byref(cfg), C.byref(r)), NODEV)
    _expect(lib, lib.sl_flush_l2(None), NODEV)
    _expect(lib, lib.sl_fill_splitmix64(16, 16, 1, None), NODEV)
    assert b"device" in lib.sl_last_error()
