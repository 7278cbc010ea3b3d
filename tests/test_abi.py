"""The C-ABI library builds, loads and exports every function that
include/*.h declares; the ctypes mirror matches the C layout.  CPU only: no
compute call is made (this machine has no GPU)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from paper_2608_15764_gb300 import _abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _abi.load()


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(sl_[a-z0-9_]+)\s*\(", text, re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["sl_run", "sl_sweep", "sl_enqueue", "sl_run_host", "sl_plan", "sl_fill_splitmix64",
                     "sl_flush_l2", "sl_device_info", "sl_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name
    # and the binding knows a prototype for each
    assert set(_declared_functions()) <= set(_abi.PROTOTYPES)


def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "streamload.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(sl_config), sizeof(sl_result), sizeof(sl_devinfo));
  printf("%zu %zu %zu\n", offsetof(sl_config, stream), offsetof(sl_result, sum_u32), offsetof(sl_result, smem_bytes));
  printf("%zu %zu\n", offsetof(sl_devinfo, name), offsetof(sl_devinfo, l2_bytes));
  printf("%zu %zu %zu\n", sizeof(sl_twostream_result), offsetof(sl_twostream_result, sum_u32),
         offsetof(sl_twostream_result, b_covers_a));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    vals = list(map(int, out))
    assert vals[0] == ctypes.sizeof(_abi.sl_config)
    assert vals[1] == ctypes.sizeof(_abi.sl_result)
    assert vals[2] == ctypes.sizeof(_abi.sl_devinfo)
    assert vals[3] == _abi.sl_config.stream.offset
    assert vals[4] == _abi.sl_result.sum_u32.offset
    assert vals[5] == _abi.sl_result.smem_bytes.offset
    assert vals[6] == _abi.sl_devinfo.name.offset
    assert vals[7] == _abi.sl_devinfo.l2_bytes.offset
    assert vals[8] == ctypes.sizeof(_abi.sl_twostream_result)
    assert vals[9] == _abi.sl_twostream_result.sum_u32.offset
    assert vals[10] == _abi.sl_twostream_result.b_covers_a.offset


def test_library_targets_sm_103a_only():
    # every CUDA translation unit is compiled with exactly one -gencode for sm_103a
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(_abi, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _abi.load(str(tmp_path / "nope.so"))
