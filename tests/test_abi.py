"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/*.h.  CPU only: nothing here launches a kernel."""
import ctypes
import glob
import os
import re
import shutil

import pytest

import paper_1307_5700_gb300 as tp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(tp_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    tp.build()
    return ctypes.CDLL(tp.LIB_PATH)


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 20
    assert declared == set(tp.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_struct_layouts():
    assert ctypes.sizeof(tp.tp_candidate) == 24
    assert tp.CAND_DTYPE.itemsize == 24
    assert ctypes.sizeof(tp.tp_rfi_params) == 40


def test_host_only_entry_points(lib):
    p = tp.tp_rfi_defaults()
    assert (p.enable_channel, p.enable_spectrum, p.chunk_width) == (1, 1, 256)
    assert (p.tau_channel, p.tau_spectrum, p.stats_mode) == (5.0, 6.0, tp.TP_STATS_BLOCK)
    assert tp.tp_version() >= 100


def test_engine_create_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(tp.TpError) as ei:
        tp.tp_engine_create(0)
    assert ei.value.code in (tp.TP_ECUDA, tp.TP_EINVAL)
