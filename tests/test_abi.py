"""The C-ABI library loads and exports every symbol include/seas.h declares; struct layouts match; argument
checks of the binding.  No GPU needed (no compute calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2603_00383_gb300 import seas

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "seas.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(seas_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = seas.lib()
    decl = declared_symbols()
    assert len(decl) >= 20
    missing = [s for s in decl if not hasattr(L, s)]
    assert missing == []
    assert sorted(seas.EXPORTED) == decl


def test_struct_layouts_match_header():
    assert ctypes.sizeof(seas.seas_fault) == 40
    assert ctypes.sizeof(seas.seas_medium) == 32
    assert ctypes.sizeof(seas.seas_hparams) == 64
    assert ctypes.sizeof(seas.seas_net_info) == 16
    assert ctypes.sizeof(seas.seas_op_stats) == 13 * 8
    assert ctypes.sizeof(seas.seas_timing) == 7 * 8 + 7 * 8 + 16


def test_strerror_covers_every_status():
    for st in (0, -1, -2, -3, -4, -5, -6, -7):
        assert seas.seas_strerror(st) != "unknown status"
    assert seas.seas_strerror(-99) == "unknown status"


def test_no_device_is_an_error_status_not_a_crash():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(seas.SeasError) as e:
        seas.seas_create(0)
    assert e.value.status == seas.SEAS_ECUDA


def test_binding_rejects_bad_buffers():
    with pytest.raises(ValueError):
        seas._buf(np.zeros(4, dtype=np.float32), 4, "V")
    with pytest.raises(ValueError):
        seas._buf(np.zeros((4, 2))[:, 0], 4, "V")
    with pytest.raises(ValueError):
        seas._buf(np.zeros(5), 4, "V")
    ptr, mem = seas._buf(np.zeros(4), 4, "V")
    assert mem == seas.SEAS_MEM_HOST
