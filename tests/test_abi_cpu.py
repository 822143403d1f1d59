"""The C-ABI library loads and exports every entry point that include/blink.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "blink.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(blink_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2505_15204_gb300.build import build
    return build()


def test_library_exports_every_declared_entry_point(lib_path):
    names = declared_entry_points()
    assert {"blink_correlate", "blink_grid", "blink_image", "blink_pipeline"} <= set(names)
    lib = ctypes.CDLL(lib_path)
    for n in names:
        assert hasattr(lib, n), n


def test_binding_wraps_every_declared_entry_point(lib_path):
    from paper_2505_15204_gb300 import blink as B
    assert sorted(B.ENTRY_POINTS) == declared_entry_points()
    for n in B.ENTRY_POINTS:
        assert callable(getattr(B, n)), n


def test_host_only_calls_without_gpu(lib_path):
    from paper_2505_15204_gb300 import blink as B
    assert B.blink_n_baselines(128) == 8256
    assert B.blink_n_baselines(144) == 10440
    assert B.blink_status_name(B.BLINK_ERR_INVALID_ARG) == "BLINK_ERR_INVALID_ARG"
    # argument errors are reported before any device work
    with pytest.raises(B.BlinkError) as e:
        B.blink_correlate(None, B.Array(__import__("numpy").zeros((4, 3))),
                          B.Obs(__import__("numpy").ones(2), 1, 1, 1), 0, 0, 0)
    assert e.value.status == B.BLINK_ERR_INVALID_ARG


def test_struct_layout_matches_header(lib_path):
    from paper_2505_15204_gb300 import blink as B
    assert ctypes.sizeof(B.blink_array) == 40
    assert ctypes.sizeof(B.blink_obs) == 32
    assert ctypes.sizeof(B.blink_imaging) == 32
    assert ctypes.sizeof(B.blink_set) == 48
