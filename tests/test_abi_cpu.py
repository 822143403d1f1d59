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
    assert ctypes.sizeof(B.blink_imaging) == 48
    assert ctypes.sizeof(B.blink_set) == 64


C_CHECK = r"""
#include <stddef.h>
#include <stdio.h>
#include <string.h>
#include "blink.h"

#define OFF(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))

int main(void) {
    printf("sizeof.blink_array %zu\nsizeof.blink_obs %zu\nsizeof.blink_imaging %zu\nsizeof.blink_set %zu\n",
           sizeof(blink_array), sizeof(blink_obs), sizeof(blink_imaging), sizeof(blink_set));
    OFF(blink_array, n_tiles); OFF(blink_array, enu_m); OFF(blink_array, flags); OFF(blink_array, gains);
    OFF(blink_array, jones);
    OFF(blink_obs, n_fine); OFF(blink_obs, fine_stride); OFF(blink_obs, fine_freq_hz); OFF(blink_obs, chan_avg);
    OFF(blink_obs, samples_per_int); OFF(blink_obs, n_samples);
    OFF(blink_imaging, n_pix); OFF(blink_imaging, cell_lambda); OFF(blink_imaging, pol);
    OFF(blink_imaging, include_autos); OFF(blink_imaging, precision); OFF(blink_imaging, support);
    OFF(blink_imaging, phase_l); OFF(blink_imaging, phase_m);
    OFF(blink_set, fine0); OFF(blink_set, n_fine); OFF(blink_set, flags); OFF(blink_set, imaging);
    printf("baselines %lld\n", (long long)blink_n_baselines(144));
    /* an argument error is returned before any device work: no context */
    double enu[6] = {0}, freq[1] = {150e6};
    blink_array arr; memset(&arr, 0, sizeof arr); arr.n_tiles = 2; arr.enu_m = enu;
    blink_obs obs; memset(&obs, 0, sizeof obs); obs.n_fine = 1; obs.fine_freq_hz = freq; obs.chan_avg = 1;
    obs.samples_per_int = 1; obs.n_samples = 1;
    blink_status st = blink_correlate(NULL, &arr, &obs, 0, NULL, NULL, NULL);
    printf("status %s\nmessage_set %d\n", blink_status_name(st), blink_last_error() != NULL);
    return 0;
}
"""


def test_header_is_plain_c_and_matches_binding_layout(lib_path, tmp_path):
    # The header compiles as strict C99 on its own, a C program links against the library and calls it,
    # and every descriptor field sits at the offset the Python binding marshals it to.
    import shutil
    import subprocess
    from paper_2505_15204_gb300 import blink as B
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    src = tmp_path / "abi_check.c"
    src.write_text(C_CHECK)
    exe = tmp_path / "abi_check"
    libdir = os.path.dirname(lib_path)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                    os.path.join(ROOT, "include"), str(src), "-o", str(exe), lib_path,
                    "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(line.rsplit(" ", 1) for line in out if line)
    for name in ("blink_array", "blink_obs", "blink_imaging", "blink_set"):
        cls = getattr(B, name)
        assert int(got["sizeof." + name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[f"{name}.{field}"]) == getattr(cls, field).offset, (name, field)
    assert got["baselines"] == "10440"
    assert got["status"] == "BLINK_ERR_INVALID_ARG"
    assert got["message_set"] == "1"
