"""The image parity gates (tests/imgcheck.py) catch a single wrong pixel that relative RMS alone lets pass.

The oracle's own image stands in for a GPU result: exact, with FP32-sized noise, and with one pixel, the
edge column or the Nyquist row perturbed.
"""
import numpy as np

import blinksynth as bs
import oracle
from imgcheck import IMG_MAXTOL, IMG_RTOL, image_errors, image_ok


def _ref():
    w = bs.build_workload("tiny")
    return oracle.pipeline(w["volt"], w["enu"], w["freqs"], 10, 1, 256)["images"][0]


def test_gates_pass_fp32_sized_errors():
    ref = _ref()
    rng = np.random.default_rng(1)
    got = (ref + 1e-7 * np.abs(ref).max() * rng.standard_normal(ref.shape)).astype(np.float32)
    assert image_ok(got, ref)


def test_single_pixel_fails_the_pointwise_gate_but_not_rms():
    ref = _ref()
    for y, x in [(128, 128), (0, 0), (255, 17), (40, 255)]:
        got = ref.copy()
        got[y, x] += 2e-5 * np.abs(ref).max()
        rms, mx = image_errors(got, ref)
        assert rms <= IMG_RTOL          # the norm over 65,536 pixels dilutes it ...
        assert mx > IMG_MAXTOL          # ... the pointwise gate does not
        assert not image_ok(got, ref)


def test_edge_column_and_nyquist_row_fail():
    ref = _ref()
    scale = 3e-5 * np.abs(ref).max()
    for sl in [(slice(None), 0), (0, slice(None)), (slice(None), 255)]:
        got = ref.copy()
        got[sl] += scale
        assert not image_ok(got, ref), sl
