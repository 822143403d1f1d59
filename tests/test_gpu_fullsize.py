"""Parity at the benchmark's full size (GPU): one 50 ms chunk of the full-band workload.

144 tiles, 768 output channels of 40 kHz (K = 40), 50 integrations of 1 ms, 38,400 Stokes-I images of
512^2 - the launch configuration bench.py times.  Correlation is checked bit for bit (FP8 against FP32
on every item, and against the integer oracle on sampled items); images are checked on a sample of
image ids against the FP64 oracle.
"""
import numpy as np
import pytest

import blinksynth as bs
import oracle
from imgcheck import assert_image_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def chunk():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return bs.build_workload("fullband", chunk=4, workers=8)


def test_fullband_chunk_correlation_fp8_equals_fp32_and_oracle(chunk):
    from paper_2505_15204_gb300 import blink as B
    w = chunk["workload"]
    ctx = B.blink_create(0)
    try:
        arr, obs = B.Array(chunk["enu"]), B.Obs(chunk["freqs"], w.chan_avg, w.samples_per_int, w.samples_per_chunk)
        volt = torch.from_numpy(chunk["volt"]).cuda()
        shape = (50, 768, 10440, 4, 2)
        a = torch.empty(shape, dtype=torch.float32, device="cuda")
        B.blink_correlate(ctx, arr, obs, B.BLINK_CORR_FP8, volt, a)
        b = torch.empty(shape, dtype=torch.float32, device="cuda")
        B.blink_correlate(ctx, arr, obs, B.BLINK_CORR_FP32, volt, b)
        B.blink_sync(ctx)
        assert torch.equal(a, b)
        del b
        for tau, f in [(0, 0), (7, 383), (49, 767), (25, 100)]:
            S = oracle.correlate_one(chunk["volt"], w.samples_per_int, w.chan_avg, tau, f)
            want = oracle.visibilities(S, w.k)
            got = a[tau, f].cpu().numpy()
            assert np.array_equal(got[..., 0], want.real) and np.array_equal(got[..., 1], want.imag), (tau, f)
    finally:
        B.blink_destroy(ctx)


def test_fullband_chunk_images_on_sampled_ids(chunk):
    from paper_2505_15204_gb300 import blink as B
    w = chunk["workload"]
    ctx = B.blink_create(0)
    try:
        arr, obs = B.Array(chunk["enu"]), B.Obs(chunk["freqs"], w.chan_avg, w.samples_per_int, w.samples_per_chunk)
        volt = torch.from_numpy(chunk["volt"]).cuda()
        img = torch.empty((38400, 512, 512), dtype=torch.float32, device="cuda")
        B.blink_pipeline(ctx, arr, obs, B.Imaging(512), B.BLINK_CORR_FP8, B.BLINK_MODE_BATCHED, volt, img)
        B.blink_sync(ctx)
        ids = np.array([0, 1, 767, 768, 12345, 19200, 30001, 38399])
        ref = oracle.pipeline(chunk["volt"], chunk["enu"], chunk["freqs"], w.samples_per_int, w.chan_avg, 512, ids=ids,
                              n_threads=8)
        got = img[torch.from_numpy(ids).cuda()].cpu().numpy()
        for k, q in enumerate(ids):
            assert_image_close(got[k], ref["images"][k], q)
    finally:
        B.blink_destroy(ctx)
