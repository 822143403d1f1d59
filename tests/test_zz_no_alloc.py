"""The allocation-free imaging entry point against the regular one (GPU).

blink_image_noalloc serves callers that cannot allocate device memory during imaging (a real-time
pipeline that reserved its memory up front, or an application whose memory belongs to another
allocator).  It uses a static scratch array shared by all calls, so this test calls it twice in a row with
different grids and checks each result against blink_image within the imaging-stage tolerance.  The file
is named to be collected after the core parity suite (its graph captures run before the static scratch
exists).
"""
import numpy as np
import pytest

import blinksynth as bs
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

IMAGE_STAGE_RTOL = 1e-5      # relative RMS, the tolerance of the imaging-stage tests


def _grids(name, n_pix, n_samples=None, fine=None):
    w = bs.build_workload(name, n_samples=n_samples)
    volt, freqs = w["volt"], w["freqs"]
    if fine is not None:
        volt, freqs = np.ascontiguousarray(volt[:, :fine]), freqs[:fine]
    ref = oracle.pipeline(volt, w["enu"], freqs, 10, 1, n_pix, want_grids=True, n_threads=4)
    h = ref["grids"][:, :, : n_pix // 2 + 1]
    g = np.stack([h.real, h.imag], axis=-1).astype(np.float32)
    return g, ref["W"].astype(np.float32)


def test_image_noalloc_matches_image_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_15204_gb300 import blink as B
    ctx = B.blink_create(0)
    try:
        calls = [(512, _grids("precision", 512)), (256, _grids("coarse", 256, n_samples=10, fine=5))]
        for n_pix, (g, wts) in calls:
            n = g.shape[0]
            d_g = torch.from_numpy(g).cuda()
            d_w = torch.from_numpy(wts).cuda()
            im = B.Imaging(n_pix)
            want = torch.empty((n, n_pix, n_pix), dtype=torch.float32, device="cuda")
            got = torch.full((n, n_pix, n_pix), float("nan"), dtype=torch.float32, device="cuda")
            B.blink_image(ctx, im, d_g, n, d_w, want)
            B.blink_image_noalloc(im, d_g, n, d_w, got)
            torch.cuda.synchronize()
            B.blink_sync(ctx)
            a, b = got.cpu().numpy(), want.cpu().numpy()
            for q in range(n):
                err = float(np.linalg.norm(a[q] - b[q]) / np.linalg.norm(b[q]))
                assert err <= IMAGE_STAGE_RTOL, (n_pix, q, err)
    finally:
        B.blink_destroy(ctx)


def test_image_noalloc_rejects_a_side_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_15204_gb300 import blink as B
    d = torch.zeros(16, device="cuda")
    with pytest.raises(B.BlinkError) as e:
        B.blink_image_noalloc(B.Imaging(2048), d, 1, d, d)
    assert e.value.status == B.BLINK_ERR_UNSUPPORTED
