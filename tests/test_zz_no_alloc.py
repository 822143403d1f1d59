"""The allocation-free imaging entry point against the regular one (GPU).

blink_image_noalloc serves callers that cannot allocate device memory during imaging: a real-time
pipeline that reserved all of its device memory when the observation started, or an application whose
device memory belongs to another allocator.  It works in a static scratch array that every call shares,
so each test calls it several times in a row with different grids and checks every result against
blink_image within the imaging-stage tolerance.  The cases cover one pass (the whole batch in the
scratch), several passes (1024^2 with FP32 storage: three images per pass) and the largest side (2048^2
with BF16 storage: one image per pass).  The file sorts last, so that under ``-x`` a failure here leaves
every other result reported; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

import blinksynth as bs
import oracle
from imgcheck import assert_image_close

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


def _random_grids(n, n_pix, seed):
    # half planes of random cells: the two entry points run the same passes, so any grid compares them
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, n_pix, n_pix // 2 + 1, 2)).astype(np.float32)
    return g, rng.uniform(1e3, 2e4, n).astype(np.float32)


def _compare(B, ctx, n_pix, g, wts, precision):
    n = g.shape[0]
    d_g = torch.from_numpy(g).cuda()
    d_w = torch.from_numpy(wts).cuda()
    im = B.Imaging(n_pix, precision=precision)
    want = torch.empty((n, n_pix, n_pix), dtype=torch.float32, device="cuda")
    got = torch.full((n, n_pix, n_pix), float("nan"), dtype=torch.float32, device="cuda")
    B.blink_image(ctx, im, d_g, n, d_w, want)
    B.blink_image_noalloc(im, d_g, n, d_w, got)
    torch.cuda.synchronize()
    B.blink_sync(ctx)
    a, b = got.cpu().numpy(), want.cpu().numpy()
    for q in range(n):
        assert_image_close(a[q], b[q], (n_pix, precision, q), rms_tol=IMAGE_STAGE_RTOL)


def test_image_noalloc_matches_image_on_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_15204_gb300 import blink as B
    ctx = B.blink_create(0)
    try:
        B.blink_image_noalloc(B.Imaging(512), torch.zeros(2, device="cuda"), 0, torch.zeros(2, device="cuda"),
                              torch.zeros(2, device="cuda"))                 # a zero-image call: the warm-up
        _compare(B, ctx, 512, *_grids("precision", 512), B.BLINK_PREC_FP32)
        _compare(B, ctx, 256, *_grids("coarse", 256, n_samples=10, fine=5), B.BLINK_PREC_FP32)
        _compare(B, ctx, 1024, *_random_grids(7, 1024, 3), B.BLINK_PREC_FP32)     # three passes
        _compare(B, ctx, 2048, *_random_grids(2, 2048, 4), B.BLINK_PREC_BF16)     # one image per pass
        _compare(B, ctx, 512, *_grids("precision", 512), B.BLINK_PREC_FP32)       # after the larger calls
    finally:
        B.blink_destroy(ctx)


def test_pipeline_captures_in_a_graph_after_noalloc_calls():
    # the allocation-free entry point loaded and used first; a new context's pipeline then runs eagerly
    # (plan and workspace) and replays from a CUDA graph to the same images
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_15204_gb300 import blink as B
    g, wts = _random_grids(3, 256, 5)
    out = torch.empty((3, 256, 256), dtype=torch.float32, device="cuda")
    B.blink_image_noalloc(B.Imaging(256), torch.from_numpy(g).cuda(), 3, torch.from_numpy(wts).cuda(), out)
    torch.cuda.synchronize()
    w = bs.build_workload("coarse", n_samples=20)
    volt, freqs = np.ascontiguousarray(w["volt"][:, :16]), w["freqs"][:16]
    ctx = B.blink_create(0)
    try:
        arr, obs, im = B.Array(w["enu"]), B.Obs(freqs, 1, 10, 20), B.Imaging(256)
        d = torch.from_numpy(volt).cuda()
        eager = torch.empty((32, 256, 256), dtype=torch.float32, device="cuda")
        rep = torch.zeros_like(eager)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            B.blink_pipeline(ctx, arr, obs, im, 1, 0, d, eager, stream=s)
        s.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s, capture_error_mode="relaxed"):
            B.blink_pipeline(ctx, arr, obs, im, 1, 0, d, rep, stream=s)
        graph.replay()
        torch.cuda.synchronize()
        B.blink_sync(ctx)
        assert torch.equal(rep, eager)
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
