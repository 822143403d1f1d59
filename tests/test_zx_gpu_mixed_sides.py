"""Parity of the mixed-radix imaging path with the CPU oracle (GPU): image sides that are not powers of
two (the 1200 x 1200 images of the paper's 20 ms demonstration, and 96, 150, 600, 2400) and sides above
2048 (the 8192 x 8192 images of its long-exposure test), through every entry point that images.

Whole images are compared with the oracle where its transform finishes in seconds; the 8192 image is
compared on sampled pixels, each summed directly by the oracle over the grid's nonzero cells.  The file
sorts after the core parity suite so that a failure here, under ``-x``, leaves the core results reported.
"""
import numpy as np
import pytest

import blinksynth as bs
import oracle

from test_gpu_parity import B, _case, ctx, dev, rel_rms  # noqa: F401
from imgcheck import assert_image_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _grids(n, name="precision"):
    w, volt, freqs, _ = _case(name)
    ref = oracle.pipeline(volt, w["enu"], freqs, 10, 1, n, want_grids=True)
    h = ref["grids"][0][:, : n // 2 + 1]
    return np.stack([h.real, h.imag], axis=-1).astype(np.float32)[None], ref


@pytest.mark.parametrize("n", [96, 150, 600, 1200])
def test_image_stage_on_mixed_sides(B, ctx, n):
    # 150 = 2 x 3 x 5^2: the row transform has the odd length 75
    g, ref = _grids(n)
    img = torch.full((1, n, n), float("nan"), dtype=torch.float32, device="cuda")
    wt = torch.tensor([ref["W"][0]], dtype=torch.float32, device="cuda")
    B.blink_image(ctx, B.Imaging(n), dev(g), 1, wt, img)
    B.blink_sync(ctx)
    assert_image_close(img[0].cpu().numpy(), ref["images"][0], n, rms_tol=1e-5)


def test_image_stage_sides_in_descending_order(B, ctx):
    # the shared-memory limit is raised per kernel instance: a larger side first must not leave a smaller
    # side's instance (same signature) without its own limit
    for n in (2048, 1024, 2400, 1200):
        g, ref = _grids(n)
        img = torch.full((1, n, n), float("nan"), dtype=torch.float32, device="cuda")
        wt = torch.tensor([ref["W"][0]], dtype=torch.float32, device="cuda")
        B.blink_image(ctx, B.Imaging(n), dev(g), 1, wt, img)
        B.blink_sync(ctx)
        assert_image_close(img[0].cpu().numpy(), ref["images"][0], n, rms_tol=1e-5)


def test_image_stage_nyquist_column_on_a_mixed_side(B, ctx):
    n = 120
    G = np.zeros((n, n), complex)
    G[7, n // 2] = 1 + 2j
    G[-7 % n, n // 2] = 1 - 2j
    G[3, 11] = 0.5 - 0.25j
    G[-3 % n, -11 % n] = 0.5 + 0.25j
    a = np.fft.ifft2(G) * n * n
    want = np.roll(a.real, (n // 2, n // 2), axis=(0, 1))
    g = np.stack([G[:, : n // 2 + 1].real, G[:, : n // 2 + 1].imag], -1).astype(np.float32)[None]
    img = torch.empty((1, n, n), dtype=torch.float32, device="cuda")
    B.blink_image(ctx, B.Imaging(n), dev(g), 1, torch.ones(1, device="cuda"), img)
    B.blink_sync(ctx)
    assert np.abs(img[0].cpu().numpy() - want).max() < 1e-5


MIXED_CASES = [
    # name, n_samples, fine, chan_avg, n_pix, pol, autos, flags
    ("precision", None, None, 1, 1200, 0, 1, False),
    ("coarse", 20, 8, 4, 150, 0, 1, False),
    ("uneven", 20, 3, 1, 96, 1, 0, True),
    ("coarse", 30, 4, 1, 600, 0, 1, False),
]


@pytest.mark.parametrize("arith", [0, 1], ids=["fp32", "fp8"])
@pytest.mark.parametrize("mode", [0, 1], ids=["batched", "plain"])
@pytest.mark.parametrize("case", MIXED_CASES, ids=[f"{c[0]}-{c[4]}" for c in MIXED_CASES])
def test_pipeline_on_mixed_sides_matches_oracle(B, ctx, case, mode, arith):
    name, ns_total, fine, c, n_pix, pol, autos, flags = case
    w, volt, freqs, fl = _case(name, ns_total, fine, flags)
    T = volt.shape[0] // 10
    F = len(freqs) // c
    img = torch.full((T * F, n_pix, n_pix), float("nan"), dtype=torch.float32, device="cuda")
    wts = torch.empty(T * F, dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, B.Array(w["enu"], fl), B.Obs(freqs, c, 10, volt.shape[0]),
                     B.Imaging(n_pix, pol=pol, include_autos=autos), arith, mode, dev(volt), img, wts)
    B.blink_sync(ctx)
    ref = oracle.pipeline(volt, w["enu"], freqs, 10, c, n_pix, flags=fl, pol=pol, autos=bool(autos), n_threads=8)
    got = img.cpu().numpy()
    for q in range(T * F):
        assert_image_close(got[q], ref["images"][q], q)
        assert wts[q].item() == ref["W"][q]


@pytest.mark.parametrize("arith", [0, 1], ids=["fp32", "fp8"])
@pytest.mark.parametrize("n_pix,W,pc", [(600, 6, (0.0, 0.0)), (150, 4, (0.2, -0.1)), (1200, 8, (0.0, 0.0))])
def test_kernel_gridding_and_phase_centre_on_mixed_sides(B, ctx, n_pix, W, pc, arith):
    # grid side 2 n_pix (1200, 300, 2400) through the mixed-radix passes with the crop and grid correction
    w, volt, freqs, fl = _case("coarse", 20, 4, False)
    T, F = 2, 4
    img = torch.full((T * F, n_pix, n_pix), float("nan"), dtype=torch.float32, device="cuda")
    wts = torch.empty(T * F, dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, B.Array(w["enu"]), B.Obs(freqs, 1, 10, 20), B.Imaging(n_pix, support=W, phase_centre=pc),
                     arith, 0, dev(volt), img, wts)
    B.blink_sync(ctx)
    ref = oracle.pipeline(volt, w["enu"], freqs, 10, 1, n_pix, n_threads=8, support=W, phase_centre=pc)
    got = img.cpu().numpy()
    for q in range(T * F):
        assert_image_close(got[q], ref["images"][q], q)
        assert wts[q].item() == ref["W"][q]


def test_mixed_side_pipeline_is_bitwise_reproducible(B, ctx):
    w, volt, freqs, _ = _case("coarse", 20, 8)
    outs = []
    for _ in range(2):
        img = torch.empty((16, 1200, 1200), dtype=torch.float32, device="cuda")
        B.blink_pipeline(ctx, B.Array(w["enu"]), B.Obs(freqs, 1, 10, 20), B.Imaging(1200), 1, 0, dev(volt), img)
        B.blink_sync(ctx)
        outs.append(img.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_mixed_side_bf16_storage_error_is_reported(B, ctx):
    w, volt, freqs, _ = _case("precision")
    img = torch.empty((1, 1200, 1200), dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, B.Array(w["enu"]), B.Obs(freqs, 1, 10, 10), B.Imaging(1200, precision=1), 1, 0, dev(volt),
                     img)
    B.blink_sync(ctx)
    ref = oracle.pipeline(volt, w["enu"], freqs, 10, 1, 1200)["images"][0]
    got = img[0].cpu().numpy()
    err = (rel_rms(got, ref), float(np.abs(got - ref).max()))
    print("bf16 storage at 1200: rel RMS / max abs", err)
    assert err[0] < 2e-2


def test_many_waves_on_a_mixed_side_sampled(B, ctx):
    # 3 integrations x 64 channels of 1200^2 (5.8 MB of column results each): several waves of the
    # column and row passes; the oracle checks a sample of images across wave boundaries
    w, volt, freqs, _ = _case("coarse", 30, 64)
    n = 3 * 64
    img = torch.empty((n, 1200, 1200), dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, B.Array(w["enu"]), B.Obs(freqs, 1, 10, 30), B.Imaging(1200), 1, 0, dev(volt), img)
    B.blink_sync(ctx)
    ids = np.array([0, 7, 8, 9, 63, 64, 100, 191])
    ref = oracle.pipeline(volt, w["enu"], freqs, 10, 1, 1200, ids=ids, n_threads=8)
    for k, q in enumerate(ids):
        assert_image_close(img[q].cpu().numpy(), ref["images"][k], q)


def test_8192_image_on_sampled_pixels(B, ctx):
    # one 8192 x 8192 image (the paper's long-exposure side): grid and W from the oracle's steps, pixels summed
    # directly by the oracle over the grid's nonzero cells, at the phase centre, along the middle row and
    # column, at the edges and at random positions
    n = 8192
    w = bs.build_workload("tiny")
    volt, enu, freqs = w["volt"], w["enu"], w["freqs"]
    img = torch.full((1, n, n), float("nan"), dtype=torch.float32, device="cuda")
    wts = torch.empty(1, dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, B.Array(enu), B.Obs(freqs, 1, 10, 10), B.Imaging(n), 1, 0, dev(volt), img, wts)
    B.blink_sync(ctx)
    S = oracle.correlate(volt, 10, 1)[0, 0]
    nu = float(oracle.output_freqs(freqs, 1)[0])
    du = oracle.default_cell(enu, nu, n)
    iu, iv, keep = oracle.cells(oracle.uvw(enu, nu), du, n)
    G, Wsum = oracle.grid(S, enu.shape[0], 10, iu, iv, keep, n)
    assert wts[0].item() == Wsum
    rng = np.random.default_rng(8192)
    pts = [(n // 2, n // 2), (0, 0), (n - 1, n - 1), (0, n - 1), (n - 1, 0)]
    pts += [(n // 2, x) for x in range(0, n, 97)] + [(y, n // 2) for y in range(0, n, 89)]
    pts += [tuple(p) for p in rng.integers(0, n, size=(600, 2))]
    yx = np.array(pts, dtype=np.int32)
    want = oracle.image_pixels(G, Wsum, yx)
    full = img[0]
    got = full[torch.from_numpy(yx[:, 0]).long().cuda(), torch.from_numpy(yx[:, 1]).long().cuda()].cpu().numpy()
    scale = float(np.sqrt(np.mean(want ** 2)))
    err = np.abs(got.astype(np.float64) - want)
    print("8192 sampled pixels: rel RMS", float(np.sqrt(np.mean(err ** 2))) / scale, "max abs / RMS", err.max() / scale)
    assert np.sqrt(np.mean(err ** 2)) <= 1e-4 * scale
    assert err.max() <= 1e-3 * scale
    assert not torch.isnan(full).any().item()


def test_dedispersion_on_a_mixed_side(B, ctx):
    rng = np.random.default_rng(5)
    T, F, n = 5, 3, 150
    cube = rng.standard_normal((T, F, n, n)).astype(np.float32)
    delays = [0, 2, 1]
    out = torch.empty((T - 2, n, n), dtype=torch.float32, device="cuda")
    B.blink_dedisperse(ctx, dev(cube), T, F, n, delays, out)
    B.blink_sync(ctx)
    ref = oracle.dedisperse(cube.astype(np.float64), delays)
    assert np.abs(out.cpu().numpy() - ref).max() < 1e-5


# ---------------------------------------------------------------------------------------------------
# averaged images: one transform per output, averaged in the uv plane
# ---------------------------------------------------------------------------------------------------

AVG_CASES = [
    # name, n_samples, fine, chan_avg, n_pix, support, t_avg, f_avg, pointing, flags
    ("coarse", 40, 8, 1, 256, 0, 1, 8, (0.0, 0.0), False),      # band average of every integration
    ("coarse", 40, 8, 1, 256, 0, 4, 1, (0.0, 0.0), False),      # time average of every channel
    ("coarse", 40, 8, 2, 1200, 0, 2, 2, (0.0, 0.0), False),     # both
    ("uneven", 20, 6, 1, 150, 0, 2, 6, (0.0, 0.0), True),       # one long-exposure image, flagged tiles
    ("coarse", 20, 4, 1, 300, 6, 2, 4, (0.2, -0.1), False),     # kernel gridding, off zenith
    ("precision", None, None, 1, 512, 0, 1, 1, (0.0, 0.0), False),   # nothing averaged
    ("coarse", 20, 16, 1, 256, 0, 1, 16, (0.0, 0.0), False),    # 16 channels: the grid summed first
    ("coarse", 20, 16, 1, 1200, 0, 2, 16, (0.15, -0.2), True),  # the same, time too, off zenith, flags
]


@pytest.mark.parametrize("arith", [0, 1], ids=["fp32", "fp8"])
@pytest.mark.parametrize("case", AVG_CASES, ids=[f"{c[0]}-{c[4]}-t{c[6]}-f{c[7]}-W{c[5]}" for c in AVG_CASES])
def test_averaged_pipeline_equals_the_mean_of_the_oracle_images(B, ctx, case, arith):
    name, ns_total, fine, c, n_pix, W, ta, fa, pc, flags = case
    w, volt, freqs, fl = _case(name, ns_total, fine, flags)
    T, F = volt.shape[0] // 10, len(freqs) // c
    out = torch.full((T // ta, F // fa, n_pix, n_pix), float("nan"), dtype=torch.float32, device="cuda")
    B.blink_pipeline_averaged(ctx, B.Array(w["enu"], fl), B.Obs(freqs, c, 10, volt.shape[0]),
                              B.Imaging(n_pix, support=W, phase_centre=pc), arith, ta, fa, dev(volt), out)
    B.blink_sync(ctx)
    ref = oracle.pipeline(volt, w["enu"], freqs, 10, c, n_pix, flags=fl, n_threads=8, support=W, phase_centre=pc)
    imgs = ref["images"].reshape(T // ta, ta, F // fa, fa, n_pix, n_pix).mean(axis=(1, 3))
    got = out.cpu().numpy()
    for t in range(T // ta):
        for f in range(F // fa):
            assert_image_close(got[t, f], imgs[t, f], (t, f))


def test_band_average_equals_dedispersion_with_zero_delays(B, ctx):
    # the uv-plane band average against the image-plane one: blink_pipeline images, then blink_dedisperse
    # with zero delays (the mean over channels), on the same data
    w, volt, freqs, _ = _case("coarse", 30, 16)
    T, F, n = 3, 16, 256
    img = torch.empty((T * F, n, n), dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, B.Array(w["enu"]), B.Obs(freqs, 1, 10, 30), B.Imaging(n), 1, 0, dev(volt), img)
    band = torch.empty((T, n, n), dtype=torch.float32, device="cuda")
    B.blink_dedisperse(ctx, img, T, F, n, np.zeros(F, np.int32), band)
    avg = torch.empty((T, 1, n, n), dtype=torch.float32, device="cuda")
    B.blink_pipeline_averaged(ctx, B.Array(w["enu"]), B.Obs(freqs, 1, 10, 30), B.Imaging(n), 1, 1, F, dev(volt), avg)
    B.blink_sync(ctx)
    a, b = avg[:, 0].cpu().numpy(), band.cpu().numpy()
    for t in range(T):
        assert_image_close(a[t], b[t], t, rms_tol=1e-5)


def test_long_exposure_8192_on_sampled_pixels(B, ctx):
    # the paper's long-exposure product at its 8192 x 8192 side: four channels and two integrations averaged
    # into one image, checked on sampled pixels against the mean of the oracle's per-image pixels
    n = 8192
    w, volt, freqs, _ = _case("coarse", 20, 4)
    enu = w["enu"]
    out = torch.full((1, 1, n, n), float("nan"), dtype=torch.float32, device="cuda")
    B.blink_pipeline_averaged(ctx, B.Array(enu), B.Obs(freqs, 1, 10, 20), B.Imaging(n), 1, 2, 4, dev(volt), out)
    B.blink_sync(ctx)
    S = oracle.correlate(volt, 10, 1)
    nus = oracle.output_freqs(freqs, 1)
    du = oracle.default_cell(enu, float(nus.max()), n)
    rng = np.random.default_rng(81920)
    pts = [(n // 2, n // 2), (0, 0), (n - 1, n - 1)] + [(n // 2, x) for x in range(0, n, 211)]
    pts += [tuple(p) for p in rng.integers(0, n, size=(200, 2))]
    yx = np.array(pts, dtype=np.int32)
    want = np.zeros(len(yx))
    for t in range(2):
        for f in range(4):
            iu, iv, keep = oracle.cells(oracle.uvw(enu, float(nus[f])), du, n)
            G, Wsum = oracle.grid(S[t, f], enu.shape[0], 10, iu, iv, keep, n)
            want += oracle.image_pixels(G, Wsum, yx) / 8.0
            del G
    got = out[0, 0][torch.from_numpy(yx[:, 0]).long().cuda(), torch.from_numpy(yx[:, 1]).long().cuda()].cpu().numpy()
    scale = float(np.sqrt(np.mean(want ** 2)))
    err = np.abs(got.astype(np.float64) - want)
    print("8192 long exposure, sampled pixels: rel RMS", float(np.sqrt(np.mean(err ** 2))) / scale)
    assert np.sqrt(np.mean(err ** 2)) <= 1e-4 * scale
    assert err.max() <= 1e-3 * scale
