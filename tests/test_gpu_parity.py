"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Correlation and cell maps must match bit for bit; grids and images within the FP32 tolerances below
(images: relative RMS <= 1e-4 against the FP64 oracle, the precision gate of the method's mixed-precision
form, and max |diff| <= 1e-5 max |ref| pointwise; tests/imgcheck.py).  Sizes span several tiles and waves and include ragged ends.
"""
import numpy as np
import pytest

import blinksynth as bs
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from imgcheck import IMG_MAXTOL, IMG_RTOL, assert_image_close, image_errors  # noqa: F401  (shared gates)

GRID_RTOL = 2e-6         # max |diff| / max |G|, FP32 gridding sums of FP32 visibilities


def rel_rms(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2505_15204_gb300 import blink
    return blink


@pytest.fixture(scope="module")
def ctx(B):
    c = B.blink_create(0)
    yield c
    B.blink_destroy(c)


def _case(name, n_samples=None, fine=None, flags=False):
    w = bs.build_workload(name, n_samples=n_samples)
    volt, freqs = w["volt"], w["freqs"]
    if fine is not None:
        volt = np.ascontiguousarray(volt[:, :fine])
        freqs = freqs[:fine]
    fl = None
    if flags:
        fl = bs.tile_flags(w["enu"].shape[0], 0.15, w["workload"].seed, 99)
        fl[3] = 1
    return w, volt, freqs, fl


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# ---------------------------------------------------------------------------------------------------
# correlation
# ---------------------------------------------------------------------------------------------------

CORR_CASES = [
    ("tiny", None, None, 1, False),
    ("precision", None, None, 1, False),
    ("coarse", 30, 8, 4, False),        # 3 integrations x 2 output channels of 4 fine channels
    ("uneven", 20, 6, 2, True),         # flagged tiles
]


@pytest.mark.parametrize("arith", [0, 1], ids=["fp32", "fp8"])
@pytest.mark.parametrize("case", CORR_CASES, ids=[c[0] for c in CORR_CASES])
def test_correlate_bit_exact(B, ctx, case, arith):
    name, ns_total, fine, c, flags = case
    w, volt, freqs, fl = _case(name, ns_total, fine, flags)
    S = oracle.correlate(volt, 10, c, flags=fl)
    want = oracle.visibilities(S, 10 * c)
    T, F = S.shape[:2]
    out = torch.full(S.shape, float("nan"), dtype=torch.float32, device="cuda")
    B.blink_correlate(ctx, B.Array(w["enu"], fl), B.Obs(freqs, c, 10, volt.shape[0]), arith, dev(volt), out)
    B.blink_sync(ctx)
    got = out.cpu().numpy()
    assert np.array_equal(got[..., 0], want.real.astype(np.float32))
    assert np.array_equal(got[..., 1], want.imag.astype(np.float32))


def test_correlate_sub_band_with_fine_stride(B, ctx):
    # channels 4..11 of a 16-channel buffer: d_volt offset + fine_stride
    w, volt, freqs, _ = _case("coarse", 20, 16)
    S = oracle.correlate(np.ascontiguousarray(volt[:, 4:12]), 10, 2)
    want = oracle.visibilities(S, 20)
    d = dev(volt)
    out = torch.empty(S.shape, dtype=torch.float32, device="cuda")
    off = 4 * 128 * 2
    B.blink_correlate(ctx, B.Array(w["enu"]), B.Obs(freqs[4:12], 2, 10, 20, fine_stride=16), 0,
                      d.data_ptr() + off, out)
    B.blink_sync(ctx)
    got = out.cpu().numpy()
    assert np.array_equal(got[..., 0], want.real.astype(np.float32))


# ---------------------------------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------------------------------

def check_cells_and_uvw(B, ctx, name, n_pix, fine, c, flags, pc=(0.0, 0.0)):
    # off zenith: (u, v, w) on the pointing's basis and the default cell over the projected baselines
    w, volt, freqs, fl = _case(name, 10, fine, flags)
    arr = B.Array(w["enu"], fl)
    F = len(freqs) // c
    nb = B.blink_n_baselines(w["enu"].shape[0])
    cells = torch.empty((F, nb), dtype=torch.int32, device="cuda")
    uvw = torch.empty((F, nb, 3), dtype=torch.float64, device="cuda")
    du = B.blink_cells(ctx, arr, B.Obs(freqs, c, 10, 10), B.Imaging(n_pix, phase_centre=pc), cells, uvw)
    B.blink_sync(ctx)
    fout = oracle.output_freqs(freqs, c)
    du_ref = oracle.default_cell(w["enu"], fout.max(), n_pix, flags=fl, phase_centre=pc)
    assert du == du_ref
    got_c = cells.cpu().numpy().view(np.uint32)
    got_uvw = uvw.cpu().numpy()
    for f in range(F):
        uv = oracle.uvw_phased(w["enu"], fout[f], *pc)
        assert np.array_equal(got_uvw[f], uv)
        iu, iv, keep = oracle.cells(uv, du_ref, n_pix)
        if fl is not None:
            ij = np.array([(i, j) for i in range(len(fl)) for j in range(i + 1)])
            keep = keep & (fl[ij[:, 0]] == 0) & (fl[ij[:, 1]] == 0)
        want = np.where(keep.astype(bool), (iu.astype(np.uint32) & 0xFFFF) | (iv.astype(np.uint32) << 16),
                        np.uint32(0x80008000))
        assert np.array_equal(got_c[f], want)


@pytest.mark.parametrize("name,n_pix,fine,c,flags", [("tiny", 256, None, 1, False), ("precision", 512, None, 1, False),
                                                     ("coarse", 512, 128, 4, False), ("uneven", 1024, 8, 1, True)])
def test_cells_and_uvw_bit_exact(B, ctx, name, n_pix, fine, c, flags):
    check_cells_and_uvw(B, ctx, name, n_pix, fine, c, flags)


# ---------------------------------------------------------------------------------------------------
# gridding and imaging stages
# ---------------------------------------------------------------------------------------------------

def _half(G):
    n = G.shape[0]
    return G[:, : n // 2 + 1]


@pytest.mark.parametrize("pol", [0, 1], ids=["stokesI", "xx"])
def test_grid_matches_oracle(B, ctx, pol):
    w, volt, freqs, fl = _case("uneven", 20, 2, True)
    n_pix = 256
    arr, obs = B.Array(w["enu"], fl), B.Obs(freqs, 1, 10, 20)
    im = B.Imaging(n_pix, pol=pol)
    S = oracle.correlate(volt, 10, 1, flags=fl)
    vis = torch.empty(S.shape, dtype=torch.float32, device="cuda")
    B.blink_correlate(ctx, arr, obs, 0, dev(volt), vis)
    n_img = S.shape[0] * S.shape[1]
    grid = torch.empty((n_img, n_pix, n_pix // 2 + 1, 2), dtype=torch.float32, device="cuda")
    wts = torch.empty(n_img, dtype=torch.float32, device="cuda")
    B.blink_grid(ctx, arr, obs, im, vis, 0, n_img, grid, wts)
    B.blink_sync(ctx)
    ref = oracle.pipeline(volt, w["enu"], freqs, 10, 1, n_pix, flags=fl, pol=pol, want_grids=True)
    g = grid.cpu().numpy()
    g = g[..., 0] + 1j * g[..., 1]
    for q in range(n_img):
        h = _half(ref["grids"][q])
        assert np.abs(g[q] - h).max() <= GRID_RTOL * np.abs(h).max(), q
        assert wts[q].item() == ref["W"][q]


def test_image_stage_on_oracle_grid(B, ctx):
    w, volt, freqs, _ = _case("precision")
    for n_pix in (64, 256, 512, 1024, 2048):
        ref = oracle.pipeline(volt, w["enu"], freqs, 10, 1, n_pix, want_grids=True)
        h = _half(ref["grids"][0])
        g = np.stack([h.real, h.imag], axis=-1).astype(np.float32)[None]
        img = torch.empty((1, n_pix, n_pix), dtype=torch.float32, device="cuda")
        wt = torch.tensor([ref["W"][0]], dtype=torch.float32, device="cuda")
        B.blink_image(ctx, B.Imaging(n_pix), dev(g), 1, wt, img)
        B.blink_sync(ctx)
        assert_image_close(img[0].cpu().numpy(), ref["images"][0], n_pix, rms_tol=1e-5)


def test_image_stage_nyquist_column(B, ctx):
    # a grid whose only non-zero entries sit in the Nyquist column u = N/2 (allowed by the ABI layout)
    n = 64
    G = np.zeros((n, n), complex)
    G[5, n // 2] = 1 + 2j
    G[-5 % n, n // 2] = 1 - 2j
    a = np.fft.ifft2(G) * n * n
    want = np.roll(a.real, (n // 2, n // 2), axis=(0, 1))
    g = np.stack([G[:, : n // 2 + 1].real, G[:, : n // 2 + 1].imag], -1).astype(np.float32)[None]
    img = torch.empty((1, n, n), dtype=torch.float32, device="cuda")
    B.blink_image(ctx, B.Imaging(n), dev(g), 1, torch.ones(1, device="cuda"), img)
    B.blink_sync(ctx)
    assert np.abs(img[0].cpu().numpy() - want).max() < 1e-5


# ---------------------------------------------------------------------------------------------------
# the whole path
# ---------------------------------------------------------------------------------------------------

PIPE_CASES = [
    # name, n_samples, fine, chan_avg, n_pix, pol, autos, flags
    ("tiny", None, None, 1, 256, 0, 1, False),
    ("precision", None, None, 1, 256, 0, 1, False),
    ("precision", None, None, 1, 512, 0, 1, False),
    ("precision", None, None, 1, 1024, 0, 1, False),
    ("uneven", 20, 3, 1, 64, 1, 0, True),
    ("coarse", 20, 8, 4, 128, 0, 1, False),
    ("tiny", None, None, 1, 2048, 0, 1, False),
]


@pytest.mark.parametrize("arith", [0, 1], ids=["fp32", "fp8"])
@pytest.mark.parametrize("mode", [0, 1], ids=["batched", "plain"])
@pytest.mark.parametrize("case", PIPE_CASES, ids=[f"{c[0]}-{c[4]}-{c[2]}" for c in PIPE_CASES])
def test_pipeline_matches_oracle(B, ctx, case, mode, arith):
    name, ns_total, fine, c, n_pix, pol, autos, flags = case
    w, volt, freqs, fl = _case(name, ns_total, fine, flags)
    T = volt.shape[0] // 10
    F = len(freqs) // c
    img = torch.empty((T * F, n_pix, n_pix), dtype=torch.float32, device="cuda")
    wts = torch.empty(T * F, dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, B.Array(w["enu"], fl), B.Obs(freqs, c, 10, volt.shape[0]),
                     B.Imaging(n_pix, pol=pol, include_autos=autos), arith, mode, dev(volt), img, wts)
    B.blink_sync(ctx)
    ref = oracle.pipeline(volt, w["enu"], freqs, 10, c, n_pix, flags=fl, pol=pol, autos=bool(autos), n_threads=8)
    got = img.cpu().numpy()
    for q in range(T * F):
        assert_image_close(got[q], ref["images"][q], q)
        assert wts[q].item() == ref["W"][q]


def test_pipeline_many_waves_sampled(B, ctx):
    # 4 integrations x 128 channels = 512 images of 512^2: several waves; the oracle checks a sample
    w, volt, freqs, _ = _case("coarse", 40)
    n_pix = 512
    n = 4 * 128
    img = torch.empty((n, n_pix, n_pix), dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, B.Array(w["enu"]), B.Obs(freqs, 1, 10, 40), B.Imaging(n_pix), 0, 0, dev(volt), img)
    B.blink_sync(ctx)
    ids = np.array([0, 63, 64, 127, 255, 300, 511])
    ref = oracle.pipeline(volt, w["enu"], freqs, 10, 1, n_pix, ids=ids, n_threads=8)
    for k, q in enumerate(ids):
        assert_image_close(img[q].cpu().numpy(), ref["images"][k], q)


def test_pipeline_is_bitwise_reproducible(B, ctx):
    w, volt, freqs, _ = _case("coarse", 20, 16)
    outs = []
    for _ in range(2):
        img = torch.empty((32, 256, 256), dtype=torch.float32, device="cuda")
        B.blink_pipeline(ctx, B.Array(w["enu"]), B.Obs(freqs, 1, 10, 20), B.Imaging(256), 0, 0, dev(volt), img)
        B.blink_sync(ctx)
        outs.append(img.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_bf16_storage_error_is_reported(B, ctx):
    w, volt, freqs, _ = _case("precision")
    errs = {}
    for n_pix in (256, 512):
        img = torch.empty((1, n_pix, n_pix), dtype=torch.float32, device="cuda")
        B.blink_pipeline(ctx, B.Array(w["enu"]), B.Obs(freqs, 1, 10, 10), B.Imaging(n_pix, precision=1), 0, 0,
                         dev(volt), img)
        B.blink_sync(ctx)
        ref = oracle.pipeline(volt, w["enu"], freqs, 10, 1, n_pix)["images"][0]
        got = img[0].cpu().numpy()
        errs[n_pix] = (rel_rms(got, ref), float(np.abs(got - ref).max()))
    print("bf16 storage: rel RMS / max abs per side", errs)
    assert all(e[0] < 2e-2 for e in errs.values())


def test_pipeline_host_buffers_equal_device_path(B, ctx):
    w, volt, freqs, _ = _case("coarse", 20, 8)
    arr, obs, im = B.Array(w["enu"]), B.Obs(freqs, 1, 10, 20), B.Imaging(256)
    d = torch.empty((16, 256, 256), dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, arr, obs, im, 0, 0, dev(volt), d)
    h_volt = torch.from_numpy(volt).pin_memory()
    h_img = torch.empty((16, 256, 256), dtype=torch.float32).pin_memory()
    B.blink_pipeline_host(ctx, arr, obs, im, 0, h_volt, h_img, images_per_pass=5)
    B.blink_sync(ctx)
    assert np.array_equal(h_img.numpy(), d.cpu().numpy())


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("per_pass", [0, 3])
def test_pipeline_host_direct_and_staged_outputs(B, ctx, pinned, per_pass):
    # per_pass 0: images the device can write (page-locked, or pageable through the host page tables) are
    # written by the imaging kernel over the host link; per_pass 3: staged through device memory in passes.
    # Every form equals the device path bit for bit (FP8 correlation, 512^2)
    w, volt, freqs, _ = _case("coarse", 20, 8)
    arr, obs, im = B.Array(w["enu"]), B.Obs(freqs, 2, 10, 20), B.Imaging(512)
    n = 2 * (len(freqs) // 2)
    d = torch.empty((n, 512, 512), dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, arr, obs, im, 1, 0, dev(volt), d)
    h_volt = torch.from_numpy(volt)
    h_img = torch.full((n, 512, 512), float("nan"), dtype=torch.float32)
    if pinned:
        h_volt, h_img = h_volt.pin_memory(), h_img.pin_memory()
    B.blink_pipeline_host(ctx, arr, obs, im, 1, h_volt, h_img, images_per_pass=per_pass)
    B.blink_sync(ctx)
    assert np.array_equal(h_img.numpy(), d.cpu().numpy())


# ---------------------------------------------------------------------------------------------------
# edge cases and argument errors
# ---------------------------------------------------------------------------------------------------

def test_zero_samples_is_a_no_op(B, ctx):
    w, volt, freqs, _ = _case("tiny")
    out = torch.zeros(4, device="cuda")
    B.blink_pipeline(ctx, B.Array(w["enu"]), B.Obs(freqs, 1, 10, 0), B.Imaging(256), 0, 0, dev(volt), out)
    B.blink_correlate(ctx, B.Array(w["enu"]), B.Obs(freqs, 1, 10, 0), 0, dev(volt), out)
    B.blink_sync(ctx)
    assert not out.any()


def test_single_tile_and_all_flagged(B, ctx):
    # one tile: only its autocorrelation; all tiles flagged: an all-zero image with W = 0 treated as 1
    enu = np.zeros((1, 3))
    v = bs.constant_voltages(10, 1, 1, 2, -1)
    img = torch.empty((1, 64, 64), device="cuda")
    B.blink_pipeline(ctx, B.Array(enu), B.Obs(np.array([150e6]), 1, 10, 10), B.Imaging(64), 0, 0, dev(v), img)
    B.blink_sync(ctx)
    assert np.allclose(img[0].cpu().numpy(), 5.0)
    w, volt, freqs, _ = _case("tiny")
    fl = np.ones(128, np.uint8)
    img = torch.full((1, 256, 256), 7.0, device="cuda")
    B.blink_pipeline(ctx, B.Array(w["enu"], fl), B.Obs(freqs, 1, 10, 10), B.Imaging(256), 0, 0, dev(volt), img)
    B.blink_sync(ctx)
    assert not img.any()


@pytest.mark.parametrize("bad", ["n_pix", "chan_avg", "n_samples", "null"])
def test_invalid_arguments_are_rejected_before_launch(B, ctx, bad):
    w, volt, freqs, _ = _case("tiny")
    arr, obs, im = B.Array(w["enu"]), B.Obs(freqs, 1, 10, 10), B.Imaging(256)
    img = torch.zeros((1, 256, 256), device="cuda")
    d = dev(volt)
    if bad == "n_pix":
        im = B.Imaging(302)                 # 2 x 151: a prime factor above 5
    elif bad == "chan_avg":
        obs = B.Obs(freqs, 2, 10, 10)
    elif bad == "n_samples":
        obs = B.Obs(freqs, 1, 10, 15)
    else:
        d = None
    with pytest.raises(B.BlinkError) as e:
        B.blink_pipeline(ctx, arr, obs, im, 0, 0, d, img)
    assert e.value.status in (B.BLINK_ERR_INVALID_ARG, B.BLINK_ERR_UNSUPPORTED)
    B.blink_sync(ctx)
    assert not img.any()


def test_correlate_fp8_longer_integration_bit_exact(B, ctx):
    # K = 20 samples x 4 channels = 80: larger integer sums through the tensor-core accumulator
    w, volt, freqs, _ = _case("coarse", 40, 16)
    S = oracle.correlate(volt, 20, 4)
    want = oracle.visibilities(S, 80)
    out = torch.empty(S.shape, dtype=torch.float32, device="cuda")
    B.blink_correlate(ctx, B.Array(w["enu"]), B.Obs(freqs, 4, 20, 40), 1, dev(volt), out)
    B.blink_sync(ctx)
    got = out.cpu().numpy()
    assert np.array_equal(got[..., 0], want.real.astype(np.float32))
    assert np.array_equal(got[..., 1], want.imag.astype(np.float32))


def test_correlate_fp8_rejects_tile_count_not_multiple_of_8(B, ctx):
    enu = bs.tile_positions(12, 500.0, 3)
    v = bs.constant_voltages(10, 1, 12, 1, 1)
    out = torch.zeros((1, 1, 78, 4, 2), device="cuda")
    with pytest.raises(B.BlinkError) as e:
        B.blink_correlate(ctx, B.Array(enu), B.Obs(np.array([150e6]), 1, 10, 10), 1, dev(v), out)
    assert e.value.status == B.BLINK_ERR_UNSUPPORTED
    # the CUDA-core form handles it
    B.blink_correlate(ctx, B.Array(enu), B.Obs(np.array([150e6]), 1, 10, 10), 0, dev(v), out)
    B.blink_sync(ctx)
    assert np.all(out.cpu().numpy()[..., 0] == 2.0)


# ---------------------------------------------------------------------------------------------------
# several channel sets with their own flags and image sizes; CUDA graph capture
# ---------------------------------------------------------------------------------------------------

def test_pipeline_sets_uneven_flags_and_sizes(B, ctx):
    # the uneven workload: 4 coarse channels, each with its own flagged tiles and image side; 8 fine
    # channels of each coarse channel and one integration keep the oracle quick
    w = bs.build_workload("uneven", n_samples=10)
    volt, freqs, sets_w = w["volt"], w["freqs"], w["sets"]
    sets = [B.Set(fine0=st.fine0, n_fine=8, imaging=B.Imaging(st.n_pix), flags=st.flags) for st in sets_w]
    assert sorted({st.n_pix for st in sets_w}) == [256, 512, 1024]
    assert len({int(st.flags.sum()) for st in sets_w}) > 1
    total = sum(8 * st.n_pix ** 2 for st in sets_w)
    img = torch.full((total,), float("nan"), dtype=torch.float32, device="cuda")
    B.blink_pipeline_sets(ctx, B.Array(w["enu"]), B.Obs(freqs, 1, 10, 10), sets, 1, dev(volt), img, total)
    B.blink_sync(ctx)
    got = img.cpu().numpy()
    at = 0
    for st in sets_w:
        n = st.n_pix
        ref = oracle.pipeline(volt, w["enu"], freqs, 10, 1, n, flags=st.flags, fine0=st.fine0, n_fine=8, n_threads=8)
        part = got[at:at + 8 * n * n].reshape(8, n, n)
        for q in range(8):
            assert_image_close(part[q], ref["images"][q], (st.fine0, q))
        at += 8 * n * n
    with pytest.raises(B.BlinkError):
        B.blink_pipeline_sets(ctx, B.Array(w["enu"]), B.Obs(freqs, 1, 10, 10), sets, 1, dev(volt), img, total - 1)


def test_pipeline_replays_in_a_cuda_graph(B, ctx):
    w, volt, freqs, _ = _case("coarse", 20, 16)
    arr, obs, im = B.Array(w["enu"]), B.Obs(freqs, 1, 10, 20), B.Imaging(256)
    d = dev(volt)
    eager = torch.empty((32, 256, 256), dtype=torch.float32, device="cuda")
    out = torch.zeros((32, 256, 256), dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        B.blink_pipeline(ctx, arr, obs, im, 1, 0, d, eager, stream=s)      # plan and workspace on first use
        B.blink_pipeline(ctx, arr, obs, im, 1, 0, d, out, stream=s)
    s.synchronize()
    out.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        B.blink_pipeline(ctx, arr, obs, im, 1, 0, d, out, stream=s)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    B.blink_sync(ctx)
    assert torch.equal(out, eager)


def test_pipeline_sets_replays_in_a_cuda_graph(B, ctx):
    # the uneven form as one graph: every set's correlation and persistent FFT launch captured together
    w = bs.build_workload("uneven", n_samples=20)
    volt, freqs, sets_w = w["volt"], w["freqs"], w["sets"]
    sets = [B.Set(fine0=st.fine0, n_fine=16, imaging=B.Imaging(st.n_pix), flags=st.flags) for st in sets_w]
    total = sum(2 * 16 * st.n_pix ** 2 for st in sets_w)
    arr, obs, d = B.Array(w["enu"]), B.Obs(freqs, 1, 10, 20), dev(volt)
    eager = torch.empty(total, dtype=torch.float32, device="cuda")
    out = torch.zeros(total, dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        B.blink_pipeline_sets(ctx, arr, obs, sets, 1, d, eager, total, stream=s)   # plans, tuning, workspace
        B.blink_pipeline_sets(ctx, arr, obs, sets, 1, d, out, total, stream=s)
    s.synchronize()
    out.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        B.blink_pipeline_sets(ctx, arr, obs, sets, 1, d, out, total, stream=s)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    B.blink_sync(ctx)
    assert torch.equal(out, eager)


# ---------------------------------------------------------------------------------------------------
# calibration gains inside the correlation (diagonal Jones per output channel, tile and polarisation)
# ---------------------------------------------------------------------------------------------------

def _gains(F, n_tiles, seed):
    rng = np.random.default_rng(seed)
    g = rng.uniform(0.5, 1.5, size=(F, n_tiles, 2)) * np.exp(1j * rng.uniform(-np.pi, np.pi, size=(F, n_tiles, 2)))
    return g.astype(np.complex64)                      # the values both sides use


@pytest.mark.parametrize("arith", [0, 1])
def test_correlate_with_gains_matches_oracle(B, ctx, arith):
    w, volt, freqs, fl = _case("coarse", 20, 8, flags=True)
    F, K = 4, 20                                       # 8 fine channels averaged by 2, 10 samples per integration
    g = _gains(F, 128, 5)
    out = torch.empty((2, F, 8256, 4, 2), dtype=torch.float32, device="cuda")
    B.blink_correlate(ctx, B.Array(w["enu"], fl, g), B.Obs(freqs, 2, 10, 20), arith, dev(volt), out)
    B.blink_sync(ctx)
    got = out.cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    S = oracle.correlate(volt, 10, 2, flags=fl)
    for tau in range(2):
        for f in range(F):
            ref = oracle.apply_gains(S[tau, f], g[f].astype(np.complex128)) / K
            err = np.abs(got[tau, f] - ref).max() / np.abs(ref).max()
            assert err <= 2e-6, (arith, tau, f, err)


@pytest.mark.parametrize("arith,mode,pol", [(1, 0, 0), (0, 0, 0), (1, 0, 1), (1, 1, 0)])
def test_pipeline_with_gains_matches_oracle(B, ctx, arith, mode, pol):
    # Stokes I with gains takes the split XX / YY tensor-core chains; XX one chain; plain mode per image
    w, volt, freqs, fl = _case("coarse", 20, 8, flags=True)
    F, n = 8, 256
    g = _gains(F, 128, 6)
    img = torch.empty((2 * F, n, n), dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, B.Array(w["enu"], fl, g), B.Obs(freqs, 1, 10, 20), B.Imaging(n, pol=pol), arith, mode,
                     dev(volt), img)
    B.blink_sync(ctx)
    ref = oracle.pipeline(volt, w["enu"], freqs, 10, 1, n, flags=fl, pol=pol, gains=g.astype(np.complex128),
                          n_threads=8)["images"]
    got = img.cpu().numpy()
    for q in range(2 * F):
        assert_image_close(got[q], ref[q], (q, rel_rms(got[q], ref[q])))


@pytest.mark.parametrize("arith", [0, 1])
def test_unit_gains_equal_no_gains_bit_for_bit(B, ctx, arith):
    w, volt, freqs, _ = _case("coarse", 20, 8)
    n = 256
    a = torch.empty((16, n, n), dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    obs, im = B.Obs(freqs, 1, 10, 20), B.Imaging(n)
    B.blink_pipeline(ctx, B.Array(w["enu"]), obs, im, arith, 0, dev(volt), a)
    B.blink_pipeline(ctx, B.Array(w["enu"], None, np.ones((8, 128, 2), np.complex64)), obs, im, arith, 0, dev(volt), b)
    B.blink_sync(ctx)
    assert torch.equal(a, b)


def test_pipeline_sets_with_gains(B, ctx):
    w = bs.build_workload("uneven", n_samples=10)
    volt, freqs, sets_w = w["volt"], w["freqs"], w["sets"]
    g = _gains(len(freqs), 144, 7)                     # one row per output channel of the call (chan_avg 1)
    sets = [B.Set(fine0=st.fine0, n_fine=8, imaging=B.Imaging(st.n_pix), flags=st.flags) for st in sets_w]
    total = sum(8 * st.n_pix ** 2 for st in sets_w)
    img = torch.empty(total, dtype=torch.float32, device="cuda")
    B.blink_pipeline_sets(ctx, B.Array(w["enu"], None, g), B.Obs(freqs, 1, 10, 10), sets, 1, dev(volt), img, total)
    B.blink_sync(ctx)
    got = img.cpu().numpy()
    at = 0
    for st in sets_w:
        n = st.n_pix
        ref = oracle.pipeline(volt, w["enu"], freqs, 10, 1, n, flags=st.flags, fine0=st.fine0, n_fine=8, n_threads=8,
                              gains=g[st.fine0:st.fine0 + 8].astype(np.complex128))
        part = got[at:at + 8 * n * n].reshape(8, n, n)
        for q in range(8):
            assert_image_close(part[q], ref["images"][q], (st.fine0, q))
        at += 8 * n * n


# ---------------------------------------------------------------------------------------------------
# incoherent dedispersion of the image cube
# ---------------------------------------------------------------------------------------------------

def test_dedisperse_matches_oracle(B, ctx):
    rng = np.random.default_rng(31)
    T, F, n = 9, 13, 64                                # F not a multiple of the kernel's unroll
    img = rng.normal(size=(T, F, n, n)).astype(np.float32)
    d = np.array([0, 3, 1, 4, 2, 0, 1, 4, 3, 2, 0, 1, 2], dtype=np.int32)
    out = torch.empty((T - 4, n, n), dtype=torch.float32, device="cuda")
    B.blink_dedisperse(ctx, dev(img), T, F, n, d, out)
    B.blink_sync(ctx)
    ref = oracle.dedisperse(img.astype(np.float64), d)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()


def test_dedispersed_pipeline_images_match_oracle(B, ctx):
    # images of 4 integrations x 8 channels, then a dedispersion over their channels, against the oracle's
    w, volt, freqs, _ = _case("coarse", 40, 8)
    n, T, F = 128, 4, 8
    img = torch.empty((T * F, n, n), dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, B.Array(w["enu"]), B.Obs(freqs, 1, 10, 40), B.Imaging(n), 1, 0, dev(volt), img)
    d = np.array([2, 2, 1, 1, 1, 0, 0, 0], dtype=np.int32)
    out = torch.empty((T - 2, n, n), dtype=torch.float32, device="cuda")
    B.blink_dedisperse(ctx, img, T, F, n, d, out)
    B.blink_sync(ctx)
    ref_img = oracle.pipeline(volt, w["enu"], freqs, 10, 1, n, n_threads=8)["images"].reshape(T, F, n, n)
    ref = oracle.dedisperse(ref_img, d)
    got = out.cpu().numpy()
    for t in range(T - 2):
        assert_image_close(got[t], ref[t])


def test_dedisperse_rejects_bad_delays(B, ctx):
    img = torch.zeros((4, 2, 64, 64), dtype=torch.float32, device="cuda")
    out = torch.zeros((4, 64, 64), dtype=torch.float32, device="cuda")
    for d in ([0, 4], [-1, 0]):
        with pytest.raises(B.BlinkError):
            B.blink_dedisperse(ctx, img, 4, 2, 64, np.array(d, np.int32), out)


def _jones(F, n_tiles, seed):
    rng = np.random.default_rng(seed)
    J = (np.eye(2) + 0.3 * (rng.normal(size=(F, n_tiles, 2, 2)) + 1j * rng.normal(size=(F, n_tiles, 2, 2))))
    return J.astype(np.complex64)                      # leakage of about 30 %


@pytest.mark.parametrize("arith", [0, 1])
def test_correlate_with_jones_matches_oracle(B, ctx, arith):
    w, volt, freqs, fl = _case("coarse", 20, 8, flags=True)
    F, K = 4, 20
    J = _jones(F, 128, 8)
    out = torch.empty((2, F, 8256, 4, 2), dtype=torch.float32, device="cuda")
    B.blink_correlate(ctx, B.Array(w["enu"], fl, None, J), B.Obs(freqs, 2, 10, 20), arith, dev(volt), out)
    B.blink_sync(ctx)
    got = out.cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    S = oracle.correlate(volt, 10, 2, flags=fl)
    for tau in range(2):
        for f in range(F):
            ref = oracle.apply_jones(S[tau, f], J[f].astype(np.complex128)) / K
            err = np.abs(got[tau, f] - ref).max() / np.abs(ref).max()
            assert err <= 2e-6, (arith, tau, f, err)


@pytest.mark.parametrize("arith,pol", [(1, 0), (0, 0), (1, 1)])
def test_pipeline_with_jones_matches_oracle(B, ctx, arith, pol):
    w, volt, freqs, fl = _case("coarse", 20, 8, flags=True)
    F, n = 8, 256
    J = _jones(F, 128, 9)
    img = torch.empty((2 * F, n, n), dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, B.Array(w["enu"], fl, None, J), B.Obs(freqs, 1, 10, 20), B.Imaging(n, pol=pol), arith, 0,
                     dev(volt), img)
    B.blink_sync(ctx)
    ref = oracle.pipeline(volt, w["enu"], freqs, 10, 1, n, flags=fl, pol=pol, gains=J.astype(np.complex128),
                          n_threads=8)["images"]
    got = img.cpu().numpy()
    for q in range(2 * F):
        assert_image_close(got[q], ref[q], (q, rel_rms(got[q], ref[q])))


def test_diagonal_jones_images_equal_gains_images(B, ctx):
    # the four-product Jones kernel and the split-chain gains kernel agree to FP32 rounding
    w, volt, freqs, _ = _case("coarse", 20, 8)
    n = 256
    g = _gains(8, 128, 10)
    J = np.zeros((8, 128, 2, 2), np.complex64)
    J[..., 0, 0], J[..., 1, 1] = g[..., 0], g[..., 1]
    a = torch.empty((16, n, n), dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    obs, im = B.Obs(freqs, 1, 10, 20), B.Imaging(n)
    B.blink_pipeline(ctx, B.Array(w["enu"], None, g), obs, im, 1, 0, dev(volt), a)
    B.blink_pipeline(ctx, B.Array(w["enu"], None, None, J), obs, im, 1, 0, dev(volt), b)
    B.blink_sync(ctx)
    for q in range(16):
        assert_image_close(b[q].cpu().numpy(), a[q].cpu().numpy(), q, rms_tol=1e-6)


# ---------------------------------------------------------------------------------------------------
# gridding with a Kaiser-Bessel convolution kernel (grid of side 2N, central N x N corrected image)
# ---------------------------------------------------------------------------------------------------

KB_CASES = [
    # name, n_samples, fine, chan_avg, n_pix, pol, autos, flags, support
    ("tiny", None, None, 1, 256, 0, 1, False, 6),          # grid 512: two-row radix-16 row pass
    ("precision", None, None, 1, 512, 0, 1, False, 4),     # grid 1024: generic row pass
    ("coarse", 20, 8, 4, 128, 0, 1, False, 8),             # grid 256: several images per channel
    ("uneven", 20, 3, 1, 64, 1, 0, True, 2),               # grid 128: zeroed columns, XX, no autos, flags
    ("tiny", None, None, 1, 1024, 0, 1, False, 6),         # grid 2048
    ("uneven", 20, 3, 1, 256, 1, 0, True, 6),              # grid 512, separable list: XX, no autos, flags
    ("precision", None, None, 1, 512, 0, 1, False, 8),     # grid 1024, separable list: eight row weights
]


@pytest.mark.parametrize("arith", [0, 1], ids=["fp32", "fp8"])
@pytest.mark.parametrize("case", KB_CASES, ids=[f"{c[0]}-{c[4]}-W{c[8]}" for c in KB_CASES])
def test_kb_pipeline_matches_oracle(B, ctx, case, arith):
    name, ns_total, fine, c, n_pix, pol, autos, flags, W = case
    w, volt, freqs, fl = _case(name, ns_total, fine, flags)
    T = volt.shape[0] // 10
    F = len(freqs) // c
    img = torch.full((T * F, n_pix, n_pix), float("nan"), dtype=torch.float32, device="cuda")
    wts = torch.empty(T * F, dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, B.Array(w["enu"], fl), B.Obs(freqs, c, 10, volt.shape[0]),
                     B.Imaging(n_pix, pol=pol, include_autos=autos, support=W), arith, 0, dev(volt), img, wts)
    B.blink_sync(ctx)
    ref = oracle.pipeline(volt, w["enu"], freqs, 10, c, n_pix, flags=fl, pol=pol, autos=bool(autos), n_threads=8,
                          support=W)
    got = img.cpu().numpy()
    for q in range(T * F):
        assert_image_close(got[q], ref["images"][q], q)
        assert wts[q].item() == ref["W"][q]


def test_kb_pipeline_with_gains_and_sets(B, ctx):
    # calibrated Stokes I with a kernel, in a sets call next to a nearest-cell set (packed outputs of two
    # image sides)
    w, volt, freqs, fl = _case("coarse", 20, 8, flags=True)
    g = _gains(8, 128, 8)
    sets = [B.Set(0, 4, B.Imaging(256, support=4), flags=fl), B.Set(4, 4, B.Imaging(128))]
    total = 2 * 4 * 256 * 256 + 2 * 4 * 128 * 128
    img = torch.full((total,), float("nan"), dtype=torch.float32, device="cuda")
    B.blink_pipeline_sets(ctx, B.Array(w["enu"], None, g), B.Obs(freqs, 1, 10, 20), sets, 1, dev(volt), img, total)
    B.blink_sync(ctx)
    got = img.cpu().numpy()
    ref0 = oracle.pipeline(volt, w["enu"], freqs, 10, 1, 256, flags=fl, fine0=0, n_fine=4, support=4,
                           gains=g[0:4].astype(np.complex128), n_threads=8)["images"]
    ref1 = oracle.pipeline(volt, w["enu"], freqs, 10, 1, 128, fine0=4, n_fine=4,
                           gains=g[4:8].astype(np.complex128), n_threads=8)["images"]
    part0 = got[:8 * 256 * 256].reshape(8, 256, 256)
    part1 = got[8 * 256 * 256:].reshape(8, 128, 128)
    for q in range(8):
        assert_image_close(part0[q], ref0[q], q)
        assert_image_close(part1[q], ref1[q], q)


@pytest.mark.parametrize("per_pass", [0, 3])
def test_kb_pipeline_host_equals_device_path(B, ctx, per_pass):
    w, volt, freqs, _ = _case("coarse", 20, 8)
    arr, obs, im = B.Array(w["enu"]), B.Obs(freqs, 2, 10, 20), B.Imaging(256, support=6)
    d = torch.empty((8, 256, 256), dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, arr, obs, im, 1, 0, dev(volt), d)
    h_volt = torch.from_numpy(volt).pin_memory()
    h_img = torch.full((8, 256, 256), float("nan"), dtype=torch.float32).pin_memory()
    B.blink_pipeline_host(ctx, arr, obs, im, 1, h_volt, h_img, images_per_pass=per_pass)
    B.blink_sync(ctx)
    assert np.array_equal(h_img.numpy(), d.cpu().numpy())


# ---------------------------------------------------------------------------------------------------
# the fused launch (correlation inside the persistent imaging kernel)
# ---------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n_tiles,c,flags,pol", [(144, 1, False, 0), (144, 4, True, 0), (128, 2, False, 1),
                                                 (136, 1, True, 1)])
def test_fused_launch_equals_two_launches_and_the_oracle(B, ctx, n_tiles, c, flags, pol):
    # one persistent launch per call correlates each image's integration on the tensor cores (sums kept in an
    # L2 ring in gather order) and grids and transforms it: the same images, bit for bit, as the correlator
    # launch followed by the imaging launch, and within the image gates of the FP64 oracle
    enu = bs.tile_positions(n_tiles, 3000.0, 71)
    freqs = 155e6 + 10e3 * np.arange(8 * c)
    sky = bs.Sky(lmn=np.array([[0.05, -0.08, np.sqrt(1 - 0.0089)], [-0.2, 0.1, np.sqrt(1 - 0.05)]]),
                 power=np.array([2.0, 1.5]))
    ns = 30
    v = bs.voltages(enu, freqs, ns, sky, seed=72)
    fl = bs.tile_flags(n_tiles, 0.15, 73, 1) if flags else None
    arr, obs = B.Array(enu, fl), B.Obs(freqs, c, 10, ns)
    im = B.Imaging(512, pol=pol)
    n = 3 * 8
    fused = torch.full((n, 512, 512), float("nan"), dtype=torch.float32, device="cuda")
    split = torch.full_like(fused, float("nan"))
    d = dev(v)
    B.blink_set_fused(ctx, True)
    try:
        B.blink_pipeline(ctx, arr, obs, im, B.BLINK_CORR_FP8, B.BLINK_MODE_BATCHED, d, fused)    # plan and tuning
        B.blink_read_profile(ctx, reset=True)
        B.blink_set_profiling(ctx, True)
        B.blink_pipeline(ctx, arr, obs, im, B.BLINK_CORR_FP8, B.BLINK_MODE_BATCHED, d, fused)
        B.blink_sync(ctx)
        B.blink_set_profiling(ctx, False)
        ms, launches = B.blink_read_profile(ctx, reset=True)
        assert launches[B.BLINK_STAGE_FUSED] == 1 and launches[B.BLINK_STAGE_CORRELATE] == 0, launches
    finally:
        B.blink_set_fused(ctx, False)
    B.blink_pipeline(ctx, arr, obs, im, B.BLINK_CORR_FP8, B.BLINK_MODE_BATCHED, d, split)
    B.blink_sync(ctx)
    assert torch.equal(fused, split)
    ids = np.array([0, 5, n - 1])
    kw = {"flags": fl} if flags else {}
    ref = oracle.pipeline(v, enu, freqs, 10, c, 512, ids=ids, pol=pol, n_threads=8, **kw)["images"]
    got = fused[torch.from_numpy(ids).cuda()].cpu().numpy()
    for k, q in enumerate(ids):
        assert_image_close(got[k], ref[k], (n_tiles, c, q))
