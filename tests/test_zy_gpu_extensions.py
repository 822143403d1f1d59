"""Parity of the next-row extensions of the path with the CPU oracle (GPU): the phase centre on an
off-zenith pointing, long integrations on both correlators, dedispersion recovering an injected
dispersion measure, and the reproducibility and BF16 storage of gridding with a kernel.

The file sorts after the core parity suite so that a failure here, under ``-x``, leaves the core results
reported.  Helpers come from ``test_gpu_parity``.
"""
import numpy as np
import pytest

import blinksynth as bs
import oracle

from test_gpu_parity import IMG_RTOL, B, _case, _gains, check_cells_and_uvw, ctx, dev, rel_rms  # noqa: F401
from imgcheck import assert_image_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


# ---------------------------------------------------------------------------------------------------
# long integrations
# ---------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n_tiles,ns,c,const", [(16, 200, 4, False), (8, 10000, 4, False), (8, 10000, 4, True)])
def test_long_integrations_exact_on_both_correlators(B, ctx, n_tiles, ns, c, const):
    # K = 800 and 40,000 (20 ms and 1 s of 10 kHz channels averaged by 4): both forms stay bit-exact, the
    # tensor-core one streaming K through its operand tiles in chunks that accumulate in TMEM (|S| <= 128 K
    # < 2^24, reached by constant -8 - 8i voltages)
    enu = bs.tile_positions(n_tiles, 1500.0, 51)
    freqs = 155e6 + 10e3 * np.arange(c)
    if const:
        v = bs.constant_voltages(ns, c, n_tiles, -8, -8)
    else:
        sky = bs.Sky(lmn=np.array([[0.1, 0.05, np.sqrt(1 - 0.0125)]]), power=np.array([4.0]))
        v = bs.voltages(enu, freqs, ns, sky, seed=52)
    S = oracle.correlate(v, ns, c)
    want = oracle.visibilities(S, ns * c)
    if const:
        assert np.all(S[..., 0, 0] == ns * c * 128)
    arr, obs = B.Array(enu), B.Obs(freqs, c, ns, ns)
    for arith in (B.BLINK_CORR_FP32, B.BLINK_CORR_FP8):
        out = torch.full(S.shape, float("nan"), dtype=torch.float32, device="cuda")
        B.blink_correlate(ctx, arr, obs, arith, dev(v), out)
        B.blink_sync(ctx)
        got = out.cpu().numpy()
        assert np.array_equal(got[..., 0], want.real.astype(np.float32)), arith
        assert np.array_equal(got[..., 1], want.imag.astype(np.float32)), arith


@pytest.mark.parametrize("ns,c", [(200, 4), (2000, 4)])
def test_long_integration_images_on_the_tensor_core_form(B, ctx, ns, c):
    # Stokes-I images of 144 tiles at K = 800 and 8,000 through the batched FP8 path (gather-ordered sums,
    # K streamed in chunks), against the FP64 oracle
    w, volt, freqs, _ = _case("precision")
    enu = w["enu"]
    freqs = 155e6 + 10e3 * np.arange(2 * c)
    sky = bs.Sky(lmn=np.array([[0.05, -0.08, np.sqrt(1 - 0.0089)]]), power=np.array([2.0]))
    v = bs.voltages(enu, freqs, ns, sky, seed=61)
    ref = oracle.pipeline(v, enu, freqs, ns, c, 512, n_threads=8)["images"]
    img = torch.empty((2, 512, 512), dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, B.Array(enu), B.Obs(freqs, c, ns, ns), B.Imaging(512), B.BLINK_CORR_FP8,
                     B.BLINK_MODE_BATCHED, dev(v), img)
    B.blink_sync(ctx)
    got = img.cpu().numpy()
    for q in range(2):
        assert_image_close(got[q], ref[q], q)


# ---------------------------------------------------------------------------------------------------
# dedispersion of imaged voltages
# ---------------------------------------------------------------------------------------------------

def test_dedispersion_recovers_the_injected_dispersion_measure(B, ctx):
    # a dispersed 1 ms burst (DM 500) imaged by the path and dedispersed by blink_dedisperse at trial DMs: the
    # phase-centre peak is largest at DM 500, and the DM-500 cube equals the oracle's within the image gate
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location("pins", os.path.join(os.path.dirname(__file__), "test_oracle_pins.py"))
    pins = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(pins)
    enu, freqs, volt = pins._dispersed_burst_case()
    T, F, n = 400, 8, 64
    img = torch.empty((T * F, n, n), dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, B.Array(enu), B.Obs(freqs, 1, 10, 4000), B.Imaging(n), 1, 0, dev(volt), img)
    peaks, out500 = {}, None
    for dm in range(0, 1001, 100):
        d = pins._delays(freqs, dm)
        out = torch.empty((T - int(d.max()), n, n), dtype=torch.float32, device="cuda")
        B.blink_dedisperse(ctx, img, T, F, n, d, out)
        B.blink_sync(ctx)
        peaks[dm] = float(out[:, n // 2, n // 2].max())
        if dm == 500:
            out500 = out.cpu().numpy()
    assert max(peaks, key=peaks.get) == 500, peaks
    ref_img = oracle.pipeline(volt, enu, freqs, 10, 1, n, n_threads=8)["images"].reshape(T, F, n, n)
    ref = oracle.dedisperse(ref_img, pins._delays(freqs, 500))
    assert_image_close(out500, ref)


# ---------------------------------------------------------------------------------------------------
# gridding with a kernel: reproducibility and BF16 storage
# ---------------------------------------------------------------------------------------------------

def test_kb_pipeline_is_bitwise_reproducible_and_bf16_error_is_reported(B, ctx):
    # fixed summation order with a kernel too; BF16 storage of the 2N grid and ring is reported, not gated
    w, volt, freqs, _ = _case("coarse", 20, 8)
    arr, obs = B.Array(w["enu"]), B.Obs(freqs, 1, 10, 20)
    outs = []
    for _ in range(2):
        img = torch.empty((16, 256, 256), dtype=torch.float32, device="cuda")
        B.blink_pipeline(ctx, arr, obs, B.Imaging(256, support=6), 1, 0, dev(volt), img)
        B.blink_sync(ctx)
        outs.append(img.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    img = torch.empty((16, 256, 256), dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, arr, obs, B.Imaging(256, support=6, precision=1), 1, 0, dev(volt), img)
    B.blink_sync(ctx)
    ref = oracle.pipeline(volt, w["enu"], freqs, 10, 1, 256, ids=np.array([0, 15]), support=6, n_threads=8)["images"]
    got = img.cpu().numpy()
    errs = [rel_rms(got[q], ref[k]) for k, q in enumerate((0, 15))]
    print("bf16 storage with a kernel: rel RMS", errs)
    assert max(errs) < 5e-2             # a sanity bound (BF16 storage is ~5e-3 at 512^2; the correction enlarges the edges')


# ---------------------------------------------------------------------------------------------------
# phase centre on an off-zenith pointing (geometric corrections)
# ---------------------------------------------------------------------------------------------------

PC_CASES = [
    # name, n_samples, fine, chan_avg, n_pix, support, pointing, mode
    ("coarse", 20, 8, 4, 256, 0, (0.31, -0.22), 0),
    ("precision", None, None, 1, 512, 0, (-0.05, 0.4), 0),
    ("uneven", 20, 3, 1, 128, 0, (0.2, 0.1), 1),
    ("uneven", 20, 2, 1, 1024, 0, (-0.15, 0.25), 0),
    ("coarse", 20, 8, 2, 128, 6, (0.31, -0.22), 0),
]


@pytest.mark.parametrize("arith", [0, 1], ids=["fp32", "fp8"])
@pytest.mark.parametrize("case", PC_CASES, ids=[f"{c[0]}-{c[4]}-W{c[5]}-{'plain' if c[7] else 'batched'}" for c in PC_CASES])
def test_phase_centred_pipeline_matches_oracle(B, ctx, case, arith):
    name, ns_total, fine, c, n_pix, W, pc, mode = case
    w, volt, freqs, fl = _case(name, ns_total, fine, name == "uneven")
    T = volt.shape[0] // 10
    F = len(freqs) // c
    img = torch.full((T * F, n_pix, n_pix), float("nan"), dtype=torch.float32, device="cuda")
    wts = torch.empty(T * F, dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, B.Array(w["enu"], fl), B.Obs(freqs, c, 10, volt.shape[0]),
                     B.Imaging(n_pix, support=W, phase_centre=pc), arith, mode, dev(volt), img, wts)
    B.blink_sync(ctx)
    ref = oracle.pipeline(volt, w["enu"], freqs, 10, c, n_pix, flags=fl, n_threads=8, support=W, phase_centre=pc)
    got = img.cpu().numpy()
    for q in range(T * F):
        assert_image_close(got[q], ref["images"][q], q)
        assert wts[q].item() == ref["W"][q]


def test_source_at_the_pointing_images_at_the_centre_pixel(B, ctx):
    enu = bs.tile_positions(48, 1500.0, 44)
    nu, n = 154.88e6, 128
    l0, m0 = 0.02, -0.015
    sky = bs.Sky(lmn=np.array([[l0, m0, np.sqrt(1 - l0 * l0 - m0 * m0)]]), power=np.array([20.0]))
    v = bs.voltages(enu, np.array([nu]), 40, sky, seed=43, sigma=0.0)
    img = torch.empty((1, n, n), dtype=torch.float32, device="cuda")
    B.blink_pipeline(ctx, B.Array(enu), B.Obs(np.array([nu]), 1, 40, 40), B.Imaging(n, phase_centre=(l0, m0)), 1,
                     0, dev(v), img)
    B.blink_sync(ctx)
    got = img[0].cpu().numpy()
    assert np.unravel_index(np.argmax(got), got.shape) == (n // 2, n // 2)


TRACK_CASES = [
    # name, n_samples, fine, chan_avg, n_pix, support, one pointing per integration
    ("coarse", 40, 8, 2, 256, 0, [(0.1, 0.05), (0.1, 0.05), (0.12, 0.04), (-0.2, 0.3)]),
    ("uneven", 30, 3, 1, 128, 0, [(0.0, 0.0), (0.3, -0.1), (0.0, 0.0)]),
    ("coarse", 20, 8, 2, 128, 6, [(0.31, -0.22), (0.29, -0.2)]),
]


@pytest.mark.parametrize("arith", [0, 1], ids=["fp32", "fp8"])
@pytest.mark.parametrize("case", TRACK_CASES, ids=[f"{c[0]}-{c[4]}-W{c[5]}" for c in TRACK_CASES])
def test_tracking_pipeline_matches_the_oracle_one_pointing_at_a_time(B, ctx, case, arith):
    # each integration against the oracle imaged on that integration's pointing, with the pixel scale fixed
    # by the first pointing (the entry point's default cell)
    name, ns_total, fine, c, n_pix, W, lm = case
    w, volt, freqs, fl = _case(name, ns_total, fine, name == "uneven")
    T, F = volt.shape[0] // 10, len(freqs) // c
    assert len(lm) == T
    img = torch.full((T * F, n_pix, n_pix), float("nan"), dtype=torch.float32, device="cuda")
    B.blink_pipeline_tracking(ctx, B.Array(w["enu"], fl), B.Obs(freqs, c, 10, volt.shape[0]),
                              B.Imaging(n_pix, support=W), np.array(lm), arith, dev(volt), img)
    B.blink_sync(ctx)
    nu_max = float(np.max(oracle.output_freqs(freqs, c)))
    du = oracle.default_cell(w["enu"], nu_max, n_pix, fl, W, lm[0])
    got = img.cpu().numpy()
    for t in range(T):
        ids = np.arange(t * F, (t + 1) * F)
        ref = oracle.pipeline(volt, w["enu"], freqs, 10, c, n_pix, ids=ids, flags=fl, n_threads=8, support=W,
                              phase_centre=lm[t], cell_lambda=du)
        for f in range(F):
            assert_image_close(got[t * F + f], ref["images"][f], (t, f))


def test_tracking_pipeline_rejects_a_pointing_off_the_sky(B, ctx):
    w, volt, freqs, fl = _case("coarse", 20, 8, False)
    img = torch.empty((8, 128, 128), dtype=torch.float32, device="cuda")
    for lm in ([(0.1, 0.0), (0.8, 0.7)], [(0.1, 0.0), (float("nan"), 0.0)]):
        with pytest.raises(B.BlinkError) as e:
            B.blink_pipeline_tracking(ctx, B.Array(w["enu"]), B.Obs(freqs, 2, 10, 20), B.Imaging(128),
                                      np.array(lm), 1, dev(volt), img)
        assert e.value.status == B.BLINK_ERR_INVALID_ARG


@pytest.mark.parametrize("name,n_pix,fine,c,flags,pc", [("precision", 512, None, 1, False, (0.31, -0.22)),
                                                        ("uneven", 256, 8, 1, True, (-0.05, 0.4))])
def test_cells_and_uvw_bit_exact_off_zenith(B, ctx, name, n_pix, fine, c, flags, pc):
    check_cells_and_uvw(B, ctx, name, n_pix, fine, c, flags, pc)


# ---------------------------------------------------------------------------------------------------
# bounded device-side waits
# ---------------------------------------------------------------------------------------------------

def test_bounded_wait_runs_out_and_reports_timeout(B):
    # The batched imaging kernel's row tasks are made to wait for one more column task than an image has
    # (a count nothing reaches); each such wait gives up after its budget (2e6 cycles, about a millisecond),
    # the launch stops and returns, and blink_sync reports BLINK_ERR_TIMEOUT.  Nothing faults or hangs; the
    # same context then images correctly again once the setting is restored, and so does a fresh one.
    w, volt, freqs, _ = _case("coarse", n_samples=20, fine=16)
    n = 2 * 16
    arr, obs, im = B.Array(w["enu"]), B.Obs(freqs, 1, 10, 20), B.Imaging(512)
    ref = oracle.pipeline(volt, w["enu"], freqs, 10, 1, 512, ids=np.array([0, n - 1]), n_threads=8)["images"]
    c = B.blink_create(0)
    try:
        img = torch.empty((n, 512, 512), dtype=torch.float32, device="cuda")
        d_volt = dev(volt)
        B.blink_pipeline(c, arr, obs, im, B.BLINK_CORR_FP8, B.BLINK_MODE_BATCHED, d_volt, img)   # plan + tuning
        B.blink_sync(c)
        B.blink_set_wait_budget(c, 2_000_000, unreachable=True)
        B.blink_pipeline(c, arr, obs, im, B.BLINK_CORR_FP8, B.BLINK_MODE_BATCHED, d_volt, img)
        with pytest.raises(B.BlinkError) as e:
            B.blink_sync(c)
        assert e.value.status == B.BLINK_ERR_TIMEOUT
        B.blink_sync(c)                                   # the status word was cleared by the report
        B.blink_set_wait_budget(c, 0, unreachable=False)
        img.fill_(float("nan"))
        B.blink_pipeline(c, arr, obs, im, B.BLINK_CORR_FP8, B.BLINK_MODE_BATCHED, d_volt, img)
        B.blink_sync(c)
        got = img.cpu().numpy()
        for k, q in enumerate((0, n - 1)):
            assert_image_close(got[q], ref[k], q)
    finally:
        B.blink_destroy(c)
    c2 = B.blink_create(0)
    try:
        img = torch.full((n, 512, 512), float("nan"), dtype=torch.float32, device="cuda")
        B.blink_pipeline(c2, arr, obs, im, B.BLINK_CORR_FP8, B.BLINK_MODE_BATCHED, dev(volt), img)
        B.blink_sync(c2)
        assert_image_close(img[n - 1].cpu().numpy(), ref[1], "fresh context")
    finally:
        B.blink_destroy(c2)
