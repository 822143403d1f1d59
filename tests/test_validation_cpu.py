"""Argument validation of every C-ABI entry point (CPU only).

Each entry point checks its arguments before it touches the context or the device, so every rejected case
is reported with its status and message without a GPU, and a call whose arguments are all valid reaches
the context check ("context is NULL").  The pointers below are never dereferenced: each call is
rejected before any device work.
"""
import numpy as np
import pytest

from paper_2505_15204_gb300 import blink as B

PTR = 1 << 20            # a 16-byte aligned stand-in address


def _enu(n=4):
    return np.arange(3 * n, dtype=np.float64).reshape(n, 3)


def _obs(**kw):
    args = dict(fine_freq_hz=np.full(4, 150e6), chan_avg=2, samples_per_int=10, n_samples=20)
    args.update(kw)
    return B.Obs(**args)


def _err(fn, *args):
    with pytest.raises(B.BlinkError) as e:
        fn(*args)
    return e.value.status, str(e.value)


def _expect(status, text, fn, *args):
    st, msg = _err(fn, *args)
    assert st == status and text in msg, (st, msg)


NO_CTX = (B.BLINK_ERR_INVALID_ARG, "context is NULL")


@pytest.mark.parametrize("array,obs,status,text", [
    (B.Array(_enu(0)), _obs(), B.BLINK_ERR_INVALID_ARG, "n_tiles must be in [1, 512]"),
    (B.Array(_enu(513)), _obs(), B.BLINK_ERR_INVALID_ARG, "n_tiles must be in [1, 512]"),
    (B.Array(np.where(_enu() == 5, np.nan, _enu())), _obs(), B.BLINK_ERR_INVALID_ARG, "non-finite"),
    (B.Array(_enu()), _obs(chan_avg=3), B.BLINK_ERR_INVALID_ARG, "chan_avg must be >= 1 and divide n_fine"),
    (B.Array(_enu()), _obs(chan_avg=0), B.BLINK_ERR_INVALID_ARG, "chan_avg must be >= 1 and divide n_fine"),
    (B.Array(_enu()), _obs(fine_freq_hz=np.zeros(0)), B.BLINK_ERR_INVALID_ARG, "n_fine must be >= 1"),
    (B.Array(_enu()), _obs(fine_stride=2), B.BLINK_ERR_INVALID_ARG, "fine_stride must be 0 or >= n_fine"),
    (B.Array(_enu()), _obs(samples_per_int=0), B.BLINK_ERR_INVALID_ARG, "samples_per_int must be >= 1"),
    (B.Array(_enu()), _obs(n_samples=25), B.BLINK_ERR_INVALID_ARG, "multiple of samples_per_int"),
    (B.Array(_enu()), _obs(n_samples=-10), B.BLINK_ERR_INVALID_ARG, "multiple of samples_per_int"),
    # the exact-integer bound of the FP32 sums: |S| <= 128 K < 2^24
    (B.Array(_enu()), _obs(samples_per_int=65537, n_samples=0), B.BLINK_ERR_UNSUPPORTED, "above 131072"),
    (B.Array(_enu()), _obs(samples_per_int=1, n_samples=2**31 - 1), B.BLINK_ERR_UNSUPPORTED, "2^31 - 1 images"),
])
def test_correlate_rejects_bad_array_and_obs(array, obs, status, text):
    _expect(status, text, B.blink_correlate, None, array, obs, B.BLINK_CORR_FP8, PTR, PTR)


def test_correlate_buffers_and_arith():
    a, o = B.Array(_enu()), _obs()
    _expect(B.BLINK_ERR_INVALID_ARG, "arith must be", B.blink_correlate, None, a, o, 7, PTR, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "d_volt or d_vis is NULL", B.blink_correlate, None, a, o, 0, None, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "16-byte aligned", B.blink_correlate, None, a, o, 0, PTR, PTR + 8)
    _expect(B.BLINK_ERR_INVALID_ARG, "2-byte", B.blink_correlate, None, a, o, 0, PTR + 1, PTR)
    _expect(*NO_CTX, B.blink_correlate, None, a, o, B.BLINK_CORR_FP8, PTR, PTR)
    _expect(*NO_CTX, B.blink_correlate, None, a, o, B.BLINK_CORR_FP32, PTR, PTR)


@pytest.mark.parametrize("imaging,status,text", [
    (B.Imaging(98), B.BLINK_ERR_UNSUPPORTED, "no prime factor above 5"),         # 2 x 7^2
    (B.Imaging(1202), B.BLINK_ERR_UNSUPPORTED, "no prime factor above 5"),       # 2 x 601
    (B.Imaging(75), B.BLINK_ERR_UNSUPPORTED, "even, in [64, 8192]"),
    (B.Imaging(32), B.BLINK_ERR_UNSUPPORTED, "even, in [64, 8192]"),
    (B.Imaging(16384), B.BLINK_ERR_UNSUPPORTED, "even, in [64, 8192]"),
    (B.Imaging(8640), B.BLINK_ERR_UNSUPPORTED, "even, in [64, 8192]"),
    (B.Imaging(64, pol=5), B.BLINK_ERR_INVALID_ARG, "imaging.pol"),
    (B.Imaging(64, precision=9), B.BLINK_ERR_INVALID_ARG, "imaging.precision"),
    (B.Imaging(64, cell_lambda=float("inf")), B.BLINK_ERR_INVALID_ARG, "cell_lambda is not finite"),
])
def test_pipeline_rejects_bad_imaging(imaging, status, text):
    _expect(status, text, B.blink_pipeline, None, B.Array(_enu()), _obs(), imaging, 0, 0, PTR, PTR)


def test_pipeline_frequencies_mode_and_buffers():
    a, o, i = B.Array(_enu()), _obs(), B.Imaging(64)
    for f in (np.array([150e6, -1.0, 150e6, 150e6]), np.array([150e6, np.inf, 150e6, 150e6])):
        _expect(B.BLINK_ERR_INVALID_ARG, "positive and finite", B.blink_pipeline, None, a, _obs(fine_freq_hz=f), i,
                0, 0, PTR, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "mode must be", B.blink_pipeline, None, a, o, i, 0, 3, PTR, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "arith must be", B.blink_pipeline, None, a, o, i, 2, 0, PTR, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "d_volt or d_img is NULL", B.blink_pipeline, None, a, o, i, 0, 0, PTR, None)
    _expect(B.BLINK_ERR_INVALID_ARG, "8-byte aligned", B.blink_pipeline, None, a, o, i, 0, 0, PTR, PTR + 4)
    for mode in (B.BLINK_MODE_BATCHED, B.BLINK_MODE_PLAIN):
        _expect(*NO_CTX, B.blink_pipeline, None, a, o, i, B.BLINK_CORR_FP8, mode, PTR, PTR)


def test_pipeline_sets_validate_every_set_and_the_capacity():
    a, o = B.Array(_enu()), _obs()              # 4 fine channels, chan_avg 2, T = 2
    im = B.Imaging(64)
    fn = B.blink_pipeline_sets
    cap = 4 * 2 * 64 * 64                       # T * F * N^2 for both output channels
    _expect(B.BLINK_ERR_INVALID_ARG, "no sets", fn, None, a, o, [], 0, PTR, PTR, cap)
    for s in (B.Set(3, 2, im), B.Set(0, 1, im), B.Set(-2, 2, im), B.Set(0, 0, im)):
        _expect(B.BLINK_ERR_INVALID_ARG, "set channel range", fn, None, a, o, [s], 0, PTR, PTR, cap)
    _expect(B.BLINK_ERR_UNSUPPORTED, "no prime factor", fn, None, a, o, [B.Set(0, 2, B.Imaging(98))], 0, PTR, PTR, cap)
    sets = [B.Set(0, 2, B.Imaging(64)), B.Set(2, 2, B.Imaging(128))]
    need = 2 * 1 * 64 * 64 + 2 * 1 * 128 * 128  # packed per set: T * F_set * N_set^2
    _expect(B.BLINK_ERR_INVALID_ARG, "img_capacity", fn, None, a, o, sets, 0, PTR, PTR, need - 1)
    _expect(*NO_CTX, fn, None, a, o, sets, 0, PTR, PTR, need)
    # with calibration every set starts on an output channel (the gains table is indexed per output channel)
    o1 = _obs(chan_avg=1)
    g = B.Array(_enu(), gains=np.ones((4, 4, 2), np.complex64))
    _expect(B.BLINK_ERR_INVALID_ARG, "start on an output channel", fn, None, g, _obs(), [B.Set(1, 2, im)], 0, PTR,
            PTR, cap)
    _expect(*NO_CTX, fn, None, g, o1, [B.Set(1, 2, im)], 0, PTR, PTR, cap)


def test_grid_image_and_cells():
    a, o, i = B.Array(_enu()), _obs(), B.Imaging(64)      # T * F = 4 images
    _expect(B.BLINK_ERR_INVALID_ARG, "negative image range", B.blink_grid, None, a, o, i, PTR, -1, 1, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "image range beyond", B.blink_grid, None, a, o, i, PTR, 3, 2, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "8-byte aligned", B.blink_grid, None, a, o, i, PTR + 4, 0, 4, PTR)
    _expect(*NO_CTX, B.blink_grid, None, a, o, i, PTR, 0, 4, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "n_images < 0", B.blink_image, None, i, PTR, -1, PTR, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "is NULL", B.blink_image, None, i, PTR, 1, None, PTR)
    _expect(*NO_CTX, B.blink_image, None, i, PTR, 0, PTR, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "d_cells is NULL", B.blink_cells, None, a, o, i, None)
    _expect(*NO_CTX, B.blink_cells, None, a, o, i, PTR)


def test_image_noalloc_limits_without_context():
    fn = B.blink_image_noalloc
    _expect(B.BLINK_ERR_UNSUPPORTED, "16 MiB static scratch", fn, B.Imaging(2048), PTR, 1, PTR, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "imaging.precision", fn, B.Imaging(64, precision=5), PTR, 1, PTR, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "8-byte aligned", fn, B.Imaging(64), PTR, 1, PTR, PTR + 4)
    # the checks of blink_image: support, polarisation, phase centre, cell
    _expect(B.BLINK_ERR_INVALID_ARG, "imaging.support", fn, B.Imaging(64, support=-1), PTR, 1, PTR, PTR)
    _expect(B.BLINK_ERR_UNSUPPORTED, "convolution kernel", fn, B.Imaging(64, support=4), PTR, 1, PTR, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "imaging.pol", fn, B.Imaging(64, pol=7), PTR, 1, PTR, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "direction cosines", fn, B.Imaging(64, phase_centre=(0.9, 0.9)), PTR, 1, PTR, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "cell_lambda", fn, B.Imaging(64, cell_lambda=float("inf")), PTR, 1, PTR, PTR)
    # no images: only the set-up (the scratch's address on the current device) runs, a warm-up; without a GPU
    # that set-up reports the CUDA error
    try:
        fn(B.Imaging(64), PTR, 0, PTR, PTR)
    except B.BlinkError as e:
        assert e.status == B.BLINK_ERR_CUDA, str(e)


def test_dedisperse_validates_delays_before_any_device_work():
    fn = B.blink_dedisperse
    _expect(B.BLINK_ERR_INVALID_ARG, "delays must be >= 0", fn, None, PTR, 4, 3, 64, [0, -1, 0], PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "max(delays) must be < n_int", fn, None, PTR, 4, 3, 64, [0, 4, 0], PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "n_int and n_chan must be >= 1", fn, None, PTR, 0, 3, 64, [0, 0, 0], PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "even, in [64, 8192]", fn, None, PTR, 4, 3, 101, [0, 0, 0], PTR)
    _expect(*NO_CTX, fn, None, PTR, 4, 3, 1200, [0, 0, 0], PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "16-byte aligned", fn, None, PTR + 8, 4, 3, 64, [0, 0, 0], PTR)
    _expect(*NO_CTX, fn, None, PTR, 4, 3, 64, [0, 3, 1], PTR)
    with pytest.raises(ValueError):
        fn(None, PTR, 4, 3, 64, [0, 1], PTR)     # one delay per channel, checked by the binding


def test_dedisperse_stream_validates_before_any_device_work():
    fn = B.blink_dedisperse_stream
    _expect(B.BLINK_ERR_INVALID_ARG, "delays must be >= 0", fn, None, PTR, 0, PTR, 4, 3, 64, [0, -1, 0], PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "n_int and n_chan must be >= 1", fn, None, PTR, 0, PTR, 0, 3, 64, [0, 0, 0], PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "t0 must be >= 0", fn, None, PTR, -1, PTR, 4, 3, 64, [0, 0, 0], PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "even, in [64, 8192]", fn, None, PTR, 0, PTR, 4, 3, 66 * 129, [0, 0, 0], PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "d_carry is NULL", fn, None, None, 0, PTR, 4, 3, 64, [0, 2, 0], PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "16-byte aligned", fn, None, PTR + 4, 0, PTR, 4, 3, 64, [0, 2, 0], PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "h_n_out is NULL", fn, None, PTR, 0, None, 4, 3, 64, [0, 2, 0], PTR)
    # a delay longer than the cube is allowed here (the carry spans cubes); no carry is needed for zero delays
    _expect(*NO_CTX, fn, None, PTR, 0, PTR, 4, 3, 64, [0, 9, 1], PTR)
    _expect(*NO_CTX, fn, None, None, 5, PTR, 4, 3, 1200, [0, 0, 0], PTR)
    with pytest.raises(ValueError):
        fn(None, PTR, 0, PTR, 4, 3, 64, [0, 1], PTR)     # one delay per channel, checked by the binding


def test_pipeline_host_arguments():
    a, o, i = B.Array(_enu()), _obs(), B.Imaging(64)
    h_volt = np.zeros(16, np.uint8)
    h_img = np.zeros(16, np.float32)
    fn = B.blink_pipeline_host
    _expect(B.BLINK_ERR_INVALID_ARG, "images_per_pass < 0", fn, None, a, o, i, 0, h_volt, h_img, -1)
    _expect(B.BLINK_ERR_INVALID_ARG, "h_volt or h_img is NULL", fn, None, a, o, i, 0, None, h_img)
    _expect(*NO_CTX, fn, None, a, o, i, 0, h_volt, h_img, 0)


def test_convolution_kernel_options():
    a, o = B.Array(_enu()), _obs()
    _expect(B.BLINK_ERR_INVALID_ARG, "imaging.support", B.blink_pipeline, None, a, o, B.Imaging(64, support=17), 0, 0,
            PTR, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "imaging.support", B.blink_pipeline, None, a, o, B.Imaging(64, support=-1), 0, 0,
            PTR, PTR)
    _expect(B.BLINK_ERR_UNSUPPORTED, "at most 4096", B.blink_pipeline, None, a, o, B.Imaging(8192, support=4), 0, 0,
            PTR, PTR)
    _expect(*NO_CTX, B.blink_pipeline, None, a, o, B.Imaging(1200, support=6), 0, B.BLINK_MODE_BATCHED, PTR, PTR)
    k = B.Imaging(64, support=6)
    _expect(*NO_CTX, B.blink_pipeline, None, a, o, k, 0, B.BLINK_MODE_BATCHED, PTR, PTR)
    _expect(*NO_CTX, B.blink_pipeline, None, a, o, B.Imaging(64, support=1), 0, B.BLINK_MODE_PLAIN, PTR, PTR)
    # the kernel runs in the batched forms only
    only = "batched pipeline forms only"
    _expect(B.BLINK_ERR_UNSUPPORTED, only, B.blink_pipeline, None, a, o, k, 0, B.BLINK_MODE_PLAIN, PTR, PTR)
    _expect(B.BLINK_ERR_UNSUPPORTED, only, B.blink_grid, None, a, o, k, PTR, 0, 1, PTR)
    _expect(B.BLINK_ERR_UNSUPPORTED, only, B.blink_image, None, k, PTR, 1, PTR, PTR)
    _expect(B.BLINK_ERR_UNSUPPORTED, only, B.blink_cells, None, a, o, k, PTR)
    _expect(B.BLINK_ERR_UNSUPPORTED, only, B.blink_image_noalloc, k, PTR, 1, PTR, PTR)
    _expect(*NO_CTX, B.blink_pipeline_sets, None, a, o, [B.Set(0, 2, k), B.Set(2, 2, B.Imaging(64))], 0, PTR, PTR,
            2 * 2 * 64 * 64)
    _expect(*NO_CTX, B.blink_pipeline_host, None, a, o, k, 0, np.zeros(4, np.uint8), np.zeros(4, np.float32), 0)


def test_phase_centre_options():
    a, o = B.Array(_enu()), _obs()
    for pc in ((0.8, 0.6), (1.0, 0.0), (float("nan"), 0.0), (0.0, float("inf"))):
        _expect(B.BLINK_ERR_INVALID_ARG, "direction cosines", B.blink_pipeline, None, a, o,
                B.Imaging(64, phase_centre=pc), 0, 0, PTR, PTR)
    k = B.Imaging(64, phase_centre=(0.3, -0.2))
    for mode in (B.BLINK_MODE_BATCHED, B.BLINK_MODE_PLAIN):
        _expect(*NO_CTX, B.blink_pipeline, None, a, o, k, 0, mode, PTR, PTR)
    _expect(*NO_CTX, B.blink_cells, None, a, o, k, PTR)
    _expect(*NO_CTX, B.blink_image, None, k, PTR, 0, PTR, PTR)          # the image stage ignores the pointing
    _expect(B.BLINK_ERR_UNSUPPORTED, "pipeline forms only", B.blink_grid, None, a, o, k, PTR, 0, 1, PTR)


def test_tracking_pointings():
    a, o, k = B.Array(_enu()), _obs(), B.Imaging(64)          # two integrations
    for lm in ([(0.1, 0.0), (0.8, 0.7)], [(float("nan"), 0.0), (0.0, 0.0)], [(0.0, 0.0), (1.0, 0.0)]):
        _expect(B.BLINK_ERR_INVALID_ARG, "h_lm", B.blink_pipeline_tracking, None, a, o, k, np.array(lm), 1, PTR, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "arith", B.blink_pipeline_tracking, None, a, o, k, np.zeros((2, 2)), 5, PTR, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "NULL", B.blink_pipeline_tracking, None, a, o, k, np.zeros((2, 2)), 1, 0, PTR)
    _expect(*NO_CTX, B.blink_pipeline_tracking, None, a, o, k, np.array([(0.1, 0.2), (0.3, -0.1)]), 1, PTR, PTR)
    with pytest.raises(ValueError):
        B.blink_pipeline_tracking(None, a, o, k, np.zeros(4), 1, PTR, PTR)


@pytest.mark.parametrize("n", [96, 150, 1200, 2400, 4096, 8192])
def test_mixed_radix_sides_reach_the_context_check(n):
    a, o, k = B.Array(_enu()), _obs(), B.Imaging(n)
    for mode in (B.BLINK_MODE_BATCHED, B.BLINK_MODE_PLAIN):
        _expect(*NO_CTX, B.blink_pipeline, None, a, o, k, 0, mode, PTR, PTR)
    _expect(*NO_CTX, B.blink_image, None, k, PTR, 1, PTR, PTR)
    _expect(*NO_CTX, B.blink_grid, None, a, o, k, PTR, 0, 1, PTR)
    _expect(*NO_CTX, B.blink_cells, None, a, o, k, PTR)


def test_image_noalloc_scratch_limit_on_mixed_radix_sides():
    fn = B.blink_image_noalloc
    # 2400 x 1204 FP32 pairs exceed the 16 MiB scratch; BF16 pairs fit.  Both are rejected or accepted before
    # any device work: the accepted call stops at the scratch look-up, which fails without a device.
    _expect(B.BLINK_ERR_UNSUPPORTED, "16 MiB static scratch", fn, B.Imaging(2400), PTR, 1, PTR, PTR)


def test_averaged_pipeline_arguments():
    a, o, k = B.Array(_enu()), _obs(), B.Imaging(64)          # T = 2 integrations, F = 2 output channels
    fn = B.blink_pipeline_averaged
    for t_avg, f_avg in ((0, 1), (1, 0), (3, 1), (1, 3), (-1, 2)):
        _expect(B.BLINK_ERR_INVALID_ARG, "t_avg and f_avg", fn, None, a, o, k, 1, t_avg, f_avg, PTR, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "arith", fn, None, a, o, k, 7, 1, 1, PTR, PTR)
    _expect(B.BLINK_ERR_INVALID_ARG, "NULL", fn, None, a, o, k, 1, 1, 1, 0, PTR)
    for t_avg, f_avg in ((1, 1), (2, 1), (1, 2), (2, 2)):
        _expect(*NO_CTX, fn, None, a, o, k, 1, t_avg, f_avg, PTR, PTR)
    _expect(*NO_CTX, fn, None, a, o, B.Imaging(1200, support=6), 0, 2, 2, PTR, PTR)
