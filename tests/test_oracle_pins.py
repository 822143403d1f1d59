"""Pins of the CPU oracle against things other than itself (CPU only).

Each test fixes one oracle function with a closed form, an invariant, a brute-force sum, an independent
library routine or a number printed in the paper, chosen so that a plausible slip (a dropped term, a
wrong sign or conjugate, a swapped index or polarisation, a wrong shift or normalisation) fails a test.
"""
import json
import math
import os

import numpy as np
import pytest

import blinksynth as bs
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
C_LIGHT = 299_792_458.0


def _bidx(i, j):
    return i * (i + 1) // 2 + j


# ----------------------------------------------------------------------------------------------
# correlation (Eq. 2; Sec. 5.2.2)
# ----------------------------------------------------------------------------------------------

def test_correlate_constant_voltages_closed_form():
    # every sample of every input = a + ib  =>  S_ij^pq = K (a^2 + b^2), imaginary part 0
    a, b, ns, c, nt = 3, -2, 5, 2, 6
    v = bs.constant_voltages(ns * 2, c * 3, nt, a, b)
    S = oracle.correlate(v, ns, c)
    K = ns * c
    assert S.shape == (2, 3, nt * (nt + 1) // 2, 4, 2)
    assert np.all(S[..., 0] == K * (a * a + b * b))
    assert np.all(S[..., 1] == 0)


def test_correlate_phase_pattern_conjugates_second_tile():
    # x_i^p = 2 * i^(k_ip) with distinct powers per tile and polarisation:
    # S_ij^pq = K * 4 * i^(k_ip - k_jq) exactly.  A conjugate on the wrong factor flips the sign of Im;
    # swapping XY and YX or i and j changes which power appears.
    nt, ns = 5, 3
    rng = np.random.default_rng(7)
    k = rng.integers(0, 4, size=(nt, 2))
    x = 2 * (1j ** k)
    v = np.broadcast_to(bs.pack_complex(x), (ns, 1, nt, 2)).copy()
    S = oracle.correlate(v, ns, 1)[0, 0]
    for i in range(nt):
        for j in range(i + 1):
            for p in range(2):
                for q in range(2):
                    want = ns * 4 * (1j ** ((k[i, p] - k[j, q]) % 4))
                    got = S[_bidx(i, j), 2 * p + q]
                    assert got[0] == round(want.real) and got[1] == round(want.imag), (i, j, p, q)


def test_correlate_unpacks_every_byte_value():
    # one sample per channel, channel f carries byte f on tile 1 (X) against 1 + 0i on tile 0 (X):
    # S_10^XX = x_1 conj(1) = x_1 reads back the decoded byte, S_11^XX = |x_1|^2.  The format (Sec. 5.2.1,
    # 4-bit complex) is low nibble = real, high nibble = imaginary, each two's complement in [-8, 7].
    v = np.zeros((1, 256, 2, 2), dtype=np.uint8)
    v[0, :, 0, 0] = 0x01
    v[0, :, 1, 0] = np.arange(256, dtype=np.uint8)
    S = oracle.correlate(v, 1, 1)[0]
    for b in range(256):
        re_, im_ = ((b & 15) ^ 8) - 8, ((b >> 4) ^ 8) - 8
        assert tuple(S[b, _bidx(1, 0), 0]) == (re_, im_), b
        assert tuple(S[b, _bidx(1, 1), 0]) == (re_ * re_ + im_ * im_, 0), b
        assert not S[b, :, 1:].any()


def test_correlate_single_product_lands_in_its_slot():
    # one non-zero sample on tile 4 pol X and tile 1 pol Y: only S_41^XY = x conj(y) is non-zero
    nt = 6
    v = np.zeros((1, 1, nt, 2), np.uint8)
    v[0, 0, 4, 0] = bs.pack_complex(np.array(3 - 1j))
    v[0, 0, 1, 1] = bs.pack_complex(np.array(-2 + 5j))
    S = oracle.correlate(v, 1, 1)[0, 0]
    want = (3 - 1j) * np.conj(-2 + 5j)
    nz = np.argwhere(np.any(S != 0, axis=-1))
    # autos of the two tiles and the cross product
    slots = {tuple(r) for r in nz}
    assert (_bidx(4, 1), 1) in slots                     # XY of baseline (4, 1)
    got = S[_bidx(4, 1), 1]
    assert got[0] == want.real and got[1] == want.imag
    assert slots == {(_bidx(4, 1), 1), (_bidx(4, 4), 0), (_bidx(1, 1), 3)}


def test_correlate_autos_real_nonnegative_and_hermitian_pol_pairs():
    w = bs.build_workload("tiny")
    S = oracle.correlate(w["volt"], 10, 1)[0, 0]
    nt = w["enu"].shape[0]
    for i in range(nt):
        b = _bidx(i, i)
        assert S[b, 0, 1] == 0 and S[b, 3, 1] == 0           # XX, YY autos real
        assert S[b, 0, 0] >= 0 and S[b, 3, 0] >= 0
        assert S[b, 1, 0] == S[b, 2, 0] and S[b, 1, 1] == -S[b, 2, 1]   # XY = conj(YX)


def test_correlate_blocks_add_up():
    # an integration of N_s samples over c channels is the sum of its single-sample, single-channel products
    w = bs.build_workload("coarse", n_samples=20)
    v = w["volt"][:, :8]
    S = oracle.correlate(v, 10, 4)
    S1 = oracle.correlate(v, 1, 1)
    for tau in range(2):
        for f in range(2):
            want = S1[tau * 10:(tau + 1) * 10, f * 4:(f + 1) * 4].sum(axis=(0, 1))
            assert np.array_equal(S[tau, f], want)


def test_correlate_flags_zero_their_baselines_only():
    w = bs.build_workload("tiny")
    flags = np.zeros(128, np.uint8)
    flags[[3, 77]] = 1
    S = oracle.correlate(w["volt"], 10, 1)[0, 0]
    Sf = oracle.correlate(w["volt"], 10, 1, flags=flags)[0, 0]
    for i in (0, 3, 50, 77, 127):
        for j in range(i + 1):
            b = _bidx(i, j)
            if flags[i] or flags[j]:
                assert not Sf[b].any()
            else:
                assert np.array_equal(Sf[b], S[b])


def test_correlate_noise_power_statistics():
    # E[S_ii^XX / K] = E|x|^2 for the quantised noise; with sigma = 2 per component the quantised
    # variance per component is sigma^2 + 1/12 to within a few percent (Sheppard's correction).
    sky = bs.Sky(lmn=np.zeros((0, 3)), power=np.zeros(0))
    enu = bs.tile_positions(16, 100.0, 1)
    v = bs.voltages(enu, np.array([150e6]), 4000, sky, seed=5)
    S = oracle.correlate(v, 4000, 1)[0, 0]
    autos = np.array([S[_bidx(i, i), 0, 0] for i in range(16)]) / 4000.0
    assert abs(autos.mean() - 2 * (4 + 1 / 12)) < 0.1
    cross = np.array([S[_bidx(i, j), 0] for i in range(16) for j in range(i)]) / 4000.0
    assert np.abs(cross).max() < 6 * 8 / math.sqrt(4000)


def test_visibility_is_one_float32_division():
    S = np.array([[7, -3], [1, 1], [2 ** 20 + 1, -(2 ** 19)]], np.int64)
    V = oracle.visibilities(S, 30)
    assert V.dtype == np.complex64
    assert np.float32(V[0].real) == np.float32(7) / np.float32(30)
    assert np.float32(V[2].imag) == np.float32(-(2 ** 19)) / np.float32(30)


# ----------------------------------------------------------------------------------------------
# geometry (Sec. 5.2.3-5.2.4)
# ----------------------------------------------------------------------------------------------

def test_uvw_hand_computed():
    enu = np.array([[0.0, 0.0, 0.0], [100.0, -50.0, 3.0], [10.0, 20.0, 0.0]])
    nu = C_LIGHT            # wavelength 1 m => (u, v, w) = baseline in metres
    u = oracle.uvw(enu, nu)
    assert np.allclose(u[_bidx(1, 0)], [100.0, -50.0, 3.0], rtol=0, atol=1e-12)
    assert np.allclose(u[_bidx(2, 1)], [-90.0, 70.0, -3.0], rtol=0, atol=1e-12)
    assert np.all(u[[_bidx(i, i) for i in range(3)]] == 0.0)
    u2 = oracle.uvw(enu, 2 * nu)
    assert np.allclose(u2, 2 * u, rtol=0, atol=1e-12)


def test_output_freqs_mean_of_fine_centres():
    fine = bs.fine_frequencies([121])
    out = oracle.output_freqs(fine, 4)
    # group g of 4 covers fine channels 4g..4g+3, centre = f_cc - 640 kHz + (4g + 2) * 10 kHz
    g = np.arange(32)
    assert np.allclose(out, 121 * 1.28e6 - 640e3 + (4 * g + 2) * 10e3, rtol=0, atol=1e-6)


def test_default_cell_puts_longest_baseline_in_outer_cell():
    w = bs.build_workload("tiny")
    enu, nu = w["enu"], 154.88e6
    for n in (64, 256, 512):
        du = oracle.default_cell(enu, nu, n)
        iu, iv, keep = oracle.cells(oracle.uvw(enu, nu), du, n)
        assert keep.all()
        r = np.hypot(iu, iv)
        assert max(np.abs(iu).max(), np.abs(iv).max()) <= n // 2 - 1
        assert r.max() >= n // 2 - 2
        # the longest baseline's |(u, v)| is exactly u_max = du * (N/2 - 1) up to rounding
        uv = oracle.uvw(enu, nu)
        assert math.isclose(np.hypot(uv[:, 0], uv[:, 1]).max(), du * (n // 2 - 1), rel_tol=1e-12)


def test_cells_round_half_up_and_drop_outside():
    uvw = np.array([[2.5, -2.5, 0], [127.4, 0, 0], [127.6, 0, 0], [-127.6, 3.49, 0], [0.49, -0.51, 0]])
    iu, iv, keep = oracle.cells(uvw, 1.0, 256)
    assert list(keep) == [1, 1, 0, 0, 1]
    assert (iu[0], iv[0]) == (3, -2)
    assert iu[1] == 127
    assert (iu[4], iv[4]) == (0, -1)


# ----------------------------------------------------------------------------------------------
# gridding (Sec. 5.2.4)
# ----------------------------------------------------------------------------------------------

def _tiny_grid(n=64, pol=oracle.POL_I, autos=True, flags=None):
    w = bs.build_workload("tiny")
    S = oracle.correlate(w["volt"], 10, 1, flags=flags)[0, 0]
    nu = 154.88e6
    du = oracle.default_cell(w["enu"], nu, n, flags=flags)
    iu, iv, keep = oracle.cells(oracle.uvw(w["enu"], nu), du, n)
    G, W = oracle.grid(S, 128, 10, iu, iv, keep, n, pol=pol, autos=autos, flags=flags)
    return S, G, W, (iu, iv, keep)


def test_grid_is_hermitian():
    _, G, _, _ = _tiny_grid()
    n = G.shape[0]
    idx = (-np.arange(n)) % n
    assert np.array_equal(G[np.ix_(idx, idx)], np.conj(G))


def test_grid_sum_and_weights():
    S, G, W, (iu, iv, keep) = _tiny_grid()
    nt, K = 128, 10
    assert keep.all()
    assert W == nt * nt                          # N_a(N_a - 1) cross + N_a autos, weight 1 each
    I = (S[:, 0] + S[:, 3]) / (2.0 * K)          # Stokes I per baseline (re, im)
    autos = np.array([_bidx(i, i) for i in range(nt)])
    cross = np.setdiff1d(np.arange(len(S)), autos)
    want = 2 * I[cross, 0].sum() + I[autos, 0].sum()
    assert math.isclose(G.sum().real, want, rel_tol=1e-12)
    assert abs(G.sum().imag) < 1e-9 * abs(want)
    # without autos, W = N_a (N_a - 1) and the DC cell loses exactly the autos' sum
    _, G2, W2, _ = _tiny_grid(autos=False)
    assert W2 == nt * (nt - 1)
    assert math.isclose(G[0, 0].real - G2[0, 0].real, I[autos, 0].sum(), rel_tol=1e-12)


def test_grid_places_visibility_and_mirror_at_its_cell():
    nt, n = 3, 16
    S = np.zeros((6, 4, 2), np.int64)
    S[_bidx(2, 0), 0] = [20, 6]      # XX
    S[_bidx(2, 0), 3] = [4, 2]       # YY
    iu = np.array([0, 0, 0, 3, 0, 0], np.int32)
    iv = np.array([0, 0, 0, -5, 0, 0], np.int32)
    keep = np.ones(6, np.uint8)
    G, W = oracle.grid(S, nt, 2, iu, iv, keep, n, autos=False)
    I = ((20 + 4) + 1j * (6 + 2)) / 4.0
    assert G[(-5) % n, 3] == I
    assert G[5, (-3) % n] == np.conj(I)
    Gx, _ = oracle.grid(S, nt, 2, iu, iv, keep, n, pol=oracle.POL_XX, autos=False)
    assert Gx[(-5) % n, 3] == (20 + 6j) / 2.0


def test_grid_flags_change_weight_sum():
    flags = np.zeros(128, np.uint8)
    flags[:10] = 1
    _, _, W, _ = _tiny_grid(flags=flags)
    assert W == 118 * 118


# ----------------------------------------------------------------------------------------------
# transform and image (Eq. 4; Sec. 5.2.4)
# ----------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [4, 8, 16, 6, 10, 12, 15, 30, 49, 60])
def test_fft_matches_direct_dft(n):
    # powers of two take the radix-2 path, the other sides the mixed-radix recursion (factors 2, 3, 5, and 7 x 7)
    rng = np.random.default_rng(n)
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    a = oracle.ifft2(G)
    d = oracle.idft2(G)
    assert np.abs(a - d).max() <= 1e-12 * np.abs(d).max()


@pytest.mark.parametrize("n", [128, 150, 1200])
def test_fft_matches_numpy_library(n):
    rng = np.random.default_rng(3)
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    a = oracle.ifft2(G)
    ref = np.fft.ifft2(G) * n * n
    assert np.abs(a - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("n", [64, 90])
def test_fft_parseval(n):
    rng = np.random.default_rng(4)
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    a = oracle.ifft2(G)
    assert math.isclose((np.abs(a) ** 2).sum(), n * n * (np.abs(G) ** 2).sum(), rel_tol=1e-12)


@pytest.mark.parametrize("n", [32, 120])
def test_fft_delta_and_single_cell_closed_forms(n):
    G = np.zeros((n, n), complex)
    G[0, 0] = 2.5 - 1j
    assert np.allclose(oracle.ifft2(G), 2.5 - 1j, rtol=0, atol=1e-13)
    # a cell and its mirror: a[y][x] = 2 cos(2 pi (u0 x + v0 y) / n)
    u0, v0 = 3, 5
    G = np.zeros((n, n), complex)
    G[v0, u0] = 1
    G[-v0 % n, -u0 % n] = 1
    y, x = np.mgrid[0:n, 0:n]
    want = 2 * np.cos(2 * np.pi * (u0 * x + v0 * y) / n)
    assert np.abs(oracle.ifft2(G) - want).max() < 1e-12


def test_fft_rejects_an_empty_side():
    with pytest.raises(ValueError):
        oracle.ifft2(np.zeros((0, 0), complex))


@pytest.mark.parametrize("n", [64, 60])
def test_image_pixels_equal_the_whole_image(n):
    # the direct per-pixel sum over a sparse grid's cells against the transform and shift of the whole grid
    rng = np.random.default_rng(n)
    G = np.zeros((n, n), complex)
    for _ in range(40):
        u, v = rng.integers(0, n, 2)
        z = complex(rng.standard_normal(), rng.standard_normal())
        G[v, u] += z
        G[-v % n, -u % n] += np.conj(z)
    img, _ = oracle.image(oracle.ifft2(G), 3.0)
    yx = np.array([(y, x) for y in range(n) for x in range(n)], dtype=np.int32)
    got = oracle.image_pixels(G, 3.0, yx).reshape(n, n)
    assert np.abs(got - img).max() <= 1e-12 * np.abs(img).max()


def test_image_shift_puts_phase_centre_in_middle_pixel():
    n = 16
    a = np.zeros((n, n), complex)
    a[0, 0] = 8.0
    a[0, 1] = 4.0                 # l > 0 neighbour -> x = N/2 + 1
    a[n - 1, 0] = 2.0             # m < 0 neighbour -> y = N/2 - 1
    img, mx = oracle.image(a, 2.0)
    assert img[n // 2, n // 2] == 4.0
    assert img[n // 2, n // 2 + 1] == 2.0
    assert img[n // 2 - 1, n // 2] == 1.0
    assert mx == 0.0


# ----------------------------------------------------------------------------------------------
# end to end
# ----------------------------------------------------------------------------------------------

def test_point_source_at_phase_centre_gives_flux_in_centre_pixel():
    # identical voltages at every tile = a noiseless source at the phase centre: every visibility is
    # |x|^2, so the centre pixel is exactly that flux and it is the image maximum
    w = bs.build_workload("tiny")
    v = bs.constant_voltages(10, 1, 128, 2, 1)
    out = oracle.pipeline(v, w["enu"], w["freqs"], 10, 1, 64)
    img = out["images"][0]
    assert math.isclose(img[32, 32], 5.0, rel_tol=1e-12)
    assert img.max() == img[32, 32]
    assert out["max_im"][0] < 1e-12


@pytest.mark.parametrize("n", [96, 1200])
def test_point_source_at_phase_centre_on_a_mixed_radix_side(n):
    # the same closed form on sides that are not powers of two (the paper's 1200 x 1200 images)
    w = bs.build_workload("tiny")
    v = bs.constant_voltages(10, 1, 128, 2, 1)
    out = oracle.pipeline(v, w["enu"], w["freqs"], 10, 1, n)
    img = out["images"][0]
    assert math.isclose(img[n // 2, n // 2], 5.0, rel_tol=1e-12)
    assert img.max() == img[n // 2, n // 2]
    assert out["max_im"][0] < 1e-12


def test_off_centre_source_peaks_at_its_direction():
    # A strong noiseless source at direction (l, m) drawn by the generator (sign convention of Eq. 3):
    # the dirty image peaks at pixel (N/2 + l N du, N/2 + m N du), not at its mirror.
    enu = bs.tile_positions(64, 1500.0, 11)
    nu = 154.88e6
    n = 128
    du = oracle.default_cell(enu, nu, n)
    fov = 1.0 / du                      # image spans l in [-fov/2, fov/2)
    lm = np.array([0.23 * fov, -0.17 * fov])
    sky = bs.Sky(lmn=np.array([[lm[0], lm[1], math.sqrt(1 - lm @ lm)]]), power=np.array([20.0]))
    v = bs.voltages(enu, np.array([nu]), 40, sky, seed=9, sigma=0.0)
    out = oracle.pipeline(v, enu, np.array([nu]), 40, 1, n)
    img = out["images"][0]
    y, x = np.unravel_index(np.argmax(img), img.shape)
    assert abs(x - (n / 2 + lm[0] * n * du)) <= 1.0
    assert abs(y - (n / 2 + lm[1] * n * du)) <= 1.0


def test_noisy_source_at_phase_centre_adds_autocorrelation_noise_share():
    # Voltage-level source of power S at the phase centre in noise of quantised power P_n per sample: every
    # cross visibility has mean S and every auto S + P_n, so with autos gridded (weight N_a^2) the centre
    # pixel has mean S + P_n / N_a.  Its spread per integration is the thermal sigma_img plus the source's own
    # power fluctuation over K samples (at most S / sqrt(K)); the mean of 16 integrations must sit within
    # 3 of those of S + P_n / N_a.  The autos' share alone is several times that margin, so dropping the
    # autos or the 1/2 of Stokes I fails.
    n_a, K, T = 64, 40, 16
    enu = bs.tile_positions(n_a, 1500.0, 14)
    sigma_img = bs.image_noise(2.0, n_a, K)
    S = 10 * sigma_img
    sky = bs.Sky(lmn=np.array([[0.0, 0.0, 1.0]]), power=np.array([S]))
    v = bs.voltages(enu, np.array([150e6]), K * T, sky, seed=15)
    out = oracle.pipeline(v, enu, np.array([150e6]), K, 1, 64)
    centre = out["images"][:, 32, 32]
    p_n = 2 * (4 + 1 / 12)
    assert centre.shape == (T,)
    spread = math.sqrt(sigma_img ** 2 + S ** 2 / K)
    assert abs(centre.mean() - (S + p_n / n_a)) < 3 * spread / math.sqrt(T)


def test_noise_level_of_pure_noise_image():
    # One polarisation: sigma_img = P_n / sqrt(2 N_cross K); Stokes I averages two independent
    # polarisations, so its noise is smaller by sqrt(2).  P_n is the quantised noise power per sample.
    enu = bs.tile_positions(64, 1500.0, 12)
    sky = bs.Sky(lmn=np.zeros((0, 3)), power=np.zeros(0))
    v = bs.voltages(enu, np.array([150e6]), 40, sky, seed=13)
    p_n = 2 * (4 + 1 / 12)
    xx = p_n / math.sqrt(2 * 64 * 63 / 2 * 40)
    for pol, want in ((oracle.POL_XX, xx), (oracle.POL_I, xx / math.sqrt(2))):
        out = oracle.pipeline(v, enu, np.array([150e6]), 40, 1, 128, autos=False, pol=pol)
        img = out["images"][0]
        assert 0.85 * want < img.std() < 1.15 * want, pol
    assert math.isclose(bs.image_noise(2.0, 64, 40), 8 / math.sqrt(2 * 2016 * 40) / math.sqrt(2))


def test_layout_sizes_match_paper_data_volume_table():
    # the data-volume table (Sec. 7): visibilities and images per second of data for the two test cases,
    # reproduced by this layout (lower triangle with autos, 4 polarisations, complex64; float32 images).
    with open(os.path.join(GOLDEN, "paper_data_volumes.json")) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        nt = case["n_tiles"]
        B = nt * (nt + 1) // 2
        vis = case["n_integrations"] * case["n_channels"] * B * 4 * 8
        img = case["n_integrations"] * case["n_channels"] * case["n_pix"] ** 2 * 4 // case["images_averaged"]
        assert abs(vis / 2 ** 20 - case["visibilities_MiB"]) / case["visibilities_MiB"] < 0.01, case["name"]
        assert abs(img / 2 ** 20 - case["images_MiB"]) / case["images_MiB"] < 0.01, case["name"]


def test_pipeline_matches_stepwise_functions():
    w = bs.build_workload("tiny")
    out = oracle.pipeline(w["volt"], w["enu"], w["freqs"], 10, 1, 64, want_grids=True)
    S = oracle.correlate(w["volt"], 10, 1)[0, 0]
    du = oracle.default_cell(w["enu"], 154.88e6, 64)
    iu, iv, keep = oracle.cells(oracle.uvw(w["enu"], 154.88e6), du, 64)
    G, W = oracle.grid(S, 128, 10, iu, iv, keep, 64)
    assert np.array_equal(out["grids"][0], G)
    img, _ = oracle.image(oracle.ifft2(G), W)
    assert np.array_equal(out["images"][0], img)


# ----------------------------------------------------------------------------------------------
# calibration gains (Sec. 5.2.3): V_ij^pq = g_i^p S_ij^pq conj(g_j^q)
# ----------------------------------------------------------------------------------------------

def _unpack(volt):
    b = volt.astype(np.int64)
    lo, hi = b & 0xF, (b >> 4) & 0xF
    return (np.where(lo >= 8, lo - 16, lo) + 1j * np.where(hi >= 8, hi - 16, hi)).astype(np.complex128)


def _random_gains(n_tiles, seed, shape=()):
    rng = np.random.default_rng(seed)
    amp = rng.uniform(0.5, 1.5, size=shape + (n_tiles, 2))
    ph = rng.uniform(-np.pi, np.pi, size=shape + (n_tiles, 2))
    return amp * np.exp(1j * ph)


def test_gains_equal_brute_force_on_calibrated_voltages():
    # gains applied to the voltages before the products, summed directly in complex FP64: another order of
    # the same arithmetic (catches a conjugate on the wrong gain or a swapped polarisation)
    rng = np.random.default_rng(11)
    nt, ns = 5, 7
    volt = rng.integers(0, 256, size=(ns, 1, nt, 2), dtype=np.uint8)
    g = _random_gains(nt, 12)
    x = _unpack(volt)[:, 0] * g[None]                  # [t][tile][pol]
    S = oracle.correlate(volt, ns, 1)[0, 0]
    V = oracle.apply_gains(S, g)
    for i in range(nt):
        for j in range(i + 1):
            for p in range(2):
                for q in range(2):
                    ref = np.sum(x[:, i, p] * np.conj(x[:, j, q]))
                    assert abs(V[_bidx(i, j), 2 * p + q] - ref) <= 1e-12 * max(1.0, abs(ref))


def test_unit_gains_change_nothing():
    w = bs.build_workload("tiny")
    S = oracle.correlate(w["volt"], 10, 1)[0, 0]
    V = oracle.apply_gains(S, np.ones((128, 2), dtype=np.complex128))
    assert np.array_equal(V, S[..., 0] + 1j * S[..., 1])
    a = oracle.pipeline(w["volt"], w["enu"], w["freqs"], 10, 1, 64)
    b = oracle.pipeline(w["volt"], w["enu"], w["freqs"], 10, 1, 64, gains=np.ones((1, 128, 2), np.complex128))
    assert np.array_equal(a["images"], b["images"]) and np.array_equal(a["W"], b["W"])


def test_gains_keep_autocorrelations_hermitian():
    # S_ii^XY = conj S_ii^YX survives calibration: g^X S conj(g^Y) = conj(g^Y conj(S) conj(g^X))
    w = bs.build_workload("tiny")
    S = oracle.correlate(w["volt"], 10, 1)[0, 0]
    V = oracle.apply_gains(S, _random_gains(128, 3))
    for i in range(0, 128, 7):
        b = _bidx(i, i)
        assert abs(V[b, 1] - np.conj(V[b, 2])) <= 1e-9 * abs(V[b, 1]) + 1e-9
        assert abs(V[b, 0].imag) <= 1e-9 * abs(V[b, 0]) and V[b, 0].real >= 0


def test_gains_undo_a_per_tile_phase_corruption():
    # identical voltages at every tile (a noiseless source at the phase centre) seen through per-tile
    # phases exp(i phi_a): uncalibrated, the centre pixel loses flux; with gains exp(-i phi_a) the image
    # equals the uncorrupted one (the corruption is applied exactly, by rotating the unit-modulus samples
    # 1 + 0i by quarter turns, which the 4-bit format represents without rounding)
    nt, ns = 8, 10
    turns = np.arange(nt) % 4                           # phi_a = turns * pi / 2
    rot = {0: (1, 0), 1: (0, 1), 2: (-1 & 0xF, 0), 3: (0, -1 & 0xF)}
    volt = np.zeros((ns, 1, nt, 2), dtype=np.uint8)
    clean = np.zeros_like(volt)
    for a in range(nt):
        re, im = rot[turns[a]]
        volt[:, 0, a, :] = re | (im << 4)
        clean[:, 0, a, :] = 1
    enu = bs.tile_positions(nt, 200.0, 5)
    freqs = np.array([150e6])
    g = np.exp(-1j * turns * np.pi / 2)[None, :, None] * np.ones((1, nt, 2))
    ref = oracle.pipeline(clean, enu, freqs, ns, 1, 32)["images"][0]
    bad = oracle.pipeline(volt, enu, freqs, ns, 1, 32)["images"][0]
    fixed = oracle.pipeline(volt, enu, freqs, ns, 1, 32, gains=g)["images"][0]
    assert np.allclose(fixed, ref, rtol=0, atol=1e-12)
    assert bad[16, 16] < 0.5 * ref[16, 16]


# ----------------------------------------------------------------------------------------------
# incoherent dedispersion of the image cube (the FRB search after imaging)
# ----------------------------------------------------------------------------------------------

def test_dedisperse_zero_delays_is_the_band_mean():
    rng = np.random.default_rng(21)
    img = rng.normal(size=(6, 5, 4, 3))
    out = oracle.dedisperse(img, np.zeros(5, np.int32))
    assert np.allclose(out, img.mean(axis=1), rtol=1e-14, atol=1e-14)


def test_dedisperse_realigns_a_dispersed_pulse():
    # a pulse reaching channel f at integration t0 + d_f: dedispersion with those delays stacks it at t0 with
    # its full amplitude and nothing elsewhere; one channel's delay wrong by one loses exactly 1/F of it
    T, F, t0 = 12, 6, 2
    d = np.array([5, 4, 2, 1, 1, 0], dtype=np.int32)
    img = np.zeros((T, F, 3, 3))
    for f in range(F):
        img[t0 + d[f], f, 1, 2] = 7.0
    out = oracle.dedisperse(img, d)
    assert out.shape == (T - 5, 3, 3)
    assert out[t0, 1, 2] == 7.0 and np.count_nonzero(out) == 1
    bad = d.copy()
    bad[3] += 1
    assert oracle.dedisperse(img, bad)[t0, 1, 2] == pytest.approx(7.0 * (F - 1) / F)


def test_dedisperse_equals_direct_sum():
    rng = np.random.default_rng(22)
    img = rng.normal(size=(9, 4, 5))
    d = np.array([0, 3, 1, 2], dtype=np.int32)
    out = oracle.dedisperse(img, d)
    for t in range(9 - 3):
        ref = sum(img[t + d[f], f] for f in range(4)) / 4
        assert np.allclose(out[t], ref, rtol=0, atol=1e-15)


def _random_jones(n_tiles, seed, shape=()):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=shape + (n_tiles, 2, 2)) + 1j * rng.normal(size=shape + (n_tiles, 2, 2)))


def test_jones_equal_brute_force_on_mixed_voltages():
    # J applied to each tile's voltage pair before the products (x' = J x), summed directly: another order
    rng = np.random.default_rng(13)
    nt, ns = 4, 6
    volt = rng.integers(0, 256, size=(ns, 1, nt, 2), dtype=np.uint8)
    J = _random_jones(nt, 14)
    x = np.einsum("apr,tar->tap", J, _unpack(volt)[:, 0])      # [t][tile][pol]
    V = oracle.apply_jones(oracle.correlate(volt, ns, 1)[0, 0], J)
    for i in range(nt):
        for j in range(i + 1):
            for p in range(2):
                for q in range(2):
                    ref = np.sum(x[:, i, p] * np.conj(x[:, j, q]))
                    assert abs(V[_bidx(i, j), 2 * p + q] - ref) <= 1e-12 * max(1.0, abs(ref))


def test_diagonal_jones_are_gains():
    w = bs.build_workload("tiny")
    S = oracle.correlate(w["volt"], 10, 1)[0, 0]
    g = _random_gains(128, 4)
    J = np.zeros((128, 2, 2), np.complex128)
    J[:, 0, 0], J[:, 1, 1] = g[:, 0], g[:, 1]
    assert np.allclose(oracle.apply_jones(S, J), oracle.apply_gains(S, g), rtol=1e-13, atol=1e-9)
    a = oracle.pipeline(w["volt"], w["enu"], w["freqs"], 10, 1, 64, gains=g[None])
    b = oracle.pipeline(w["volt"], w["enu"], w["freqs"], 10, 1, 64, gains=J[None])
    assert np.allclose(a["images"], b["images"], rtol=0, atol=1e-12)


# ----------------------------------------------------------------------------------------------
# gridding with a Kaiser-Bessel convolution kernel (Sec. 5.2.4; kernels are work in progress in Sec. 8)
# ----------------------------------------------------------------------------------------------

def test_i0_series_matches_library():
    special = pytest.importorskip("scipy.special")
    for x in (0.0, 1e-3, 0.5, 1.0, 5.62, 9.0, 13.86, 24.97, 40.0):
        assert math.isclose(oracle.i0(x), float(special.i0(x)), rel_tol=2e-15), x


@pytest.mark.parametrize("W", [2, 4, 6, 8, 16])
def test_kb_kernel_has_unit_integral_and_its_support(W):
    integrate = pytest.importorskip("scipy.integrate")
    val, err = integrate.quad(lambda t: oracle.kb(t, W), -W / 2, W / 2, epsabs=1e-14, epsrel=1e-13, limit=200)
    assert math.isclose(val, 1.0, rel_tol=1e-11)
    assert oracle.kb(W / 2, W) == 0.0 and oracle.kb(-W / 2 - 0.1, W) == 0.0
    assert oracle.kb(W / 2 - 1e-9, W) > 0.0
    ts = np.linspace(0.0, W / 2 - 1e-6, 50)
    vals = [oracle.kb(t, W) for t in ts]
    assert all(a >= b for a, b in zip(vals, vals[1:]))                 # peaked at 0, decreasing
    assert all(oracle.kb(t, W) == oracle.kb(-t, W) for t in ts)


@pytest.mark.filterwarnings("ignore::UserWarning")          # quad's round-off notice at this tolerance
@pytest.mark.parametrize("W", [2, 4, 6, 8])
def test_kb_transform_closed_form_equals_quadrature(W):
    # the closed form of c(nu) on both sides of a = beta (sinh and sin branches) against a numerical
    # Fourier integral of the kernel itself
    integrate = pytest.importorskip("scipy.integrate")
    for nu in (0.0, 0.1, 0.25, 0.4, 0.5, 0.7, 1.0, 1.6):
        q, _ = integrate.quad(lambda t: oracle.kb(t, W) * math.cos(2 * math.pi * nu * t), -W / 2, W / 2,
                              epsabs=1e-15, epsrel=1e-13, limit=400)
        assert abs(oracle.kb_ft(nu, W) - q) < 1e-11 + 1e-9 * abs(q), (W, nu)
    assert oracle.kb_ft(0.0, W) == pytest.approx(1.0, rel=1e-15)


def test_grid_kb_spreads_a_visibility_and_its_mirror_over_the_support():
    # two tiles, one cross visibility I at a known continuous cell position: the W x W cells around it hold
    # C(cu - gu) C(cv - gv) I, the mirrored cells the conjugate, nothing else (autos off); W = 2
    n, W, du = 64, 6, 1.0
    enu = np.array([[0.0, 0.0, 0.0], [7.3, -3.6, 0.0]])
    uvw = oracle.uvw(enu, C_LIGHT)              # at nu = c, (u, v) in wavelengths equal the baseline in metres
    gu, gv = uvw[1, 0] / du, uvw[1, 1] / du
    S = np.zeros((3, 4, 2))
    S[1, 0] = (20.0, -8.0)                      # XX of baseline (1, 0)
    S[1, 3] = (12.0, 4.0)                       # YY
    K = 4
    I = complex(20 + 12, -8 + 4) / (2 * K)
    G, Wsum = oracle.grid_kb(S, 2, K, uvw, du, W, n, autos=False)
    assert Wsum == 2.0
    want = np.zeros((n, n), complex)
    cells = 0
    for cv in range(-n // 2, n // 2):
        for cu in range(-n // 2, n // 2):
            if abs(cu - gu) < W / 2 and abs(cv - gv) < W / 2:
                w = oracle.kb(cu - gu, W) * oracle.kb(cv - gv, W)
                want[cv % n, cu % n] += w * I
                want[-cv % n, -cu % n] += w * np.conj(I)
                cells += 1
    assert cells == W * W                       # gu, gv are not integers here
    assert np.allclose(G, want, rtol=0, atol=1e-15)
    assert np.array_equal(G[(-np.arange(n)) % n][:, (-np.arange(n)) % n], np.conj(G))


def test_grid_kb_drops_visibilities_whose_support_leaves_the_grid():
    n, W = 64, 8
    enu = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    S = np.zeros((3, 4, 2))
    S[1, 0] = (8.0, 0.0)
    lim = n / 2 - W / 2
    for g, kept in ((lim, True), (lim * (1 + 1e-12), False), (-lim, True)):
        uvw = oracle.uvw(enu, C_LIGHT) * g      # baseline length 1 m at nu = c: u = g wavelengths
        G, Wsum = oracle.grid_kb(S, 2, 1, uvw, 1.0, W, n, autos=False, pol=oracle.POL_XX)
        assert (Wsum == 2.0) == kept and (np.abs(G).sum() > 0) == kept


def test_kb_point_source_at_phase_centre_keeps_its_flux():
    # identical voltages at every tile: every visibility equals |x|^2 at its true (u, v); the corrected image
    # at the phase centre is sum_c G_c / W, which equals the flux up to the kernel's aliasing: each
    # visibility's weights sum to 1 + 2 sum_n c(n) cos(2 pi n g) per axis (Poisson summation)
    w = bs.build_workload("tiny")
    v = bs.constant_voltages(10, 1, 128, 2, 1)
    for W in (2, 4, 6, 8, 16):
        out = oracle.pipeline(v, w["enu"], w["freqs"], 10, 1, 64, support=W)
        img = out["images"][0]
        a = 2 * sum(abs(oracle.kb_ft(n, W)) for n in range(1, 8))
        assert abs(img[32, 32] - 5.0) <= 5.0 * ((1 + a) ** 2 - 1) + 1e-12, W
        assert img.max() == img[32, 32]
        assert out["W"][0] == 128 * 128


def _direct_dirty_image(I, uvw, W, du, n, n_grid):
    # dirty image as the direct Fourier sum of the visibilities at their exact (u, v) and their mirrors,
    # sampled at pixel (x, y) <-> (l, m) = ((x - N/2), (y - N/2)) / (N_grid du)
    l = (np.arange(n) - n / 2) / (n_grid * du)
    ph_u = np.exp(2j * np.pi * np.outer(uvw[:, 0], l))        # [b][x]
    ph_v = np.exp(2j * np.pi * np.outer(uvw[:, 1], l))        # [b][y]
    a = np.einsum("b,by,bx->yx", I, ph_v, ph_u)
    return 2.0 * a.real / W


@pytest.mark.parametrize("W", [4, 6, 8])
def test_kb_image_approximates_the_direct_fourier_sum(W):
    # Random visibilities of a 24-tile array gridded with the kernel on the 2N grid, transformed, cropped
    # and corrected, against the direct (ungridded) Fourier sum at the same pixels: within the kernel's
    # aliasing error over the whole image.  A swapped axis, a conjugate on the wrong side, a wrong kernel
    # width or shape parameter, a wrong crop or a missing / inverted correction each leave errors of order
    # one; nearest-cell gridding of the same data is an order of magnitude further off.
    n, nt = 64, 24
    enu = bs.tile_positions(nt, 1500.0, 21)
    nu = 150e6
    du = oracle.default_cell(enu, nu, n, support=W)
    uvw = oracle.uvw(enu, nu)
    B = nt * (nt + 1) // 2
    rng = np.random.default_rng(5)
    S = np.zeros((B, 4, 2), dtype=np.int64)
    S[:, 0] = rng.integers(-50, 51, size=(B, 2))
    S[:, 3] = S[:, 0]                           # Stokes I = XX for these sums (K = 1)
    cross = np.array([i != j for i in range(nt) for j in range(i + 1)])
    G, Wsum = oracle.grid_kb(S, nt, 1, uvw, du, W, 2 * n, autos=False)
    assert Wsum == 2 * cross.sum()              # the default cell keeps every baseline
    full, _ = oracle.image(oracle.ifft2(G), Wsum)
    img = oracle.kb_crop_correct(full, W)
    I = (S[:, 0, 0] + 1j * S[:, 0, 1])[cross]
    ref = _direct_dirty_image(I, uvw[cross], Wsum, du, n, 2 * n)
    err = np.abs(img - ref).max() / np.abs(ref).max()
    assert err < {4: 2e-3, 6: 3e-5, 8: 1e-6}[W], err
    iu, iv, keep = oracle.cells(uvw, du, 2 * n)
    Gn, Wn = oracle.grid(S, nt, 1, iu, iv, keep, 2 * n, autos=False)
    fulln, _ = oracle.image(oracle.ifft2(Gn), Wn)
    errn = np.abs(fulln[n // 2:3 * n // 2, n // 2:3 * n // 2] - ref).max() / np.abs(ref).max()
    assert errn > 10 * err


def test_kb_pipeline_matches_stepwise_functions():
    w = bs.build_workload("tiny")
    W = 6
    out = oracle.pipeline(w["volt"], w["enu"], w["freqs"], 10, 1, 64, want_grids=True, support=W)
    S = oracle.correlate(w["volt"], 10, 1)[0, 0]
    du = oracle.default_cell(w["enu"], 154.88e6, 64, support=W)
    G, Wsum = oracle.grid_kb(S, 128, 10, oracle.uvw(w["enu"], 154.88e6), du, W, 128)
    assert np.array_equal(out["grids"][0], G)
    full, _ = oracle.image(oracle.ifft2(G), Wsum)
    assert np.array_equal(out["images"][0], oracle.kb_crop_correct(full, W))
    assert out["W"][0] == 128 * 128


def _dispersed_burst_case(dm=500.0):
    # 16 tiles, 8 channels 20 kHz apart below 155 MHz, 400 integrations of 1 ms (K = 10): a 1 ms burst at the
    # phase centre arriving 5.3 ms into the data at the top channel and later below it by the cold-plasma law
    # 4.148808e3 s MHz^2 DM (nu^-2 - nu_top^-2) (Sec. 2, 7: the FRB search the images feed)
    enu = bs.tile_positions(16, 1500.0, 31)
    freqs = 155e6 - 20e3 * np.arange(8)
    sky = bs.Sky(lmn=np.zeros((0, 3)), power=np.zeros(0), burst_lmn=np.array([0.0, 0.0, 1.0]), burst_power=4.0,
                 burst_dm=dm, burst_t0_s=5.3e-3, burst_width_s=1e-3, burst_f_top_hz=freqs[0])
    volt = bs.voltages(enu, freqs, 4000, sky, seed=33)
    return enu, freqs, volt


def _delays(freqs, dm, t_int=1e-3):
    nu = freqs / 1e6
    return np.rint(4.148808e3 * dm * (nu ** -2 - nu.max() ** -2) / t_int).astype(np.int32)


def test_dedispersion_recovers_the_injected_dispersion_measure():
    # the oracle's images of a dispersed burst, dedispersed at trial DMs 0..1000: the phase-centre peak is
    # largest at the injected DM 500, where it holds most of the burst's power and stands far above the noise
    enu, freqs, volt = _dispersed_burst_case()
    out = oracle.pipeline(volt, enu, freqs, 10, 1, 64, n_threads=4)
    cube = out["images"].reshape(400, 8, 64, 64)
    peaks = {}
    for dm in range(0, 1001, 100):
        series = oracle.dedisperse(cube[:, :, 32, 32], _delays(freqs, dm))
        peaks[dm] = series.max()
    best = max(peaks, key=peaks.get)
    assert best == 500, peaks
    noise = bs.image_noise(2.0, 16, 10) / math.sqrt(8)
    assert peaks[500] > 2.0 and peaks[500] > 20 * noise
    assert peaks[500] > 2 * max(v for k, v in peaks.items() if abs(k - 500) >= 200)


# ----------------------------------------------------------------------------------------------
# phase centre on a pointing direction (Sec. 5.2.3, geometric corrections)
# ----------------------------------------------------------------------------------------------

POINTINGS = [(0.0, 0.0), (0.2, -0.1), (-0.35, 0.25), (0.0, 0.6), (-0.7, 0.0), (1e-9, -2e-9)]


@pytest.mark.parametrize("l0,m0", POINTINGS)
def test_phase_basis_is_the_minimal_rotation_of_east_and_north(l0, m0):
    # against scipy's rotation (an independent library): the rotation about Up x s0 by the angle between Up and
    # s0 carries (E, N, Up) to (e_l, e_m, s0); the basis is orthonormal and right-handed
    Rotation = pytest.importorskip("scipy.spatial.transform").Rotation
    el, em, s0 = oracle.phase_basis(l0, m0)
    n0 = math.sqrt(1 - l0 * l0 - m0 * m0)
    assert np.allclose(s0, [l0, m0, n0], atol=0, rtol=0)
    axis = np.cross([0.0, 0.0, 1.0], s0)
    if np.linalg.norm(axis) > 0:
        rot = Rotation.from_rotvec(axis / np.linalg.norm(axis) * math.atan2(math.hypot(l0, m0), n0))
        E, N, U = rot.apply(np.eye(3))
        assert np.allclose(el, E, atol=1e-12) and np.allclose(em, N, atol=1e-12) and np.allclose(s0, U, atol=1e-12)
    B3 = np.array([el, em, s0])
    assert np.allclose(B3 @ B3.T, np.eye(3), atol=1e-14)
    assert np.allclose(np.cross(el, em), s0, atol=1e-14)
    with pytest.raises(ValueError):
        oracle.phase_basis(0.8, 0.6)


def test_phased_uvw_at_zenith_is_the_plain_uvw_and_keeps_lengths():
    enu = bs.tile_positions(20, 1500.0, 41)
    enu[:, 2] = np.linspace(-3.0, 3.0, 20)      # some height differences
    assert np.array_equal(oracle.uvw_phased(enu, 150e6, 0.0, 0.0), oracle.uvw(enu, 150e6))
    a = oracle.uvw_phased(enu, 150e6, 0.3, -0.2)
    b = oracle.uvw(enu, 150e6)
    assert np.allclose(np.linalg.norm(a, axis=1), np.linalg.norm(b, axis=1), rtol=1e-13, atol=1e-12)
    _, _, s0 = oracle.phase_basis(0.3, -0.2)
    assert np.allclose(a[:, 2], b @ s0, rtol=1e-13, atol=1e-12)     # w = b.s0 nu / c


def test_apply_phase_rotates_by_w_turns():
    rng = np.random.default_rng(3)
    V = rng.normal(size=(6, 4)) + 1j * rng.normal(size=(6, 4))
    uvw = np.zeros((6, 3))
    uvw[:, 2] = [0.0, 0.25, -0.5, 1500.125, -2750.75, 0.1]
    got = oracle.apply_phase(V, uvw)
    want = V * np.exp(2j * np.pi * np.array([0.0, 0.25, -0.5, 0.125, 0.25, 0.1]))[:, None]
    assert np.allclose(got, want, rtol=0, atol=1e-14)


def _source_voltages(enu, nu, lmn, power=20.0, n=40):
    sky = bs.Sky(lmn=np.array([lmn]), power=np.array([power]))
    return bs.voltages(enu, np.array([nu]), n, sky, seed=43, sigma=0.0)


def test_phase_centred_source_lands_in_the_centre_pixel():
    # a noiseless source at the pointing: every phase-centred visibility is its (quantised) power, so the image
    # peaks exactly at the centre pixel with the power the autocorrelations measure (the realised signal power
    # plus the 4-bit rounding's 1/6 per sample); without phase centring it peaks at its offset (l0, m0)
    enu = bs.tile_positions(48, 1500.0, 44)
    nu, n = 154.88e6, 128
    l0, m0 = 0.02, -0.015
    v = _source_voltages(enu, nu, [l0, m0, math.sqrt(1 - l0 * l0 - m0 * m0)])
    out = oracle.pipeline(v, enu, np.array([nu]), 40, 1, n, phase_centre=(l0, m0))
    img = out["images"][0]
    y, x = np.unravel_index(np.argmax(img), img.shape)
    assert (y, x) == (n // 2, n // 2)
    S = oracle.correlate(v, 40, 1)[0, 0]
    autos = np.array([(S[_bidx(i, i), 0, 0] + S[_bidx(i, i), 3, 0]) / 80.0 for i in range(48)])
    assert abs(img[n // 2, n // 2] - autos.mean()) < 0.03 * autos.mean()
    du = oracle.default_cell(enu, nu, n)
    zen = oracle.pipeline(v, enu, np.array([nu]), 40, 1, n)["images"][0]
    y, x = np.unravel_index(np.argmax(zen), zen.shape)
    assert abs(x - (n / 2 + l0 * n * du)) <= 1 and abs(y - (n / 2 + m0 * n * du)) <= 1


def test_offset_source_peaks_at_its_tangent_plane_coordinates():
    # pointing (l0, m0) far from zenith, source a little off it: the peak sits at (s.e_l, s.e_m) in the image
    # plane of the pointing, i.e. pixel (N/2 + (s.e_l) N du, N/2 + (s.e_m) N du)
    enu = bs.tile_positions(48, 1500.0, 45)
    nu, n = 154.88e6, 128
    l0, m0 = 0.3, 0.2
    el, em, s0 = oracle.phase_basis(l0, m0)
    du = oracle.default_cell(enu, nu, n, phase_centre=(l0, m0))
    fov = 1.0 / du
    off = np.array([0.21 * fov, -0.13 * fov])
    s = s0 + off[0] * el + off[1] * em
    s /= np.linalg.norm(s)
    v = _source_voltages(enu, nu, s)
    img = oracle.pipeline(v, enu, np.array([nu]), 40, 1, n, phase_centre=(l0, m0))["images"][0]
    y, x = np.unravel_index(np.argmax(img), img.shape)
    assert abs(x - (n / 2 + (s @ el) * n * du)) <= 1
    assert abs(y - (n / 2 + (s @ em) * n * du)) <= 1


def test_phase_centre_and_kernel_together_keep_the_source_at_the_centre():
    # the kernel spreads the phase-centred visibilities at their exact (u, v) on the pointing's basis: a source
    # at the pointing still peaks at the centre pixel, with the autocorrelations' measured power
    enu = bs.tile_positions(48, 1500.0, 44)
    nu, n = 154.88e6, 128
    l0, m0 = 0.02, -0.015
    v = _source_voltages(enu, nu, [l0, m0, math.sqrt(1 - l0 * l0 - m0 * m0)])
    img = oracle.pipeline(v, enu, np.array([nu]), 40, 1, n, phase_centre=(l0, m0), support=6)["images"][0]
    assert np.unravel_index(np.argmax(img), img.shape) == (n // 2, n // 2)
    S = oracle.correlate(v, 40, 1)[0, 0]
    autos = np.array([(S[_bidx(i, i), 0, 0] + S[_bidx(i, i), 3, 0]) / 80.0 for i in range(48)])
    assert abs(img[n // 2, n // 2] - autos.mean()) < 0.03 * autos.mean()


def test_mean_of_short_integrations_is_the_long_integration_image():
    # gridding and the transform are linear with fixed cells and weights: the mean of four 1 ms images of a
    # channel equals the image of the 4 ms integration (time averaging needs no kernel of its own)
    w = bs.build_workload("coarse", n_samples=40)
    volt, freqs = w["volt"][:, :2], w["freqs"][:2]
    short = oracle.pipeline(volt, w["enu"], freqs, 10, 1, 64)["images"].reshape(4, 2, 64, 64)
    long_ = oracle.pipeline(volt, w["enu"], freqs, 40, 1, 64)["images"]
    assert np.allclose(short.mean(axis=0), long_, rtol=0, atol=1e-12 * np.abs(long_).max())
