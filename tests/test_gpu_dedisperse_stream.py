"""Streaming incoherent dedispersion (Sec. 2 and 7: a dispersive sweep outlasts one cube of images) against the
oracle's dedispersion of the whole concatenated cube.  The stream is cut into cubes shorter than, equal to and
longer than the largest delay, and the outputs each call completes are compared in order."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


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


def _stream(B, ctx, cube, delays, cuts, carry):
    """Pass cube [T][F][n][n] in pieces of the given lengths; return the concatenated outputs and the counts."""
    T, F, n, _ = cube.shape
    outs, counts, t0 = [], [], 0
    for m in cuts:
        img = torch.from_numpy(np.ascontiguousarray(cube[t0:t0 + m])).cuda()
        out = torch.full((m, n, n), np.nan, dtype=torch.float32, device="cuda")
        k = B.blink_dedisperse_stream(ctx, carry, t0, img, m, F, n, delays, out)
        B.blink_sync(ctx)
        counts.append(k)
        outs.append(out[:k].cpu().numpy())
        t0 += m
    assert t0 == T
    return np.concatenate(outs), counts


@pytest.mark.parametrize("cuts", [[3, 5, 10, 2, 12], [1] * 16 + [16], [32], [7, 7, 7, 11]])
def test_streamed_cubes_equal_oracle_on_the_whole_cube(B, ctx, cuts):
    rng = np.random.default_rng(7)
    T, F, n = 32, 13, 64                              # F not a multiple of the kernel's unroll
    cube = rng.normal(size=(T, F, n, n)).astype(np.float32)
    d = np.array([0, 7, 1, 4, 2, 0, 6, 5, 3, 2, 0, 1, 2], dtype=np.int32)
    D = int(d.max())
    carry = torch.empty((D, n, n), dtype=torch.float32, device="cuda")
    carry.fill_(np.nan)                               # ignored by the first call (t0 = 0)
    got, counts = _stream(B, ctx, cube, d, cuts, carry)
    ref = oracle.dedisperse(cube.astype(np.float64), d)
    assert got.shape == ref.shape == (T - D, n, n)
    # each call completes the outputs t in [max(0, t0 - D), t0 + m - D)
    t0, want = 0, []
    for m in cuts:
        want.append(max(0, t0 + m - D - max(0, t0 - D)))
        t0 += m
    assert counts == want
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()


def test_zero_delays_stream_is_the_band_mean_of_each_cube(B, ctx):
    rng = np.random.default_rng(8)
    T, F, n = 6, 5, 64
    cube = rng.normal(size=(T, F, n, n)).astype(np.float32)
    d = np.zeros(F, np.int32)
    got, counts = _stream(B, ctx, cube, d, [2, 1, 3], None)       # no carry is needed
    assert counts == [2, 1, 3]
    ref = oracle.dedisperse(cube.astype(np.float64), d)
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()


def test_streamed_pulse_is_recovered_across_cube_boundaries(B, ctx):
    # a pulse at output integration 9 dispersed over 16 channels with delays up to 15 integrations, passed in
    # cubes of 4: every channel's share sits in a different cube from most others
    T, F, n = 28, 16, 64
    d = np.arange(F, dtype=np.int32)[::-1].copy()
    cube = np.zeros((T, F, n, n), np.float32)
    for f in range(F):
        cube[9 + d[f], f, 20, 30] = 3.0
    D = int(d.max())
    carry = torch.empty((D, n, n), dtype=torch.float32, device="cuda")
    got, _ = _stream(B, ctx, cube, d, [4] * 7, carry)
    assert got.shape == (T - D, n, n)
    assert got[9, 20, 30] == pytest.approx(3.0, rel=1e-6)
    got[9, 20, 30] = 0.0
    assert np.abs(got).max() == 0.0
