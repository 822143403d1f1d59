"""Seeded synthetic inputs shaped like MWA VCS voltage data.

This module is shared by the CUDA path and by the CPU oracle, and it holds none of the imaging
method's arithmetic (no correlation, no uvw, no gridding, no Fourier transform).  It only draws:

* tile positions (East, North, Up in metres), uniform in a disc, flat (Up = 0);
* fine-channel centre frequencies laid out like MWA coarse channels (1.28 MHz coarse channels of
  128 x 10 kHz fine channels, the VCS format of Sec. 5.2.1 of the paper);
* a sky of point sources within 20 degrees of zenith and an optional dispersed 1 ms burst;
* complex voltages per (sample, fine channel, tile, polarisation): circular Gaussian noise of
  standard deviation ``sigma`` per component plus the sources, each source's signal identical at
  every tile up to its geometric phase;

and quantises them to signed 4-bit integers packed one complex sample per byte:
``byte = (re & 0xF) | ((im & 0xF) << 4)`` (two's complement nibbles, re in the low nibble).

The packed buffer layout is ``uint8 [n_samples][n_fine][n_tiles][2]`` (last axis = X, Y polarisation).

Every random stream is keyed by (seed, chunk index, fine channel), so the bytes of a chunk do not
depend on how many worker processes produced them.
"""
from __future__ import annotations

import math
import multiprocessing as mp
from dataclasses import dataclass, field

import numpy as np

# Speed of light used by the generator to place source wavefronts (m/s).
_C_LIGHT_M_S = 299_792_458.0
# Cold-plasma dispersion constant, s MHz^2 pc^-1 cm^3 (standard pulsar-timing value).
_K_DM = 4.148808e3

COARSE_WIDTH_HZ = 1.28e6
FINE_PER_COARSE = 128
FINE_WIDTH_HZ = 10e3
SAMPLE_TIME_S = 100e-6


def tile_positions(n_tiles: int, radius_m: float, seed: int) -> np.ndarray:
    """Tile (E, N, U) positions in metres, uniform in a disc of ``radius_m``; U = 0."""
    g = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, 1])))
    r = radius_m * np.sqrt(g.random(n_tiles))
    th = 2.0 * np.pi * g.random(n_tiles)
    enu = np.zeros((n_tiles, 3), dtype=np.float64)
    enu[:, 0] = r * np.cos(th)
    enu[:, 1] = r * np.sin(th)
    return enu


def fine_frequencies(coarse_channels, n_fine: int = FINE_PER_COARSE) -> np.ndarray:
    """Centre frequencies (Hz) of the fine channels of MWA coarse channels.

    Coarse channel ``n`` is centred at ``n * 1.28 MHz``; its fine channel ``k`` (of 128, 10 kHz each)
    is centred at ``f_cc - 640 kHz + (k + 1/2) * 10 kHz``.
    """
    out = []
    for n in coarse_channels:
        fcc = n * COARSE_WIDTH_HZ
        k = np.arange(n_fine, dtype=np.float64)
        out.append(fcc - COARSE_WIDTH_HZ / 2 + (k + 0.5) * FINE_WIDTH_HZ)
    return np.concatenate(out)


def tile_flags(n_tiles: int, max_fraction: float, seed: int, key: int) -> np.ndarray:
    """A seeded flag vector (1 = flagged) with a fraction of flagged tiles drawn in [0, max_fraction]."""
    g = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, 2, key])))
    n_flag = int(round(g.random() * max_fraction * n_tiles))
    flags = np.zeros(n_tiles, dtype=np.uint8)
    if n_flag:
        flags[g.choice(n_tiles, size=n_flag, replace=False)] = 1
    return flags


@dataclass
class Sky:
    """Point sources (and an optional dispersed burst) as direction cosines and power per polarisation."""

    lmn: np.ndarray            # [n_src][3] direction cosines toward (E, N, Up)
    power: np.ndarray          # [n_src] mean |s|^2 per polarisation and sample
    burst_lmn: np.ndarray | None = None
    burst_power: float = 0.0
    burst_dm: float = 0.0      # pc cm^-3
    burst_t0_s: float = 0.0    # arrival time at the top of the band
    burst_width_s: float = 1e-3
    burst_f_top_hz: float = 0.0


def image_noise(sigma: float, n_tiles: int, k: int, stokes_i: bool = True) -> float:
    """Dirty-image noise level of pure-noise voltages, P_n = 2 sigma^2 the noise power per sample.

    One polarisation: P_n / sqrt(2 N_cross K).  Stokes I averages two independent polarisations, which
    divides that by sqrt(2).  This is the scale in which source fluxes are quoted ("5-20 sigma").
    """
    p_n = 2.0 * sigma * sigma
    n_cross = n_tiles * (n_tiles - 1) // 2
    s = p_n / math.sqrt(2.0 * n_cross * k)
    return s / math.sqrt(2.0) if stokes_i else s


def random_directions(n: int, g: np.random.Generator, max_zenith_deg: float) -> np.ndarray:
    cmin = math.cos(math.radians(max_zenith_deg))
    cz = cmin + (1.0 - cmin) * g.random(n)
    sz = np.sqrt(1.0 - cz * cz)
    az = 2.0 * np.pi * g.random(n)
    return np.stack([sz * np.sin(az), sz * np.cos(az), cz], axis=1)


def make_sky(n_src: int, sigma_img: float, seed: int, max_zenith_deg: float = 20.0,
             flux_sigmas=(5.0, 20.0), burst: dict | None = None) -> Sky:
    g = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, 3])))
    lmn = random_directions(n_src, g, max_zenith_deg)
    power = sigma_img * g.uniform(flux_sigmas[0], flux_sigmas[1], size=n_src)
    sky = Sky(lmn=lmn, power=power)
    if burst is not None:
        sky.burst_lmn = random_directions(1, g, max_zenith_deg)[0]
        sky.burst_power = burst["sigmas"] * sigma_img
        sky.burst_dm = burst["dm"]
        sky.burst_t0_s = burst["t0_s"]
        sky.burst_width_s = burst.get("width_s", 1e-3)
        sky.burst_f_top_hz = burst["f_top_hz"]
    return sky


def quantise_pack(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """clamp(round-half-away-from-zero(x), -8, 7) per component, packed (re | im << 4)."""
    def q(x):
        r = np.where(x >= 0, np.floor(x + 0.5), np.ceil(x - 0.5))
        return np.clip(r, -8, 7).astype(np.int16)
    return ((q(re) & 0xF) | ((q(im) & 0xF) << 4)).astype(np.uint8)


def _channel_block(args):
    (seed, chunk, ch, freq, enu, sky, n_samples, sample0, sigma) = args
    g = np.random.Generator(np.random.Philox(np.random.SeedSequence([seed, 4, chunk, ch])))
    n_tiles = enu.shape[0]
    # noise [S][tile][pol]
    re = g.standard_normal((n_samples, n_tiles, 2), dtype=np.float32) * np.float32(sigma)
    im = g.standard_normal((n_samples, n_tiles, 2), dtype=np.float32) * np.float32(sigma)
    n_src = sky.lmn.shape[0]
    if n_src:
        # geometric phase of each source at each tile: exp(-2 pi i nu (r . s) / c)
        delay = enu @ sky.lmn.T / _C_LIGHT_M_S                      # [tile][src] seconds
        ph = np.exp(-2j * np.pi * freq * delay)                     # [tile][src]
        amp = np.sqrt(sky.power / 2.0)                              # per real component
        sig = (g.standard_normal((n_samples, 2, n_src)) + 1j * g.standard_normal((n_samples, 2, n_src))) * amp
        x = np.einsum("tps,as->tap", sig, ph)                       # [S][tile][pol]
        re += x.real.astype(np.float32)
        im += x.imag.astype(np.float32)
    if sky.burst_lmn is not None and sky.burst_power > 0:
        f_mhz = freq / 1e6
        t_arr = sky.burst_t0_s + _K_DM * sky.burst_dm * (f_mhz ** -2 - (sky.burst_f_top_hz / 1e6) ** -2)
        t = (sample0 + np.arange(n_samples) + 0.5) * SAMPLE_TIME_S
        on = (t >= t_arr) & (t < t_arr + sky.burst_width_s)
        if on.any():
            delay = enu @ sky.burst_lmn / _C_LIGHT_M_S
            ph = np.exp(-2j * np.pi * freq * delay)                 # [tile]
            amp = math.sqrt(sky.burst_power / 2.0)
            n_on = int(on.sum())
            sig = (g.standard_normal((n_on, 2)) + 1j * g.standard_normal((n_on, 2))) * amp
            x = sig[:, None, :] * ph[None, :, None]
            re[on] += x.real.astype(np.float32)
            im[on] += x.imag.astype(np.float32)
    return ch, quantise_pack(re, im)                                # [S][tile][pol]


def voltages(enu: np.ndarray, freqs: np.ndarray, n_samples: int, sky: Sky, seed: int, chunk: int = 0,
             sample0: int = 0, sigma: float = 2.0, workers: int = 1) -> np.ndarray:
    """Packed 4-bit voltages ``uint8 [n_samples][n_fine][n_tiles][2]`` for one chunk of samples.

    ``sample0`` is the absolute index of the chunk's first sample (used for the burst arrival time);
    the random streams are keyed by (seed, chunk, fine channel).
    """
    n_fine = len(freqs)
    n_tiles = enu.shape[0]
    out = np.empty((n_samples, n_fine, n_tiles, 2), dtype=np.uint8)
    jobs = [(seed, chunk, ch, float(freqs[ch]), enu, sky, n_samples, sample0, sigma) for ch in range(n_fine)]
    if workers > 1 and n_fine > 1:
        ctx = mp.get_context("spawn")
        with ctx.Pool(workers) as pool:
            for ch, blk in pool.imap_unordered(_channel_block, jobs, chunksize=max(1, n_fine // (8 * workers))):
                out[:, ch] = blk
    else:
        for job in jobs:
            ch, blk = _channel_block(job)
            out[:, ch] = blk
    return out


def constant_voltages(n_samples: int, n_fine: int, n_tiles: int, re: int, im: int) -> np.ndarray:
    """Every sample of every tile and polarisation equal to ``re + i im`` (for closed-form checks)."""
    b = quantise_pack(np.float64(re), np.float64(im))
    return np.full((n_samples, n_fine, n_tiles, 2), b, dtype=np.uint8)


def pack_complex(x: np.ndarray) -> np.ndarray:
    """Pack an integer-valued complex array (values in [-8, 7]) into the 4-bit byte format."""
    return quantise_pack(np.real(x).astype(np.float64), np.imag(x).astype(np.float64))


def unpack_reference(b: np.ndarray) -> np.ndarray:
    """Inverse of :func:`pack_complex` (two's-complement nibbles -> complex integers)."""
    b = b.astype(np.int16)
    re = b & 0xF
    im = (b >> 4) & 0xF
    re = np.where(re >= 8, re - 16, re)
    im = np.where(im >= 8, im - 16, im)
    return re + 1j * im


from .configs import WORKLOADS, Workload, build_workload  # noqa: E402,F401
