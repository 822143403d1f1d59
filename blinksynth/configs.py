"""The five synthetic workloads, shaped like the paper's MWA VCS data (Sec. 5.2.1, Sec. 6.2, Table 1).

Each workload is a set of numbers (tiles, channels, samples, image sizes) plus the seeded recipe that
draws its voltages.  The seed of workload ``n`` (1-based) is ``2505152040 + n``.

=========  =====  ==============================  ===  ====  =====================  =========
name       tiles  channels (output)               K    T     image side             images
=========  =====  ==============================  ===  ====  =====================  =========
tiny       128    1 @ 154.88 MHz                  10   1     256                    1
coarse     128    128 (coarse 121, 10 kHz)        10   100   512                    12,800
precision  144    1 @ 154.88 MHz (3 km disc)      10   1     256 (and 512)          1
uneven     144    4 x 128 (coarse 119-122)        10   50    256/512/1024/512       25,600
fullband   144    24 x 32 @ 40 kHz (109-132)      40   50 per 50 ms chunk, 1000/s  512   38,400 per chunk
=========  =====  ==============================  ===  ====  =====================  =========

K = samples per integration x fine channels averaged; T = integrations of 1 ms.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2505152040


@dataclass
class ImageSet:
    """A contiguous block of fine channels imaged with one flag vector and one image size."""

    fine0: int            # first fine channel (index into the voltage buffer's channel axis)
    n_fine: int           # fine channels in the set
    n_pix: int
    flags: np.ndarray     # uint8 [n_tiles], 1 = flagged


@dataclass
class Workload:
    name: str
    index: int
    n_tiles: int
    radius_m: float
    coarse: list | None          # MWA coarse channel numbers, or None for explicit frequencies
    freqs_hz: list | None        # explicit fine-channel frequencies
    chan_avg: int
    samples_per_int: int
    samples_per_chunk: int
    n_chunks: int
    n_src: int
    n_pix: list                  # one image side per set (per coarse channel, or one for all)
    flag_max_fraction: float = 0.0
    burst: dict | None = None
    description: str = ""

    @property
    def seed(self) -> int:
        return SEED_BASE + self.index

    @property
    def k(self) -> int:
        return self.samples_per_int * self.chan_avg

    def fine_freqs(self) -> np.ndarray:
        from . import fine_frequencies
        if self.freqs_hz is not None:
            return np.asarray(self.freqs_hz, dtype=np.float64)
        return fine_frequencies(self.coarse)

    @property
    def n_fine(self) -> int:
        return len(self.fine_freqs())

    @property
    def n_out_chan(self) -> int:
        return self.n_fine // self.chan_avg

    @property
    def ints_per_chunk(self) -> int:
        return self.samples_per_chunk // self.samples_per_int

    @property
    def images_per_chunk(self) -> int:
        return self.ints_per_chunk * self.n_out_chan

    def sets(self) -> list:
        n_sets = len(self.n_pix)
        per = self.n_fine // n_sets
        out = []
        from . import tile_flags
        for s in range(n_sets):
            if self.flag_max_fraction > 0:
                flags = tile_flags(self.n_tiles, self.flag_max_fraction, self.seed, s)
            else:
                flags = np.zeros(self.n_tiles, dtype=np.uint8)
            out.append(ImageSet(fine0=s * per, n_fine=per, n_pix=self.n_pix[s], flags=flags))
        return out


WORKLOADS = {
    "tiny": Workload(
        name="tiny", index=1, n_tiles=128, radius_m=1500.0, coarse=None, freqs_hz=[154.88e6],
        chan_avg=1, samples_per_int=10, samples_per_chunk=10, n_chunks=1, n_src=3, n_pix=[256],
        description="128 tiles, 1 fine channel at 154.88 MHz, 10 samples -> 1 ms, 3 sources, 256^2, Stokes I"),
    "coarse": Workload(
        name="coarse", index=2, n_tiles=128, radius_m=1500.0, coarse=[121], freqs_hz=None,
        chan_avg=1, samples_per_int=10, samples_per_chunk=1000, n_chunks=1, n_src=10, n_pix=[512],
        description="128 tiles, 1 coarse channel of 128 x 10 kHz, 0.1 s at 1 ms -> 12,800 images of 512^2"),
    "precision": Workload(
        name="precision", index=3, n_tiles=144, radius_m=3000.0, coarse=None, freqs_hz=[154.88e6],
        chan_avg=1, samples_per_int=10, samples_per_chunk=10, n_chunks=1, n_src=3, n_pix=[256],
        description="144 tiles in a 3 km disc, 1 channel, 10 samples, FP8 correlation bit-exact, 256^2 and 512^2"),
    "uneven": Workload(
        name="uneven", index=4, n_tiles=144, radius_m=3000.0, coarse=[119, 120, 121, 122], freqs_hz=None,
        chan_avg=1, samples_per_int=10, samples_per_chunk=500, n_chunks=1, n_src=10,
        n_pix=[256, 512, 1024, 512], flag_max_fraction=0.15,
        description="144 tiles, 0-15% flagged per coarse channel, 4 x 128 channels, 50 ms, mixed image sizes"),
    "fullband": Workload(
        name="fullband", index=5, n_tiles=144, radius_m=3000.0, coarse=list(range(109, 133)), freqs_hz=None,
        chan_avg=4, samples_per_int=10, samples_per_chunk=500, n_chunks=20, n_src=50, n_pix=[512],
        burst={"dm": 500.0, "t0_s": 0.2, "sigmas": 20.0, "width_s": 1e-3, "f_top_hz": 169.6e6},
        description="144 tiles, 24 coarse x 32 channels at 40 kHz (10 kHz averaged by 4), 1 s in 50 ms chunks, "
                    "50 sources + DM 500 burst, 38,400 images of 512^2 per chunk"),
}


def build_workload(name: str, chunk: int = 0, workers: int = 1, n_samples: int | None = None) -> dict:
    """Draw the inputs of one chunk of a workload.

    Returns a dict with ``enu`` [n_tiles][3] float64, ``freqs`` [n_fine] float64, ``volt``
    uint8 [S][n_fine][n_tiles][2], ``sets`` (list of :class:`ImageSet`), ``sky`` and the workload.
    ``n_samples`` (a multiple of samples_per_int) truncates the chunk for quick tests.
    """
    from . import image_noise, make_sky, tile_positions, voltages
    w = WORKLOADS[name]
    enu = tile_positions(w.n_tiles, w.radius_m, w.seed)
    freqs = w.fine_freqs()
    sigma_img = image_noise(2.0, w.n_tiles, w.k)
    sky = make_sky(w.n_src, sigma_img, w.seed, burst=w.burst)
    s = w.samples_per_chunk if n_samples is None else n_samples
    volt = voltages(enu, freqs, s, sky, w.seed, chunk=chunk, sample0=chunk * w.samples_per_chunk,
                    workers=workers)
    return {"workload": w, "enu": enu, "freqs": freqs, "volt": volt, "sets": w.sets(), "sky": sky,
            "sigma_img": sigma_img, "chunk": chunk}
