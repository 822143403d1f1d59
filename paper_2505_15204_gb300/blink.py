"""Thin Python binding of the C ABI in ``include/blink.h`` (argument marshalling only).

Every function has the name of the C entry point it calls.  Device buffers are passed as torch CUDA
tensors (or raw integer device pointers); descriptor structs are built from numpy arrays that this
module keeps alive for the duration of the call.  A non-OK status raises :class:`BlinkError`.

There is no fallback: if the compiled library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libblink.so")

BLINK_OK = 0
BLINK_ERR_INVALID_ARG = 1
BLINK_ERR_UNSUPPORTED = 2
BLINK_ERR_OOM = 3
BLINK_ERR_CUDA = 4
BLINK_ERR_TIMEOUT = 5
BLINK_ERR_DEVICE = 6

BLINK_POL_I = 0
BLINK_POL_XX = 1
BLINK_CORR_FP32 = 0
BLINK_CORR_FP8 = 1
BLINK_PREC_FP32 = 0
BLINK_PREC_BF16 = 1
BLINK_MODE_BATCHED = 0
BLINK_MODE_PLAIN = 1

# every entry point declared in include/blink.h
ENTRY_POINTS = (
    "blink_create", "blink_destroy", "blink_last_error", "blink_status_name", "blink_sync", "blink_n_baselines",
    "blink_cells", "blink_correlate", "blink_grid", "blink_image", "blink_pipeline", "blink_pipeline_host",
    "blink_set_profiling", "blink_read_profile", "blink_image_noalloc", "blink_pipeline_sets", "blink_dedisperse",
    "blink_set_wait_budget", "blink_set_fused", "blink_tuned_shape", "blink_pipeline_tracking",
    "blink_pipeline_averaged", "blink_dedisperse_stream",
)
BLINK_STAGE_CORRELATE = 0
BLINK_STAGE_GRID_FFT = 1
BLINK_STAGE_ROW_FFT = 2
BLINK_STAGE_FUSED = 3
BLINK_N_STAGES = 4


class BlinkError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


class blink_array(C.Structure):
    _fields_ = [("n_tiles", C.c_int32), ("enu_m", C.c_void_p), ("flags", C.c_void_p), ("gains", C.c_void_p),
                ("jones", C.c_void_p)]


class blink_obs(C.Structure):
    _fields_ = [("n_fine", C.c_int32), ("fine_stride", C.c_int32), ("fine_freq_hz", C.c_void_p),
                ("chan_avg", C.c_int32), ("samples_per_int", C.c_int32), ("n_samples", C.c_int32)]


class blink_imaging(C.Structure):
    _fields_ = [("n_pix", C.c_int32), ("cell_lambda", C.c_double), ("pol", C.c_int32),
                ("include_autos", C.c_int32), ("precision", C.c_int32), ("support", C.c_int32),
                ("phase_l", C.c_double), ("phase_m", C.c_double)]


class blink_set(C.Structure):
    _fields_ = [("fine0", C.c_int32), ("n_fine", C.c_int32), ("flags", C.c_void_p), ("imaging", blink_imaging)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
    lib = C.CDLL(LIB_PATH)
    P, I32, I64, S = C.c_void_p, C.c_int32, C.c_int64, C.c_int
    sig = {
        "blink_create": (S, [I32, C.POINTER(C.c_void_p)]),
        "blink_destroy": (None, [P]),
        "blink_last_error": (C.c_char_p, []),
        "blink_status_name": (C.c_char_p, [S]),
        "blink_sync": (S, [P, P]),
        "blink_n_baselines": (I64, [I32]),
        "blink_cells": (S, [P, P, P, P, P, P, P, P]),
        "blink_correlate": (S, [P, P, P, I32, P, P, P]),
        "blink_grid": (S, [P, P, P, P, P, I32, I32, P, P, P]),
        "blink_image": (S, [P, P, P, I32, P, P, P]),
        "blink_pipeline": (S, [P, P, P, P, I32, I32, P, P, P, P]),
        "blink_pipeline_host": (S, [P, P, P, P, I32, P, P, I32, P]),
        "blink_set_profiling": (S, [P, I32]),
        "blink_read_profile": (S, [P, P, P, P, I32]),
        "blink_image_noalloc": (S, [P, P, I32, P, P, P]),
        "blink_pipeline_sets": (S, [P, P, P, P, I32, I32, P, P, C.c_size_t, P]),
        "blink_dedisperse": (S, [P, P, I32, I32, I32, P, P, P]),
        "blink_set_wait_budget": (S, [P, I64, I32]),
        "blink_set_fused": (S, [P, I32]),
        "blink_tuned_shape": (S, [P, P]),
        "blink_pipeline_tracking": (S, [P, P, P, P, P, I32, P, P, P]),
        "blink_pipeline_averaged": (S, [P, P, P, P, I32, I32, I32, P, P, P]),
        "blink_dedisperse_stream": (S, [P, P, I64, P, I32, I32, I32, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def _ptr(x):
    """Device or host address of a torch tensor, numpy array or integer (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(status: int, where: str):
    if status != BLINK_OK:
        raise BlinkError(status, where, _lib.blink_last_error().decode())


# ---- descriptors ------------------------------------------------------------------------------------

@dataclass
class Array:
    enu_m: np.ndarray
    flags: np.ndarray | None = None
    gains: np.ndarray | None = None      # complex [F][n_tiles][2] per output channel, tile, polarisation
    jones: np.ndarray | None = None      # complex [F][n_tiles][2][2] full Jones matrices J[p][r]

    def c(self):
        self._enu = np.ascontiguousarray(self.enu_m, dtype=np.float64)
        self._flags = None if self.flags is None else np.ascontiguousarray(self.flags, dtype=np.uint8)

        def pack(z):
            if z is None:
                return None
            z = np.asarray(z)
            return np.ascontiguousarray(np.stack([z.real, z.imag], axis=-1), dtype=np.float32)

        self._gains, self._jones = pack(self.gains), pack(self.jones)
        return blink_array(self._enu.shape[0], self._enu.ctypes.data,
                           None if self._flags is None else self._flags.ctypes.data,
                           None if self._gains is None else self._gains.ctypes.data,
                           None if self._jones is None else self._jones.ctypes.data)


@dataclass
class Obs:
    fine_freq_hz: np.ndarray
    chan_avg: int
    samples_per_int: int
    n_samples: int
    fine_stride: int = 0

    def c(self):
        self._f = np.ascontiguousarray(self.fine_freq_hz, dtype=np.float64)
        return blink_obs(len(self._f), self.fine_stride, self._f.ctypes.data, self.chan_avg, self.samples_per_int,
                         self.n_samples)


@dataclass
class Imaging:
    n_pix: int
    cell_lambda: float = 0.0
    pol: int = BLINK_POL_I
    include_autos: int = 1
    precision: int = BLINK_PREC_FP32
    support: int = 0                     # 0: nearest cell; W >= 2: Kaiser-Bessel kernel of W cells
    phase_centre: tuple = (0.0, 0.0)     # pointing (l0, m0) in the local East, North, Up frame; (0, 0) = zenith

    def c(self):
        l0, m0 = self.phase_centre
        return blink_imaging(self.n_pix, self.cell_lambda, self.pol, self.include_autos, self.precision,
                             self.support, float(l0), float(m0))


def _ref(x):
    return None if x is None else C.byref(x)


# ---- entry points -----------------------------------------------------------------------------------

def blink_create(device: int = 0) -> int:
    out = C.c_void_p()
    _check(_lib.blink_create(device, C.byref(out)), "blink_create")
    return out.value


def blink_destroy(ctx) -> None:
    _lib.blink_destroy(ctx)


def blink_last_error() -> str:
    return _lib.blink_last_error().decode()


def blink_status_name(status: int) -> str:
    return _lib.blink_status_name(status).decode()


def blink_sync(ctx, stream=None) -> None:
    _check(_lib.blink_sync(ctx, _stream(stream)), "blink_sync")


def blink_n_baselines(n_tiles: int) -> int:
    return int(_lib.blink_n_baselines(n_tiles))


def blink_cells(ctx, array: Array, obs: Obs, imaging: Imaging, d_cells, d_uvw=None, stream=None) -> float:
    du = C.c_double(0.0)
    a, o, i = array.c(), obs.c(), imaging.c()
    _check(_lib.blink_cells(ctx, C.byref(a), C.byref(o), C.byref(i), _ptr(d_cells), _ptr(d_uvw), C.byref(du),
                            _stream(stream)), "blink_cells")
    return du.value


def blink_correlate(ctx, array: Array, obs: Obs, arith: int, d_volt, d_vis, stream=None) -> None:
    a, o = array.c(), obs.c()
    _check(_lib.blink_correlate(ctx, C.byref(a), C.byref(o), arith, _ptr(d_volt), _ptr(d_vis), _stream(stream)),
           "blink_correlate")


def blink_grid(ctx, array: Array, obs: Obs, imaging: Imaging, d_vis, first_image: int, n_images: int, d_grid,
               d_weight=None, stream=None) -> None:
    a, o, i = array.c(), obs.c(), imaging.c()
    _check(_lib.blink_grid(ctx, C.byref(a), C.byref(o), C.byref(i), _ptr(d_vis), first_image, n_images,
                           _ptr(d_grid), _ptr(d_weight), _stream(stream)), "blink_grid")


def blink_image(ctx, imaging: Imaging, d_grid, n_images: int, d_weight, d_img, stream=None) -> None:
    i = imaging.c()
    _check(_lib.blink_image(ctx, C.byref(i), _ptr(d_grid), n_images, _ptr(d_weight), _ptr(d_img), _stream(stream)),
           "blink_image")


def blink_pipeline(ctx, array: Array, obs: Obs, imaging: Imaging, arith: int, mode: int, d_volt, d_img,
                   d_weight=None, stream=None) -> None:
    a, o, i = array.c(), obs.c(), imaging.c()
    _check(_lib.blink_pipeline(ctx, C.byref(a), C.byref(o), C.byref(i), arith, mode, _ptr(d_volt), _ptr(d_img),
                               _ptr(d_weight), _stream(stream)), "blink_pipeline")


def blink_pipeline_host(ctx, array: Array, obs: Obs, imaging: Imaging, arith: int, h_volt, h_img,
                        images_per_pass: int = 0, stream=None) -> None:
    a, o, i = array.c(), obs.c(), imaging.c()
    _check(_lib.blink_pipeline_host(ctx, C.byref(a), C.byref(o), C.byref(i), arith, _ptr(h_volt), _ptr(h_img),
                                    images_per_pass, _stream(stream)), "blink_pipeline_host")


def blink_pipeline_tracking(ctx, array: Array, obs: Obs, imaging: Imaging, lm, arith: int, d_volt, d_img,
                            stream=None) -> None:
    """Batched pipeline with one phase centre per integration: lm = (l, m) per integration, [T][2]."""
    a, o, i = array.c(), obs.c(), imaging.c()
    t = np.ascontiguousarray(lm, dtype=np.float64)
    if t.ndim != 2 or t.shape[1] != 2:
        raise ValueError("lm must be [T][2]")
    _check(_lib.blink_pipeline_tracking(ctx, C.byref(a), C.byref(o), C.byref(i), t.ctypes.data, arith, _ptr(d_volt),
                                        _ptr(d_img), _stream(stream)), "blink_pipeline_tracking")


def blink_pipeline_averaged(ctx, array: Array, obs: Obs, imaging: Imaging, arith: int, t_avg: int, f_avg: int,
                            d_volt, d_img, stream=None) -> None:
    """Mean images over t_avg integrations and f_avg output channels: d_img [T/t_avg][F/f_avg][N][N]."""
    a, o, i = array.c(), obs.c(), imaging.c()
    _check(_lib.blink_pipeline_averaged(ctx, C.byref(a), C.byref(o), C.byref(i), arith, int(t_avg), int(f_avg),
                                        _ptr(d_volt), _ptr(d_img), _stream(stream)), "blink_pipeline_averaged")


def blink_dedisperse(ctx, d_img, n_int: int, n_chan: int, n_pix: int, delays, d_out, stream=None) -> None:
    """Dedispersed channel means of an image cube [n_int][n_chan][N][N] into [n_int - max(delays)][N][N]."""
    d = np.ascontiguousarray(delays, dtype=np.int32)
    if d.shape != (n_chan,):
        raise ValueError("delays must have one entry per channel")
    _check(_lib.blink_dedisperse(ctx, _ptr(d_img), n_int, n_chan, n_pix, d.ctypes.data, _ptr(d_out), _stream(stream)),
           "blink_dedisperse")


def blink_dedisperse_stream(ctx, d_carry, t0: int, d_img, n_int: int, n_chan: int, n_pix: int, delays, d_out,
                            stream=None) -> int:
    """One cube [n_int][n_chan][N][N] of a stream starting at integration t0; writes the outputs it completes
    to d_out and returns their count (the carry d_carry [max(delays)][N][N] links consecutive calls)."""
    d = np.ascontiguousarray(delays, dtype=np.int32)
    if d.shape != (n_chan,):
        raise ValueError("delays must have one entry per channel")
    n_out = C.c_int32(0)
    _check(_lib.blink_dedisperse_stream(ctx, _ptr(d_carry), int(t0), _ptr(d_img), n_int, n_chan, n_pix, d.ctypes.data,
                                        _ptr(d_out), C.byref(n_out), _stream(stream)), "blink_dedisperse_stream")
    return int(n_out.value)


def blink_set_profiling(ctx, enable: bool) -> None:
    _check(_lib.blink_set_profiling(ctx, int(bool(enable))), "blink_set_profiling")


def blink_read_profile(ctx, stream=None, reset: bool = True):
    """Per-stage (ms, launches) summed over the recorded pipeline launches, as two lists."""
    ms = (C.c_double * BLINK_N_STAGES)()
    n = (C.c_int64 * BLINK_N_STAGES)()
    _check(_lib.blink_read_profile(ctx, _stream(stream), ms, n, int(bool(reset))), "blink_read_profile")
    return list(ms), list(n)


def blink_set_wait_budget(ctx, budget_cycles: int = 0, unreachable: bool = False) -> None:
    """Budget (SM clock cycles, 0 = default) of the imaging kernel's dependency waits; `unreachable` makes
    the row tasks' waits run out (a test of the failure path)."""
    _check(_lib.blink_set_wait_budget(ctx, int(budget_cycles), int(bool(unreachable))), "blink_set_wait_budget")


def blink_set_fused(ctx, enable: bool = True) -> None:
    """Correlation inside the side-512 imaging launch, or as its own launch (the default)."""
    _check(_lib.blink_set_fused(ctx, int(bool(enable))), "blink_set_fused")


def blink_tuned_shape(ctx):
    """(ring slots, lag, CTAs per SM) the autotuner kept for the most recent plan; zeros before tuning."""
    out = (C.c_int32 * 3)()
    _check(_lib.blink_tuned_shape(ctx, out), "blink_tuned_shape")
    return tuple(out)


def blink_image_noalloc(imaging: Imaging, d_grid, n_images: int, d_weight, d_img, stream=None) -> None:
    """blink_image without a context and without device allocation (static scratch, current device)."""
    i = imaging.c()
    _check(_lib.blink_image_noalloc(C.byref(i), _ptr(d_grid), n_images, _ptr(d_weight), _ptr(d_img),
                                    _stream(stream)), "blink_image_noalloc")


@dataclass
class Set:
    fine0: int
    n_fine: int
    imaging: Imaging
    flags: np.ndarray | None = None


def blink_pipeline_sets(ctx, array: Array, obs: Obs, sets, arith: int, d_volt, d_img, img_capacity: int,
                        stream=None) -> None:
    """Several channel sets, each with its own flags and image parameters; images packed per set."""
    a, o = array.c(), obs.c()
    keep = [None if s.flags is None else np.ascontiguousarray(s.flags, dtype=np.uint8) for s in sets]
    arr = (blink_set * len(sets))()
    for q, (s, fl) in enumerate(zip(sets, keep)):
        arr[q] = blink_set(s.fine0, s.n_fine, None if fl is None else fl.ctypes.data, s.imaging.c())
    _check(_lib.blink_pipeline_sets(ctx, C.byref(a), C.byref(o), arr, len(sets), arith, _ptr(d_volt), _ptr(d_img),
                                    img_capacity, _stream(stream)), "blink_pipeline_sets")
