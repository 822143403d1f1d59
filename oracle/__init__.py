"""CPU oracle for the BLINK dirty-imaging hot path (arXiv 2505.15204).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
are the only callers.  The product library never imports this package and shares no code with it.

The arithmetic lives in ``blink_oracle.c`` (plain loops, int64 correlation, FP64 geometry, gridding and
FFT); this module compiles it with gcc on first use and wraps it with numpy arrays.  See the C file's
header for the equation each function follows.

Every function here is pinned by ``tests/test_oracle_pins.py`` against closed forms, invariants, a
brute-force direct DFT, an independent library FFT and the paper's data-volume table.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "blink_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

POL_I = 0
POL_XX = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, -ffp-contract=off, OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.oracle_n_baselines.restype = C.c_int64
            lib.oracle_n_baselines.argtypes = [C.c_int]
            lib.oracle_correlate.restype = None
            lib.oracle_correlate.argtypes = [P, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P, P]
            lib.oracle_correlate_one.restype = None
            lib.oracle_correlate_one.argtypes = [P, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P, P]
            lib.oracle_output_freqs.restype = None
            lib.oracle_output_freqs.argtypes = [P, C.c_int, C.c_int, P]
            lib.oracle_uvw.restype = None
            lib.oracle_uvw.argtypes = [P, C.c_int, C.c_double, P]
            lib.oracle_default_cell.restype = C.c_double
            lib.oracle_default_cell.argtypes = [P, C.c_int, P, C.c_double, C.c_int, C.c_int, C.c_double, C.c_double]
            lib.oracle_phase_basis.restype = C.c_int
            lib.oracle_phase_basis.argtypes = [C.c_double, C.c_double, P, P, P]
            lib.oracle_uvw_phased.restype = C.c_int
            lib.oracle_uvw_phased.argtypes = [P, C.c_int, C.c_double, C.c_double, C.c_double, P]
            lib.oracle_apply_phase.restype = None
            lib.oracle_apply_phase.argtypes = [P, P, C.c_int64]
            lib.oracle_image_pixels.restype = None
            lib.oracle_image_pixels.argtypes = [P, C.c_int, C.c_double, P, C.c_int64, P]
            lib.oracle_cells.restype = None
            lib.oracle_cells.argtypes = [P, C.c_int64, C.c_double, C.c_int, P, P, P]
            lib.oracle_grid.restype = C.c_double
            lib.oracle_grid.argtypes = [P, C.c_int, P, C.c_int, C.c_int, C.c_int, P, P, P, C.c_int, P]
            lib.oracle_ifft2.restype = C.c_int
            lib.oracle_ifft2.argtypes = [P, C.c_int]
            lib.oracle_idft2.restype = None
            lib.oracle_idft2.argtypes = [P, C.c_int, P]
            lib.oracle_image.restype = C.c_double
            lib.oracle_image.argtypes = [P, C.c_int, C.c_double, P]
            lib.oracle_pipeline.restype = C.c_int
            lib.oracle_pipeline.argtypes = [P, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int, P, P, P,
                                            C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, C.c_double,
                                            C.c_double, P, C.c_int, P, C.c_int64, C.c_int, P, P, P, P]
            lib.oracle_i0.restype = C.c_double
            lib.oracle_i0.argtypes = [C.c_double]
            lib.oracle_kb_beta.restype = C.c_double
            lib.oracle_kb_beta.argtypes = [C.c_int]
            lib.oracle_kb.restype = C.c_double
            lib.oracle_kb.argtypes = [C.c_double, C.c_int, C.c_double]
            lib.oracle_kb_ft.restype = C.c_double
            lib.oracle_kb_ft.argtypes = [C.c_double, C.c_int, C.c_double]
            lib.oracle_grid_kb.restype = C.c_double
            lib.oracle_grid_kb.argtypes = [P, C.c_int, P, C.c_int, C.c_int, C.c_int, P, C.c_double, C.c_int,
                                           C.c_int, P]
            lib.oracle_kb_crop_correct.restype = None
            lib.oracle_kb_crop_correct.argtypes = [P, C.c_int, C.c_int, P]
            lib.oracle_apply_jones.restype = None
            lib.oracle_apply_jones.argtypes = [P, C.c_int, P, P]
            lib.oracle_dedisperse.restype = C.c_int
            lib.oracle_dedisperse.argtypes = [P, C.c_int, C.c_int, C.c_int64, P, P]
            lib.oracle_apply_gains.restype = None
            lib.oracle_apply_gains.argtypes = [P, C.c_int, P, P]
            lib.oracle_grid_v.restype = C.c_double
            lib.oracle_grid_v.argtypes = [P, C.c_int, P, C.c_int, C.c_int, C.c_int, P, P, P, C.c_int, P]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _flags(flags, n_tiles):
    if flags is None:
        return None
    f = np.ascontiguousarray(flags, dtype=np.uint8)
    assert f.shape == (n_tiles,)
    return f


def n_baselines(n_tiles: int) -> int:
    return int(_load().oracle_n_baselines(n_tiles))


def correlate(volt: np.ndarray, ns: int, c: int, flags=None) -> np.ndarray:
    """Raw integer correlation products S, int64 [T][F][B][4][2] (Eq. 2; lower triangle, XX XY YX YY).

    ``volt`` is uint8 [S][F_fine][n_tiles][2]; T = S // ns, F = F_fine // c.
    """
    volt = np.ascontiguousarray(volt, dtype=np.uint8)
    s, nf, nt, two = volt.shape
    assert two == 2
    T, F, B = s // ns, nf // c, n_baselines(nt)
    out = np.zeros((T, F, B, 4, 2), dtype=np.int64)
    fl = _flags(flags, nt)
    _load().oracle_correlate(_p(volt), nf, nt, nf, c, ns, s, _p(fl), _p(out))
    return out


def correlate_one(volt: np.ndarray, ns: int, c: int, tau: int, f: int, flags=None, fine0: int = 0,
                  n_fine: int | None = None) -> np.ndarray:
    """S for one integration and one output channel of the set starting at fine channel ``fine0``."""
    volt = np.ascontiguousarray(volt, dtype=np.uint8)
    s, nf, nt, _ = volt.shape
    B = n_baselines(nt)
    out = np.zeros((B, 4, 2), dtype=np.int64)
    fl = _flags(flags, nt)
    _load().oracle_correlate_one(volt.ctypes.data + fine0 * nt * 2, nf, nt, ns, c, tau, f, _p(fl), _p(out))
    return out


def apply_gains(S: np.ndarray, gains: np.ndarray) -> np.ndarray:
    """Calibrated sums V_ij^pq = g_i^p S_ij^pq conj(g_j^q) (Sec. 5.2.3), complex128 [B][4].

    ``S`` int64 [B][4][2] of one integration and channel; ``gains`` complex [n_tiles][2] (pol X, Y).
    """
    S = np.ascontiguousarray(S, dtype=np.int64)
    g = np.ascontiguousarray(np.stack([np.real(gains), np.imag(gains)], axis=-1), dtype=np.float64)
    nt = g.shape[0]
    assert S.shape == (n_baselines(nt), 4, 2) and g.shape == (nt, 2, 2)
    out = np.zeros((S.shape[0], 4, 2), dtype=np.float64)
    _load().oracle_apply_gains(_p(S), nt, _p(g), _p(out))
    return out[..., 0] + 1j * out[..., 1]


def apply_jones(S: np.ndarray, jones: np.ndarray) -> np.ndarray:
    """Calibrated sums V_ij = J_i S_ij J_j^H with full 2x2 Jones matrices, complex128 [B][4].

    ``jones`` complex [n_tiles][2][2] (J[p][r]).
    """
    S = np.ascontiguousarray(S, dtype=np.int64)
    J = np.ascontiguousarray(np.stack([np.real(jones), np.imag(jones)], axis=-1), dtype=np.float64)
    nt = J.shape[0]
    assert S.shape == (n_baselines(nt), 4, 2) and J.shape == (nt, 2, 2, 2)
    out = np.zeros((S.shape[0], 4, 2), dtype=np.float64)
    _load().oracle_apply_jones(_p(S), nt, _p(J), _p(out))
    return out[..., 0] + 1j * out[..., 1]


def visibilities(S: np.ndarray, K: int) -> np.ndarray:
    """V = S / K as complex64, each component one IEEE float32 division of float32(S) by float32(K)."""
    q = S.astype(np.float32) / np.float32(K)
    return q[..., 0] + 1j * q[..., 1]


def output_freqs(fine: np.ndarray, c: int) -> np.ndarray:
    fine = np.ascontiguousarray(fine, dtype=np.float64)
    out = np.zeros(len(fine) // c, dtype=np.float64)
    _load().oracle_output_freqs(_p(fine), len(fine), c, _p(out))
    return out


def uvw(enu: np.ndarray, nu: float) -> np.ndarray:
    enu = np.ascontiguousarray(enu, dtype=np.float64)
    out = np.zeros((n_baselines(enu.shape[0]), 3), dtype=np.float64)
    _load().oracle_uvw(_p(enu), enu.shape[0], float(nu), _p(out))
    return out


def default_cell(enu: np.ndarray, nu_max: float, n_pix: int, flags=None, support: int = 0,
                 phase_centre=(0.0, 0.0)) -> float:
    enu = np.ascontiguousarray(enu, dtype=np.float64)
    fl = _flags(flags, enu.shape[0])
    l0, m0 = phase_centre
    return float(_load().oracle_default_cell(_p(enu), enu.shape[0], _p(fl), float(nu_max), n_pix, support,
                                             float(l0), float(m0)))


def phase_basis(l0: float, m0: float):
    """(e_l, e_m, s0) of the pointing (l0, m0): the image plane's axes and the pointing, in (E, N, Up)."""
    el, em, s0 = np.zeros(3), np.zeros(3), np.zeros(3)
    if _load().oracle_phase_basis(float(l0), float(m0), _p(el), _p(em), _p(s0)):
        raise ValueError("pointing outside the unit disc")
    return el, em, s0


def uvw_phased(enu: np.ndarray, nu: float, l0: float, m0: float) -> np.ndarray:
    enu = np.ascontiguousarray(enu, dtype=np.float64)
    out = np.zeros((n_baselines(enu.shape[0]), 3), dtype=np.float64)
    if _load().oracle_uvw_phased(_p(enu), enu.shape[0], float(nu), float(l0), float(m0), _p(out)):
        raise ValueError("pointing outside the unit disc")
    return out


def apply_phase(V: np.ndarray, uvw_: np.ndarray) -> np.ndarray:
    """V exp(+2 pi i w) per baseline (complex [B][4] in and out)."""
    V = np.asarray(V)
    a = np.ascontiguousarray(np.stack([V.real, V.imag], axis=-1), dtype=np.float64)
    uvw_ = np.ascontiguousarray(uvw_, dtype=np.float64)
    _load().oracle_apply_phase(_p(a), _p(uvw_), a.shape[0])
    return a[..., 0] + 1j * a[..., 1]


def cells(uvw_: np.ndarray, du: float, n_pix: int):
    uvw_ = np.ascontiguousarray(uvw_, dtype=np.float64)
    B = uvw_.shape[0]
    iu = np.zeros(B, np.int32)
    iv = np.zeros(B, np.int32)
    keep = np.zeros(B, np.uint8)
    _load().oracle_cells(_p(uvw_), B, float(du), n_pix, _p(iu), _p(iv), _p(keep))
    return iu, iv, keep


def grid(S_img: np.ndarray, n_tiles: int, K: int, iu, iv, keep, n_pix: int, pol: int = POL_I,
         autos: bool = True, flags=None):
    """Full complex128 grid [N][N] (row v, column u, DC at [0][0]) and W, the sum of weights."""
    S_img = np.ascontiguousarray(S_img, dtype=np.int64)
    G = np.zeros((n_pix, n_pix, 2), dtype=np.float64)
    fl = _flags(flags, n_tiles)
    iu = np.ascontiguousarray(iu, np.int32)
    iv = np.ascontiguousarray(iv, np.int32)
    keep = np.ascontiguousarray(keep, np.uint8)
    W = _load().oracle_grid(_p(S_img), n_tiles, _p(fl), K, pol, int(bool(autos)), _p(iu), _p(iv), _p(keep),
                            n_pix, _p(G))
    return G[..., 0] + 1j * G[..., 1], float(W)


def i0(x: float) -> float:
    """Modified Bessel function I0 by the oracle's power series."""
    return float(_load().oracle_i0(float(x)))


def kb_beta(support: int) -> float:
    return float(_load().oracle_kb_beta(support))


def kb(t: float, support: int) -> float:
    """The Kaiser-Bessel gridding kernel C(t) of ``support`` cells (unit integral)."""
    return float(_load().oracle_kb(float(t), support, kb_beta(support)))


def kb_ft(nu: float, support: int) -> float:
    """Its Fourier transform c(nu), nu in cycles per cell (c(0) = 1)."""
    return float(_load().oracle_kb_ft(float(nu), support, kb_beta(support)))


def grid_kb(V: np.ndarray, n_tiles: int, K: int, uvw_: np.ndarray, du: float, support: int, n_grid: int,
            pol: int = POL_I, autos: bool = True, flags=None):
    """Convolutional gridding of raw (integer or calibrated) sums ``V`` [B][4] (complex or [B][4][2]) onto
    a grid of side ``n_grid``: full complex128 grid [n_grid][n_grid] and W."""
    V = np.asarray(V)
    if np.iscomplexobj(V):
        V = np.stack([V.real, V.imag], axis=-1)
    V = np.ascontiguousarray(V, dtype=np.float64)
    G = np.zeros((n_grid, n_grid, 2), dtype=np.float64)
    fl = _flags(flags, n_tiles)
    uvw_ = np.ascontiguousarray(uvw_, dtype=np.float64)
    W = _load().oracle_grid_kb(_p(V), n_tiles, _p(fl), K, pol, int(bool(autos)), _p(uvw_), float(du), support,
                               n_grid, _p(G))
    return G[..., 0] + 1j * G[..., 1], float(W)


def kb_crop_correct(full: np.ndarray, support: int) -> np.ndarray:
    """The central N x N of the shifted 2N x 2N image, divided by the kernel's transform along both axes
    (grid correction)."""
    full = np.ascontiguousarray(full, dtype=np.float64)
    n = full.shape[0] // 2
    out = np.zeros((n, n), dtype=np.float64)
    _load().oracle_kb_crop_correct(_p(full), n, support, _p(out))
    return out


def ifft2(G: np.ndarray) -> np.ndarray:
    """Unnormalised inverse 2D transform by the oracle's own FFT: radix 2 on power-of-two sides, the
    mixed-radix recursion on any other side."""
    n = G.shape[0]
    a = np.ascontiguousarray(np.stack([G.real, G.imag], axis=-1), dtype=np.float64)
    if _load().oracle_ifft2(_p(a), n):
        raise ValueError("side must be >= 1")
    return a[..., 0] + 1j * a[..., 1]


def idft2(G: np.ndarray) -> np.ndarray:
    """The same transform as a direct O(n^4) sum."""
    n = G.shape[0]
    g = np.ascontiguousarray(np.stack([G.real, G.imag], axis=-1), dtype=np.float64)
    a = np.zeros_like(g)
    _load().oracle_idft2(_p(g), n, _p(a))
    return a[..., 0] + 1j * a[..., 1]


def image_pixels(G: np.ndarray, W: float, yx) -> np.ndarray:
    """Pixels (y, x) of the dirty image of the full complex grid G, each summed directly over G's nonzero
    cells (for sampled checks of images too large for a whole transform)."""
    n = G.shape[0]
    g = np.ascontiguousarray(np.stack([G.real, G.imag], axis=-1), dtype=np.float64)
    p = np.ascontiguousarray(yx, dtype=np.int32).reshape(-1, 2)
    out = np.zeros(len(p), dtype=np.float64)
    _load().oracle_image_pixels(_p(g), n, float(W), _p(p), len(p), _p(out))
    return out


def image(a: np.ndarray, W: float):
    """Shifted real image / W and max |Im| / W."""
    n = a.shape[0]
    aa = np.ascontiguousarray(np.stack([a.real, a.imag], axis=-1), dtype=np.float64)
    img = np.zeros((n, n), dtype=np.float64)
    mx = _load().oracle_image(_p(aa), n, float(W), _p(img))
    return img, float(mx)


def pipeline(volt: np.ndarray, enu: np.ndarray, fine_freqs: np.ndarray, ns: int, c: int, n_pix: int,
             ids=None, flags=None, fine0: int = 0, n_fine: int | None = None, cell_lambda: float = 0.0,
             pol: int = POL_I, autos: bool = True, n_threads: int = 1, want_grids: bool = False, gains=None,
             support: int = 0, phase_centre=(0.0, 0.0)):
    """Dirty images for the listed image ids (id = tau * F + f) of one set.

    ``support`` >= 2: grid with the Kaiser-Bessel kernel of that many cells on a grid of side 2N (``grids``
    are then [n][2N][2N]) and keep the corrected central N x N of each image.  ``phase_centre`` = (l0, m0):
    phase-centre the visibilities on that pointing (direction cosines in the local E, N, Up frame).

    ``gains``: complex [F][n_tiles][2] per output channel of the set, tile and polarisation, or complex
    [F][n_tiles][2][2] full Jones matrices, or None.

    Returns dict(images [n][N][N] float64, W [n], max_im [n], grids [n][N][N] complex128 or None).
    """
    volt = np.ascontiguousarray(volt, dtype=np.uint8)
    s, nf_total, nt, _ = volt.shape
    if n_fine is None:
        n_fine = nf_total - fine0
    F = n_fine // c
    T = s // ns
    if ids is None:
        ids = np.arange(T * F, dtype=np.int64)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    n = len(ids)
    enu = np.ascontiguousarray(enu, dtype=np.float64)
    ff = np.ascontiguousarray(fine_freqs[fine0:fine0 + n_fine], dtype=np.float64)
    fl = _flags(flags, nt)
    imgs = np.zeros((n, n_pix, n_pix), dtype=np.float64)
    W = np.zeros(n, dtype=np.float64)
    mx = np.zeros(n, dtype=np.float64)
    ng = 2 * n_pix if support >= 2 else n_pix
    grids = np.zeros((n, ng, ng, 2), dtype=np.float64) if want_grids else None
    g, full = None, 0
    if gains is not None:
        gains = np.asarray(gains)
        full = int(gains.ndim == 4)
        assert gains.shape == ((F, nt, 2, 2) if full else (F, nt, 2))
        g = np.ascontiguousarray(np.stack([np.real(gains), np.imag(gains)], axis=-1), dtype=np.float64)
    rc = _load().oracle_pipeline(volt.ctypes.data + fine0 * nt * 2, nf_total, nt, n_fine, c, ns, _p(enu), _p(ff),
                                 _p(fl), n_pix, float(cell_lambda), pol, int(bool(autos)), support,
                                 float(phase_centre[0]), float(phase_centre[1]), _p(g), full, _p(ids),
                                 n, n_threads, _p(grids), _p(imgs), _p(W), _p(mx))
    if rc:
        raise ValueError("oracle_pipeline: bad arguments")
    return {"images": imgs, "W": W, "max_im": mx,
            "grids": None if grids is None else grids[..., 0] + 1j * grids[..., 1]}


def dedisperse(img: np.ndarray, delays) -> np.ndarray:
    """Incoherent dedispersion (the FRB search after imaging): ``img`` [T][F][...] images of T integrations and
    F channels, ``delays`` int [F] >= 0 in integrations; returns float64 [T - max(delays)][...] with
    out[t] = mean_f img[t + d_f][f].
    """
    img = np.ascontiguousarray(img, dtype=np.float64)
    T, F = img.shape[:2]
    P = int(np.prod(img.shape[2:])) if img.ndim > 2 else 1
    d = np.ascontiguousarray(delays, dtype=np.int32)
    assert d.shape == (F,)
    To = T - int(d.max())
    if To < 1 or d.min() < 0:
        raise ValueError("dedisperse: delays must be >= 0 and leave at least one integration")
    out = np.zeros((To,) + img.shape[2:], dtype=np.float64)
    rc = _load().oracle_dedisperse(_p(img), T, F, P, _p(d), _p(out))
    if rc != To:
        raise ValueError("oracle_dedisperse: bad arguments")
    return out

