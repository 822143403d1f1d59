"""Image parity gates shared by the GPU tests and bench.py (not a test module).

An image computed in FP32 is compared with the FP64 oracle's image of the same inputs by two norms:

* relative RMS, ||got - ref||_2 / ||ref||_2 <= 1e-4: the method's precision gate for the mixed-precision
  form (correlation exact, gridding and transform in FP32);
* max |got - ref| / max |ref| <= 1e-5: a pointwise bound, because a norm over N^2 pixels dilutes a
  localised error (at 512^2 a single pixel could be off by 1e-4 * 512 times the image RMS and still pass
  the first gate).  FP32 transform errors are spread evenly over the pixels, a few times their RMS at
  most, and the measured relative RMS is ~1e-7, so the FP32 forms sit two orders of magnitude inside it;
  a wrong edge column, Nyquist row or single cell of the output fails it.
"""
import numpy as np

IMG_RTOL = 1e-4       # relative RMS
IMG_MAXTOL = 1e-5     # max |diff| / max |ref|


def image_errors(got, ref):
    """(relative RMS, max |diff| / max |ref|) of one image or a stack of images taken as a whole."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = got - ref
    rms = float(np.linalg.norm(d) / np.linalg.norm(ref))
    mx = float(np.abs(d).max() / np.abs(ref).max())
    return rms, mx


def image_ok(got, ref, rms_tol=IMG_RTOL, max_tol=IMG_MAXTOL):
    rms, mx = image_errors(got, ref)
    return rms <= rms_tol and mx <= max_tol


def assert_image_close(got, ref, what=None, rms_tol=IMG_RTOL, max_tol=IMG_MAXTOL):
    rms, mx = image_errors(got, ref)
    assert rms <= rms_tol and mx <= max_tol, (what, "rel RMS", rms, "max |diff| / max |ref|", mx)
