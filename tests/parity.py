"""Image parity of the CUDA path against the oracle, per (frequency, source) block.

A whole-tensor norm lets a wrong quiet frequency or a wrong weak source hide under the loud
ones, so the images c (F x T x N x M) are compared block by block: for every (f, n),
  * the relative Frobenius error ||c - c_ref|| / ||c_ref|| over (t, m), and
  * the element-wise error max |c - c_ref| / max |c_ref| over (t, m),
each at most the tolerance.  Blocks whose reference is exactly zero (a source with no power
at that frequency) must be zero too.
"""
import numpy as np


def image_errors(c, c_ref):
    """(relative Frobenius error, element-wise error), each an F x N array."""
    c = np.asarray(c).astype(np.complex128)
    c_ref = np.asarray(c_ref).astype(np.complex128)
    assert c.shape == c_ref.shape and c.ndim == 4, (c.shape, c_ref.shape)
    d = np.abs(c - c_ref)
    a = np.abs(c_ref)
    num = np.sqrt((d ** 2).sum(axis=(1, 3)))
    den = np.sqrt((a ** 2).sum(axis=(1, 3)))
    dmax = d.max(axis=(1, 3))
    amax = a.max(axis=(1, 3))
    with np.errstate(divide="ignore", invalid="ignore"):
        fro = np.where(den > 0, num / den, np.where(num > 0, np.inf, 0.0))
        ele = np.where(amax > 0, dmax / amax, np.where(dmax > 0, np.inf, 0.0))
    return fro, ele


def assert_images(c, c_ref, tol, label=""):
    """Both per-block errors at most `tol`; the message names the worst block."""
    fro, ele = image_errors(c, c_ref)
    f1, n1 = np.unravel_index(int(np.argmax(fro)), fro.shape)
    f2, n2 = np.unravel_index(int(np.argmax(ele)), ele.shape)
    assert fro.max() <= tol and ele.max() <= tol, (
        f"{label} images: worst relative Frobenius error {fro.max():.3e} at (f={f1}, n={n1}), "
        f"worst element-wise error {ele.max():.3e} at (f={f2}, n={n2}), tolerance {tol:.0e}")
    return float(fro.max()), float(ele.max())
