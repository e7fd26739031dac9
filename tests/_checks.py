"""Parity checks shared by the GPU tests: every comparison of a CUDA result
with the FP64 oracle asserts a norm bound (relative L2 for single operator
outputs, the range-normalised NRMSE of Sec. 3.4 for images) AND an
element-wise bound, max |a - ref| / max |ref|, so that an error confined to a
few elements (one wrong patch-edge column, a conjugation slip in a ragged
tail) cannot hide inside a norm taken over ~10^6 outputs.

Element-wise bounds: for rounding errors the largest element error is a few
times the RMS error.  Single operator outputs carry errors of about the same
relative size everywhere, so max|d| / max|ref| stays below 4x the relative
L2 bound.  For images the NRMSE is normalised by the image range (about
max|ref|), and the largest error of a reconstruction sits a few RMS errors
above the mean, so the element bound is 10x the NRMSE bound.
"""
import numpy as np

import oracle as O

ELEM_FACTOR_OP = 4.0
ELEM_FACTOR_IMG = 10.0


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def maxrel(a, b):
    """max |a - b| / max |b| over all elements."""
    return float(np.abs(a - b).max() / np.abs(b).max())


def check_close(a, ref, tol, what=""):
    """Relative L2 error < tol and max |a - ref| / max |ref| < 4 tol."""
    a = np.asarray(a)
    ref = np.asarray(ref)
    assert a.shape == ref.shape, (what, a.shape, ref.shape)
    r, m = rel(a, ref), maxrel(a, ref)
    assert r < tol, f"{what}: relative L2 error {r:.3e} >= {tol:.1e}"
    assert m < ELEM_FACTOR_OP * tol, f"{what}: max element error {m:.3e} >= {ELEM_FACTOR_OP * tol:.1e}"
    return r, m


def check_image(x, ref, tol, what=""):
    """NRMSE (Sec. 3.4) < tol and max |x - ref| / max |ref| < 10 tol."""
    x = np.asarray(x)
    ref = np.asarray(ref)
    assert x.shape == ref.shape, (what, x.shape, ref.shape)
    e, m = O.nrmse(x, ref), maxrel(x, ref)
    assert e < tol, f"{what}: NRMSE {e:.3e} >= {tol:.1e}"
    assert m < ELEM_FACTOR_IMG * tol, f"{what}: max element error {m:.3e} >= {ELEM_FACTOR_IMG * tol:.1e}"
    return e, m
