"""Two-point autocorrelation S2 of the solid A phase (the paper's statistical error metric).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

"Autocorrelations" (Results) and "Error metrics" (Methods): S2^(A,A)(r) is the
probability that two points separated by r both lie in solid phase A, and the
hybrid solver is judged by the relative L2 error of S2 between the true and the
predicted composition fields.  READINGS: a cell is solid A when phi > 0 (solid)
and c > 0.5 (the A-rich side of the composition), decided on the FP32 fields;
shifts are periodic in both directions (the usual FFT convention), and the map
is kept for offsets |rx|, |ry| <= R.  S2(r) = counts(r) / (nx ny) with
counts(r) = sum_x I(x) I(x + r), an integer.
"""
from __future__ import annotations

import numpy as np


def indicator(phi, c) -> np.ndarray:
    return (np.asarray(phi, dtype=np.float32) > np.float32(0.0)) & (np.asarray(c, dtype=np.float32) > np.float32(0.5))


def s2_counts(phi, c, R: int) -> np.ndarray:
    """Integer counts [2R+1, 2R+1] indexed [ry + R, rx + R], through the FFT (exact after rounding)."""
    I = indicator(phi, c).astype(np.float64)
    F = np.fft.fft2(I)
    full = np.rint(np.fft.ifft2(F * np.conj(F)).real).astype(np.int64)  # full[ry, rx] = sum I(y, x) I(y+ry, x+rx)
    ny, nx = I.shape
    ry = np.arange(-R, R + 1) % ny
    rx = np.arange(-R, R + 1) % nx
    return full[np.ix_(ry, rx)]


def s2(phi, c, R: int) -> np.ndarray:
    n = np.asarray(phi).size
    return s2_counts(phi, c, R) / n


def rel_l2(s_true, s_pred) -> float:
    return float(np.linalg.norm(s_true - s_pred) / np.linalg.norm(s_true))
