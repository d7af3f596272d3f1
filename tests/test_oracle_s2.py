"""Pins of the S2 autocorrelation reference (oracle/s2_ref.py): brute-force sums of the
definition on small fields, and the identities every autocorrelation obeys."""
import numpy as np

from oracle import s2_ref as S


def brute(phi, c, R):
    I = S.indicator(phi, c).astype(np.int64)
    ny, nx = I.shape
    out = np.zeros((2 * R + 1, 2 * R + 1), dtype=np.int64)
    for ry in range(-R, R + 1):
        for rx in range(-R, R + 1):
            out[ry + R, rx + R] = sum(I[y, x] * I[(y + ry) % ny, (x + rx) % nx] for y in range(ny) for x in range(nx))
    return out


def test_fft_counts_equal_the_brute_force_sum():
    g = np.random.default_rng(0)
    phi = g.standard_normal((9, 13)).astype(np.float32)
    c = g.random((9, 13)).astype(np.float32)
    np.testing.assert_array_equal(S.s2_counts(phi, c, 4), brute(phi, c, 4))


def test_autocorrelation_identities():
    g = np.random.default_rng(1)
    phi = g.standard_normal((32, 40)).astype(np.float32)
    c = g.random((32, 40)).astype(np.float32)
    R = 6
    k = S.s2_counts(phi, c, R)
    I = S.indicator(phi, c)
    assert k[R, R] == I.sum()                    # S2(0) is the volume fraction of solid A
    np.testing.assert_array_equal(k, k[::-1, ::-1])  # S2(r) = S2(-r)
    assert k.max() == k[R, R]                    # no shift correlates more than the field with itself
    # the indicator's thresholds: phi exactly 0 is vapor, c exactly 0.5 is not A-rich
    assert not S.indicator(np.float32(0.0), np.float32(0.9)) and not S.indicator(np.float32(1.0), np.float32(0.5))


def test_stripes_have_the_closed_form_correlation():
    # vertical stripes of width 4 with period 8 in a 16 x 16 solid: S2(rx, ry) = (4 - d(rx)) / 8, d the
    # distance of rx to the nearest multiple of 8
    x = np.arange(16)
    c = np.tile(((x // 4) % 2 == 0).astype(np.float32), (16, 1)) * 0.9 + 0.05
    phi = np.ones((16, 16), dtype=np.float32)
    s = S.s2(phi, c, 4)
    for rx in range(-4, 5):
        d = min(abs(rx) % 8, 8 - abs(rx) % 8)
        np.testing.assert_allclose(s[:, rx + 4], (4 - d) / 8.0)
    assert S.rel_l2(s, s) == 0.0
