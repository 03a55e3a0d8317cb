"""Pins of the domain-selection oracle: a brute-force scan written as plain loops, the
analytic support of a Gaussian, and the limits Q0 = 0 (the maximum) and Q0 -> -inf
(the whole grid)."""
import math

import numpy as np

from oracle import domain


def _brute(f, q0):
    a = np.abs(np.asarray(f, dtype=np.complex128))
    m = a.max()
    lo, hi = [10 ** 9] * 3, [-1] * 3
    for i in range(f.shape[0]):
        for j in range(f.shape[1]):
            for k in range(f.shape[2]):
                if a[i, j, k] > 0 and math.log10(a[i, j, k] / m) >= q0 - 1e-12:
                    for ax, v in enumerate((i, j, k)):
                        lo[ax] = min(lo[ax], v)
                        hi[ax] = max(hi[ax], v)
    return tuple(lo), tuple(hi)


def test_box_matches_brute_force_scan():
    rng = np.random.default_rng(0)
    f = (rng.standard_normal((7, 9, 6)) + 1j * rng.standard_normal((7, 9, 6))).astype(np.complex64)
    f *= np.exp(-((np.arange(7)[:, None, None] - 3) ** 2 + (np.arange(9)[None, :, None] - 5) ** 2) / 4.0)
    for q0 in (-0.3, -1.0, -2.0, -4.0):
        assert domain.q0_box(f, q0) == _brute(f, q0), q0


def test_gaussian_support_is_the_analytic_box():
    n = 41
    x = np.arange(n) - 20.0
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    sig = (6.0, 3.0, 4.5)
    f = np.exp(-(X ** 2 / (2 * sig[0] ** 2) + Y ** 2 / (2 * sig[1] ** 2) + Z ** 2 / (2 * sig[2] ** 2)))
    for q0 in (-0.5, -1.5, -3.0):
        lo, hi = domain.q0_box(f.astype(np.complex64), q0)
        for ax in range(3):
            # |f| >= 10^q0 on the axis: |x| <= sig sqrt(2 ln(10) |q0|)
            r = int(math.floor(sig[ax] * math.sqrt(2 * math.log(10) * -q0)))
            assert lo[ax] == max(0, 20 - r) and hi[ax] == min(n - 1, 20 + r)


def test_limits():
    rng = np.random.default_rng(1)
    f = (rng.standard_normal((5, 6, 7)) + 1j * rng.standard_normal((5, 6, 7))).astype(np.complex64)
    i = np.unravel_index(np.argmax(np.abs(f)), f.shape)
    assert domain.q0_box(f, 0.0) == (tuple(int(v) for v in i), tuple(int(v) for v in i))
    assert domain.q0_box(f, -40.0) == ((0, 0, 0), (4, 5, 6))
    assert domain.q0_box(np.zeros((3, 4, 5), np.complex64), -1.0) == ((0, 0, 0), (2, 3, 4))
