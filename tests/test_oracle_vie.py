"""Pins of the volume-integral-equation oracle (Section 7): a manufactured solution built
with the brute-force double sum, the zero-contrast limit, and the Born series (the
correction beyond first order shrinks with the square of the contrast)."""
import numpy as np

from oracle import physics, potential, vie
from paper_2011_03009_gb300 import synth


def _setup(n=(6, 5, 4), h=2.0e-4, seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    k = physics.wavenumber(1, 1.0e6, synth.WATER)
    q = scale * 0.3 * k * k * (rng.uniform(0.5, 1.0, n) + 0.2j * rng.uniform(0.0, 1.0, n))
    return q, h, k


def test_manufactured_solution_with_bruteforce_operator():
    q, h, k = _setup()
    x_true = synth.random_field(q.shape, 1)
    b = x_true - potential.apply_bruteforce(q * x_true, h, k)
    x = vie.solve(q, b, h, k)
    assert np.linalg.norm(x - x_true) <= 1e-9 * np.linalg.norm(x_true)


def test_zero_contrast_returns_the_right_hand_side():
    q, h, k = _setup()
    b = synth.random_field(q.shape, 2)
    assert np.allclose(vie.solve(np.zeros_like(q), b, h, k), b, rtol=0, atol=1e-14)


def test_born_series_second_order():
    errs = []
    for scale in (0.2, 0.1, 0.05):
        q, h, k = _setup(n=(8, 8, 8), scale=scale)
        b = synth.random_field(q.shape, 3)
        x = vie.solve(q, b, h, k)
        born = b + potential.apply_fft(q * b, h, k)
        errs.append(np.linalg.norm(x - born) / np.linalg.norm(born - b))
    # relative size of the terms beyond first order is proportional to the contrast
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2, errs


def test_sphere_wavenumber():
    g = synth.Grid((5, 5, 5), (-2e-3, -2e-3, -2e-3), 1e-3)
    tissue = synth.Medium(c0=1540.0, rho0=1000.0, beta=3.5, alpha0=5.0, eta=1.1)
    kk = vie.sphere_wavenumber(g, (0.0, 0.0, 0.0), 1.05e-3, 2, 1.0e6, synth.WATER, tissue)
    q = vie.contrast(kk, physics.wavenumber(2, 1.0e6, synth.WATER))
    assert np.count_nonzero(q) == 7  # centre and its 6 face neighbours
    assert abs(kk[2, 2, 2] - physics.wavenumber(2, 1.0e6, tissue)) == 0.0
