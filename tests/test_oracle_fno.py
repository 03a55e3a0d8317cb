"""Pins of the FP64 FNO reference: its spectral convolution against the truncated
DFT written out as sums (no FFT library), GELU against its definition, and the
degree-n homogeneity that lets the surrogate work on normalised fields."""
import math

import numpy as np
import scipy.integrate

from oracle import fno


def _brute_spectral_conv(h, R, modes):
    N = h.shape[0]
    mx, my, mz = modes
    kx, ky = fno.kept(N, mx), fno.kept(N, my)
    n = np.arange(N)
    out = np.zeros(h.shape[:3] + (R.shape[-1],))
    for ix, a in enumerate(kx):
        for iy, b in enumerate(ky):
            for c in range(mz):
                ph = np.exp(-2j * np.pi * (a * n[:, None, None] + b * n[None, :, None] + c * n[None, None, :]) / N)
                Hk = np.einsum("xyz,xyzc->c", ph, h)
                O = Hk @ R[ix, iy, c]
                w = 1.0 if c == 0 else 2.0  # Hermitian partner of kz > 0
                # real inverse transform contribution of this mode (kz = 0: real part only)
                out += w * np.real(np.conj(ph)[..., None] * O) / N ** 3
    return out


def test_spectral_conv_matches_written_out_dft():
    rng = np.random.default_rng(0)
    N, C, O = 6, 3, 2
    modes = (4, 2, 3)
    h = rng.standard_normal((N, N, N, C))
    R = rng.standard_normal((4, 2, 3, C, O)) + 1j * rng.standard_normal((4, 2, 3, C, O))
    got = fno.spectral_conv(h, R, modes)
    ref = _brute_spectral_conv(h, R, modes)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_gelu_is_x_times_the_normal_cdf():
    for x in (-3.0, -0.7, 0.0, 0.4, 2.5):
        cdf = scipy.integrate.quad(lambda t: math.exp(-t * t / 2) / math.sqrt(2 * math.pi), -40, x)[0]
        assert abs(fno.gelu(np.array(x)) - x * cdf) < 1e-12


def test_forward_shapes_and_loss_zero_at_its_own_output():
    p = fno.init_params(8, 4, 8, 2, (4, 4, 3), seed=1)
    x = np.random.default_rng(2).standard_normal((8, 8, 8, 2))
    y = fno.forward(p, x, (4, 4, 3))
    assert y.shape == (8, 8, 8, 8)
    assert fno.loss(p, x, y, (4, 4, 3)) == 0.0


def test_features_follow_de_moivre():
    # q = r e^{i theta}: q^k = r^k (cos k theta + i sin k theta)
    r, th = 0.8, 0.37
    x = np.array([r * math.cos(th), r * math.sin(th)])
    f = fno.features(x)
    for k in range(1, 6):
        assert abs(f[2 * k - 2] - r ** k * math.cos(k * th)) < 1e-15
        assert abs(f[2 * k - 1] - r ** k * math.sin(k * th)) < 1e-15
