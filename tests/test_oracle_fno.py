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


def _hand_network(p, x):
    """The surrogate written out voxel by voxel with scalar arithmetic for N = 2 and
    modes (2, 2, 1): every kept mode has kz = 0, and on a 2-point axis the DFT phases
    are +-1, so the spectral convolution is
      out[v, o] = (1/8) Re sum_{kx, ky} (-1)^(kx x + ky y) sum_c R[kx, ky, 0, c, o] H[kx, ky, c],
      H[kx, ky, c] = sum_v (-1)^(kx x + ky y) h[v, c]."""
    vox = [(a, b, c) for a in range(2) for b in range(2) for c in range(2)]
    W = len(p["bP"])

    def gelu(t):
        return 0.5 * t * (1.0 + math.erf(t / math.sqrt(2.0)))

    h = {}
    for v in vox:
        q = complex(x[v][0], x[v][1])
        phi = []
        for k in range(1, 6):
            phi += [(q ** k).real, (q ** k).imag]
        h[v] = [sum(phi[f] * p["P"][f][c] for f in range(10)) + p["bP"][c] for c in range(W)]
    L = len(p["R"])
    for l in range(L):
        R = p["R"][l]
        H = {(kx, ky): [sum((-1) ** (kx * v[0] + ky * v[1]) * h[v][c] for v in vox) for c in range(W)]
             for kx in range(2) for ky in range(2)}
        new = {}
        for v in vox:
            row = []
            for o in range(W):
                spec = sum((-1) ** (kx * v[0] + ky * v[1]) * sum(R[kx][ky][0][c][o] * H[(kx, ky)][c] for c in range(W))
                           for kx in range(2) for ky in range(2))
                t = spec.real / 8.0 + sum(h[v][c] * p["W"][l][c][o] for c in range(W)) + p["b"][l][o]
                row.append(gelu(t) if l < L - 1 else t)
            new[v] = row
        h = new
    y = np.zeros((2, 2, 2, 8))
    Hd = len(p["bQ1"])
    for v in vox:
        g = [gelu(sum(h[v][c] * p["Q1"][c][j] for c in range(W)) + p["bQ1"][j]) for j in range(Hd)]
        for o in range(8):
            y[v][o] = sum(g[j] * p["Q2"][j][o] for j in range(Hd)) + p["bQ2"][o]
    return y


def _tiny_params(seed):
    """Two layers, width 2, hidden 3, with non-zero biases everywhere."""
    p = fno.init_params(2, 2, 3, 2, (2, 2, 1), seed=seed)
    rng = np.random.default_rng(seed + 100)
    p["bP"] = rng.standard_normal(2)
    p["b"] = [rng.standard_normal(2) for _ in range(2)]
    p["bQ1"] = rng.standard_normal(3)
    p["bQ2"] = rng.standard_normal(8)
    return p


def test_forward_matches_the_network_written_out():
    """Pins the composition: the lift with its bias, each layer's spectral and pointwise
    branches with their bias, GELU after every layer but the last, and the two-stage
    projection with GELU between."""
    p = _tiny_params(3)
    x = 0.6 * np.random.default_rng(4).standard_normal((2, 2, 2, 2))
    got = fno.forward(p, x, (2, 2, 1))
    want = _hand_network(p, x)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    # the check is sensitive to the last layer's (absent) activation
    q = dict(p)
    q["R"] = [p["R"][0]]
    q["W"] = [p["W"][0]]
    q["b"] = [p["b"][0]]
    one = fno.forward(q, x, (2, 2, 1))
    assert np.max(np.abs(one - _hand_network(q, x))) <= 1e-12 * np.max(np.abs(one))


def test_loss_is_the_mean_relative_squared_error_per_harmonic():
    """loss = (1/4) sum_n sum |y_n - t_n|^2 / sum |t_n|^2 over the 4 harmonics' (Re, Im)
    channel pairs, the target in the denominator, written out with scalar sums."""
    p = _tiny_params(5)
    rng = np.random.default_rng(6)
    x = 0.6 * rng.standard_normal((2, 2, 2, 2))
    t = rng.standard_normal((2, 2, 2, 8)) * np.array([1.0, 1.0, 3.0, 3.0, 0.2, 0.2, 7.0, 7.0])
    y = _hand_network(p, x)
    total = 0.0
    for n in range(4):
        num = den = 0.0
        for v in np.ndindex(2, 2, 2):
            for ch in (2 * n, 2 * n + 1):
                num += (y[v][ch] - t[v][ch]) ** 2
                den += t[v][ch] ** 2
        total += num / den
    assert abs(fno.loss(p, x, t, (2, 2, 1)) - total / 4.0) <= 1e-12 * total
