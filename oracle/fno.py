"""FP64 reference of the Fourier-neural-operator surrogate (test infrastructure only).

The surrogate maps the normalised fundamental q1 = p1 / s on an N^3 focal box (two
real channels: Re, Im) to the normalised harmonics q_n = p_n / s^n, n = 2..5 (eight
channels).  The cascade makes p_n homogeneous of degree n in p1 (Eq. 2.6), so the
scale s = max |p1| factors out exactly and the network only learns the shape.

Architecture (a Fourier neural operator with power features at the input):
  phi(x) = (Re q, Im q, Re q^2, Im q^2, ..., Re q^5, Im q^5),  q = x0 + i x1
  h0 = phi(x) P + bP                                       lift 10 -> W
  t_l = SpecConv_l(h_l) + h_l W_l + b_l,  h_{l+1} = GELU(t_l) for l < L-1, else t_l
  y = GELU(h_L Q1 + bQ1) Q2 + bQ2                          project W -> H -> 8
SpecConv: real 3-D FFT (rfftn over x, y, z), keep kx, ky in the lowest mx, my (half
non-negative, half negative) and kz in [0, mz), multiply each kept mode by a complex
W x W matrix, zero the rest, inverse real FFT (irfftn).
Loss: mean over n of ||y_n - q_n||^2 / ||q_n||^2 (relative squared L2 per harmonic).
GELU is the exact form x Phi(x) = x (1 + erf(x / sqrt 2)) / 2.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special


def kept(N: int, m: int) -> np.ndarray:
    """Kept frequency indices of a full axis: 0 .. m/2 - 1 and N - m/2 .. N - 1."""
    h = m // 2
    return np.concatenate([np.arange(h), np.arange(N - h, N)])


def gelu(x):
    return 0.5 * x * (1.0 + scipy.special.erf(x / math.sqrt(2.0)))


def spectral_conv(h: np.ndarray, R: np.ndarray, modes) -> np.ndarray:
    """h: (N, N, N, C) real; R: (mx, my, mz, C, O) complex; returns (N, N, N, O) real."""
    N = h.shape[0]
    mx, my, mz = modes
    H = np.fft.rfftn(h, axes=(0, 1, 2))
    kx, ky, kz = kept(N, mx), kept(N, my), np.arange(mz)
    Hk = H[np.ix_(kx, ky, kz)]
    O = np.einsum("xyzc,xyzco->xyzo", Hk, R)
    full = np.zeros((N, N, N // 2 + 1, R.shape[-1]), dtype=np.complex128)
    full[np.ix_(kx, ky, kz)] = O
    return np.fft.irfftn(full, s=(N, N, N), axes=(0, 1, 2))


POWERS = 5


def features(x: np.ndarray) -> np.ndarray:
    """(..., 2) real pairs -> (..., 10): Re and Im of q^k, k = 1..5, q = x0 + i x1."""
    q = x[..., 0] + 1j * x[..., 1]
    out = []
    for k in range(1, POWERS + 1):
        qk = q ** k
        out += [qk.real, qk.imag]
    return np.stack(out, axis=-1)


def forward(params: dict, x: np.ndarray, modes) -> np.ndarray:
    """x: (N, N, N, 2) -> (N, N, N, 8)."""
    h = features(x) @ params["P"] + params["bP"]
    L = len(params["R"])
    for l in range(L):
        t = spectral_conv(h, params["R"][l], modes) + h @ params["W"][l] + params["b"][l]
        h = gelu(t) if l < L - 1 else t
    g = gelu(h @ params["Q1"] + params["bQ1"])
    return g @ params["Q2"] + params["bQ2"]


def loss(params: dict, x: np.ndarray, target: np.ndarray, modes) -> float:
    y = forward(params, x, modes)
    total = 0.0
    for n in range(4):
        d = y[..., 2 * n:2 * n + 2] - target[..., 2 * n:2 * n + 2]
        t = target[..., 2 * n:2 * n + 2]
        total += float(np.sum(d * d) / np.sum(t * t))
    return total / 4.0


def init_params(N: int, width: int, hidden: int, layers: int, modes, seed: int) -> dict:
    """Seeded initial parameters (scaled normal), FP64."""
    rng = np.random.default_rng(seed)
    mx, my, mz = modes
    W = width

    def nrm(*shape, scale):
        return rng.standard_normal(shape) * scale

    return {
        "P": nrm(2 * POWERS, W, scale=1.0 / math.sqrt(2 * POWERS)), "bP": np.zeros(W),
        "R": [(nrm(mx, my, mz, W, W, scale=1.0 / W) + 1j * nrm(mx, my, mz, W, W, scale=1.0 / W))
              for _ in range(layers)],
        "W": [nrm(W, W, scale=1.0 / math.sqrt(W)) for _ in range(layers)],
        "b": [np.zeros(W) for _ in range(layers)],
        "Q1": nrm(W, hidden, scale=1.0 / math.sqrt(W)), "bQ1": np.zeros(hidden),
        "Q2": nrm(hidden, 8, scale=1.0 / math.sqrt(hidden)), "bQ2": np.zeros(8),
    }
