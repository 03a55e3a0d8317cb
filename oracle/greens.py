"""Green's function, self-cell integral and voxel kernel lattice (Section 3, Eqs. 3.3 and 3.9)."""
from __future__ import annotations

import math

import numpy as np

EQUAL_VOLUME_RADIUS_FACTOR = (3.0 / (4.0 * math.pi)) ** (1.0 / 3.0)


def green(k: complex, r):
    """G_k(r) = exp(i k r) / (4 pi r) for r > 0 (Eq. 3.3)."""
    r = np.asarray(r, dtype=np.float64)
    return np.exp(1j * k * r) / (4.0 * math.pi * r)


def equal_volume_radius(h: float) -> float:
    """Radius a of the sphere whose volume equals that of a cube of side h (Section 3.1)."""
    return EQUAL_VOLUME_RADIUS_FACTOR * h


def self_cell(k: complex, h: float) -> complex:
    """Integral of G_k over the equal-volume sphere about its centre (diagonal case of Eq. 3.9).

    Closed form ((1 - i k a) exp(i k a) - 1) / k^2.  For |k a| < 0.1 the closed form
    loses about eps/|k a|^2 to cancellation, so the oracle sums the power series of
    the same integral, int_0^a r exp(i k r) dr = sum_m (i k)^m a^(m+2) / (m! (m+2)),
    whose k -> 0 limit is a^2 / 2.
    """
    a = equal_volume_radius(h)
    ka = k * a
    if abs(ka) < 0.1:
        total = 0.0 + 0.0j
        term = 1.0 + 0.0j  # (i k a)^m / m!
        for m in range(0, 24):
            total += term / (m + 2)
            term *= 1j * ka / (m + 1)
        return complex(total * a * a)
    return complex(((1.0 - 1j * ka) * np.exp(1j * ka) - 1.0) / (k * k))


def kernel_lattice(n, h: float, k: complex) -> np.ndarray:
    """Voxel-to-voxel weights of the quadrature rule Eq. 3.9 for every lattice offset.

    Returns K of shape (2nx-1, 2ny-1, 2nz-1) with K[d + n - 1] the weight that voxel
    j contributes to voxel i = j + d: h^3 G_k(|d| h) for d != 0 (midpoint rule) and
    the self-cell integral for d = 0.
    """
    nx, ny, nz = (int(v) for v in n)
    dx = np.arange(-(nx - 1), nx, dtype=np.float64)[:, None, None]
    dy = np.arange(-(ny - 1), ny, dtype=np.float64)[None, :, None]
    dz = np.arange(-(nz - 1), nz, dtype=np.float64)[None, None, :]
    r = h * np.sqrt(dx * dx + dy * dy + dz * dz)
    with np.errstate(divide="ignore", invalid="ignore"):
        K = h ** 3 * np.exp(1j * k * r) / (4.0 * math.pi * r)
    K[nx - 1, ny - 1, nz - 1] = self_cell(k, h)
    return K
