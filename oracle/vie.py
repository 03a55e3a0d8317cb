"""Volume integral equation of an inhomogeneous medium (Section 7; test infrastructure only).

p(x) - int_D G_k(x - y) (k(y)^2 - kbar^2) p(y) dy = b(x)   (Eqs. 7.1-7.5)

discretised with the quadrature of Eq. 3.9 (the same discrete operator V as
``potential``): (I - V Q) p = b with Q = diag(q), q = k(y)^2 - kbar^2.  The oracle
solves it with SciPy's GMRES (a library Krylov solver as one step) to a tight
tolerance on the FFT route, which the pins tie to the brute-force double sum.
"""
from __future__ import annotations

import inspect

import numpy as np
import scipy.sparse.linalg as sla

from . import physics, potential


def contrast(k_local: np.ndarray, k_background: complex) -> np.ndarray:
    """q = k(y)^2 - kbar^2 (zero where the medium is the background)."""
    return np.asarray(k_local, dtype=np.complex128) ** 2 - k_background ** 2


def operator(q: np.ndarray, h: float, k: complex):
    """x -> x - V_k[q x] as a function on N-voxel fields (FFT route, FP64)."""
    shape = q.shape
    khat = potential.kernel_spectrum(shape, h, k)

    def apply(x):
        x = np.asarray(x, dtype=np.complex128).reshape(shape)
        return (x - potential.apply_fft(q * x, h, k, khat=khat)).reshape(-1)

    return apply


def solve(q: np.ndarray, b: np.ndarray, h: float, k: complex, tol: float = 1e-12) -> np.ndarray:
    op = operator(q, h, k)
    n = q.size
    A = sla.LinearOperator((n, n), matvec=op, dtype=np.complex128)
    rhs = np.asarray(b, dtype=np.complex128).reshape(-1)
    # the relative-tolerance keyword is rtol in newer SciPy, tol in older releases
    kw = {"rtol": tol} if "rtol" in inspect.signature(sla.gmres).parameters else {"tol": tol}
    x, info = sla.gmres(A, rhs, atol=0.0, restart=60, maxiter=200, **kw)
    if info != 0:
        raise RuntimeError(f"GMRES did not converge (info {info})")
    return x.reshape(q.shape)


def sphere_wavenumber(grid, centre, radius: float, n: int, f0: float, background, inclusion) -> np.ndarray:
    """k_n(y) on the voxel centres: the inclusion medium inside the sphere, else background."""
    X, Y, Z = np.meshgrid(grid.axis(0), grid.axis(1), grid.axis(2), indexing="ij")
    inside = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2 <= radius ** 2
    kb = physics.wavenumber(n, f0, background)
    ki = physics.wavenumber(n, f0, inclusion)
    return np.where(inside, ki, kb)
