"""The discrete volume potential u = V_k[f] on a uniform voxel grid (Section 3.1, Eq. 3.9).

u(x_i) = sum_{j != i} h^3 G_k(x_i - x_j) f(x_j) + S(k, h) f(x_i), where S is the
self-cell integral.  Two evaluations:

- ``apply_bruteforce``: the double sum written out, distances taken from the voxel
  centres, O(N^2).  It does not use ``greens.kernel_lattice``.
- ``apply_sparse``: the same sum at chosen target voxels for a source that is zero
  outside a list of voxels, O(targets x sources); it serves grids too large for the
  other two.
- ``apply_fft``: the same sum as a 3-level Toeplitz matrix-vector product, embedded in
  a circulant of size M >= 2N - 1 per axis and evaluated with FFTs (Section 3.1;
  Section 6 uses M = 2N).  Offsets d in (-N, N) sit at index d mod M; any
  remaining index is never read and is set to zero.
"""
from __future__ import annotations

import math
import os

import numpy as np
import scipy.fft

from . import greens

WORKERS = os.cpu_count() or 1


def apply_bruteforce(f: np.ndarray, h: float, k: complex, targets=None) -> np.ndarray:
    """Direct O(N^2) evaluation of Eq. 3.9.  ``targets``: optional (T, 3) int voxel indices.

    Returns the full field (shape of f) or, with targets, a length-T vector.
    """
    f = np.asarray(f, dtype=np.complex128)
    n = f.shape
    idx = np.indices(n).reshape(3, -1).T.astype(np.float64)  # (N, 3) voxel indices
    fv = f.reshape(-1)
    self_w = greens.self_cell(k, h)
    if targets is None:
        tgt = idx
    else:
        tgt = np.asarray(targets, dtype=np.float64).reshape(-1, 3)
    out = np.empty(len(tgt), dtype=np.complex128)
    chunk = max(1, 4_000_000 // max(1, len(idx)))
    for s in range(0, len(tgt), chunk):
        t = tgt[s:s + chunk]
        d = t[:, None, :] - idx[None, :, :]
        r = h * np.sqrt(np.sum(d * d, axis=2))
        same = r == 0.0
        r_safe = np.where(same, 1.0, r)
        w = h ** 3 * np.exp(1j * k * r_safe) / (4.0 * math.pi * r_safe)
        w = np.where(same, self_w, w)
        out[s:s + chunk] = w @ fv
    if targets is None:
        return out.reshape(n)
    return out


def apply_sparse(src_idx, src_val, h: float, k: complex, targets) -> np.ndarray:
    """Eq. 3.9 at the target voxels ``targets`` ((T, 3) ints) for the source that equals
    ``src_val[j]`` at voxel ``src_idx[j]`` ((S, 3) ints) and zero elsewhere:
    u(t) = sum_j w(t - s_j) f_j with w = h^3 G_k(h |t - s_j|) off the diagonal and the
    self-cell integral on it.  The grid's extent does not enter."""
    s = np.asarray(src_idx, dtype=np.float64).reshape(-1, 3)
    f = np.asarray(src_val, dtype=np.complex128).reshape(-1)
    t = np.asarray(targets, dtype=np.float64).reshape(-1, 3)
    self_w = greens.self_cell(k, h)
    out = np.empty(len(t), dtype=np.complex128)
    chunk = max(1, 4_000_000 // max(1, len(s)))
    for a in range(0, len(t), chunk):
        d = t[a:a + chunk, None, :] - s[None, :, :]
        r = h * np.sqrt(np.sum(d * d, axis=2))
        same = r == 0.0
        r_safe = np.where(same, 1.0, r)
        w = np.where(same, self_w, h ** 3 * np.exp(1j * k * r_safe) / (4.0 * math.pi * r_safe))
        out[a:a + chunk] = w @ f
    return out


def embedding_sizes(n, m=None):
    """Circulant size per axis: M = 2N (Section 6) unless given; must satisfy M >= 2N - 1."""
    if m is None:
        m = tuple(2 * int(v) for v in n)
    m = tuple(int(v) for v in m)
    for a in range(3):
        if m[a] < 2 * n[a] - 1:
            raise ValueError("embedding size M must be >= 2N - 1 on every axis")
    return m


def circulant_kernel(n, h: float, k: complex, m=None, unused_value: complex = 0.0) -> np.ndarray:
    """First column of the 3-level circulant embedding of the Toeplitz operator.

    Entry at index (m_x, m_y, m_z) holds the lattice weight of offset d with d = m for
    m < N and d = m - M for m > M - N, per axis; indices between are never used
    by the product and receive ``unused_value``.
    """
    n = tuple(int(v) for v in n)
    m = embedding_sizes(n, m)
    K = greens.kernel_lattice(n, h, k)
    C = np.full(m, unused_value, dtype=np.complex128)

    def axis_map(N, M):
        src = np.full(M, -1, dtype=np.int64)
        for i in range(M):
            if i < N:
                src[i] = i + N - 1          # d = i
            elif i > M - N:
                src[i] = (i - M) + N - 1    # d = i - M
        return src

    sx, sy, sz = (axis_map(n[a], m[a]) for a in range(3))
    vx, vy, vz = sx >= 0, sy >= 0, sz >= 0
    C[np.ix_(vx, vy, vz)] = K[np.ix_(sx[vx], sy[vy], sz[vz])]
    return C


def kernel_spectrum(n, h: float, k: complex, m=None) -> np.ndarray:
    """FFT of the circulant kernel (the Green's function spectrum on the embedding)."""
    return scipy.fft.fftn(circulant_kernel(n, h, k, m), workers=WORKERS)


def apply_fft(f: np.ndarray, h: float, k: complex, m=None, khat=None) -> np.ndarray:
    """Eq. 3.9 evaluated by zero padding to M, FFT, multiplication by the kernel spectrum,
    inverse FFT and cropping back to N."""
    f = np.asarray(f, dtype=np.complex128)
    n = f.shape
    m = embedding_sizes(n, m)
    if khat is None:
        khat = kernel_spectrum(n, h, k, m)
    F = scipy.fft.fftn(f, s=m, workers=WORKERS)
    F *= khat
    u = scipy.fft.ifftn(F, workers=WORKERS)
    return np.ascontiguousarray(u[: n[0], : n[1], : n[2]])
