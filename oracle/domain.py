"""Integration-domain selection by the localisation measure of Section 5 (test
infrastructure only).

Q(x) = log10(|f(x)| / max |f|); the integration domain D is the smallest cuboid of
voxels outside which Q < Q0.  The decision |f| >= 10^Q0 max|f| is taken, as in the
CUDA path, on squares formed in FP64 from the FP32 parts of a complex64 field:
|f|^2 >= 10^(2 Q0) max|f|^2.
"""
from __future__ import annotations

import numpy as np


def abs2_fp64(f: np.ndarray) -> np.ndarray:
    f32 = np.asarray(f, dtype=np.complex64)
    re = f32.real.astype(np.float64)
    im = f32.imag.astype(np.float64)
    return re * re + im * im


def q0_box(f: np.ndarray, q0: float):
    """(lo, hi): inclusive index bounds per axis of the voxels with Q >= q0."""
    a2 = abs2_fp64(f)
    thr = a2.max() * np.power(10.0, 2.0 * q0)
    keep = a2 >= thr
    lo, hi = [], []
    for ax in range(3):
        other = tuple(b for b in range(3) if b != ax)
        idx = np.nonzero(keep.any(axis=other))[0]
        lo.append(int(idx[0]))
        hi.append(int(idx[-1]))
    return tuple(lo), tuple(hi)


def q_field(f: np.ndarray) -> np.ndarray:
    """Q(x) in FP64 (log10 of |f| over its maximum); -inf where f = 0."""
    a = np.abs(np.asarray(f, dtype=np.complex128))
    with np.errstate(divide="ignore"):
        return np.log10(a / a.max())
