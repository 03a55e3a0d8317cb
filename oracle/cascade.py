"""Harmonic source terms and the nested-mesh cascade (Sections 2, 3 and 6).

Source of harmonic n (Eq. 2.6, neglecting every product p_i p_j with i + j > n):
f_n = C_n * sum_{m=1}^{n-1} p_m p_{n-m}, with C_n from ``physics.source_coefficient``.
Written out for n = 2..5 this is Eqs. 3.5-3.8; the pairs (m, n-m) and (n-m, m)
are both counted, which is where the factors 2 in Eqs. 3.6-3.8 come from.

The nested-mesh algorithm (Section 6): for each harmonic n >= 2, build its own
voxel grid, bring every lower harmonic onto it (p1 evaluated directly on the grid
of harmonic 2 by the Rayleigh sum, later ones by linear interpolation from the
grid each was computed on), assemble f_n and evaluate the volume potential.
"""
from __future__ import annotations

from typing import Dict, Sequence

import numpy as np

from . import interp, physics, potential


def source_term(n: int, lower: Sequence[np.ndarray], f0: float, medium) -> np.ndarray:
    """f_n = C_n sum_{m=1}^{n-1} p_m p_{n-m}; ``lower[m-1]`` is p_m on the grid of harmonic n."""
    if n < 2 or len(lower) != n - 1:
        raise ValueError("harmonic n needs exactly n-1 lower harmonics")
    acc = np.zeros_like(np.asarray(lower[0], dtype=np.complex128))
    for m in range(1, n):
        acc = acc + np.asarray(lower[m - 1]) * np.asarray(lower[n - m - 1])
    return physics.source_coefficient(n, f0, medium) * acc


def harmonic(n: int, lower: Sequence[np.ndarray], h: float, f0: float, medium,
             m=None) -> np.ndarray:
    """p_n = V_{k_n}[f_n] on the grid of spacing h (Eqs. 3.5-3.9)."""
    f = source_term(n, lower, f0, medium)
    return potential.apply_fft(f, h, physics.wavenumber(n, f0, medium), m)


def nested_run(p1_on_first: np.ndarray, grids: Dict[int, object], f0: float, medium,
               restrict=None) -> Dict[int, np.ndarray]:
    """Section 6 loop for harmonics 2..max(grids).

    ``grids[n]`` is the grid of harmonic n (objects with .n, .origin, .h);
    ``p1_on_first`` is p1 evaluated on grids[2].  Every p_m with m >= 2 lives on
    grids[m]; p1 lives on grids[2].  ``restrict`` is the inter-mesh interpolation
    (default: trilinear, as Section 6 uses; interp.restrict_quadratic is the higher-order
    option it recommends).  Returns {n: p_n on grids[n]}.
    """
    if restrict is None:
        restrict = interp.restrict_trilinear
    fields = {1: p1_on_first}
    home = {1: grids[2]}
    for n in sorted(grids):
        if n < 2:
            continue
        g = grids[n]
        lower = []
        for m in range(1, n):
            src_grid = home[m]
            if src_grid is g:
                lower.append(fields[m])
            else:
                lower.append(restrict(fields[m], src_grid, g))
        fields[n] = harmonic(n, lower, g.h, f0, medium)
        home[n] = g
    return {n: v for n, v in fields.items() if n >= 2}


# ---- the full cascade with conjugate terms (Eq. 2.5) ---------------------------------
# Matching the e^{-i n omega t} coefficients of the Westervelt equation with the field
# written as (1/2) sum_n (p_n e^{-i n omega t} + conj(p_n) e^{i n omega t}) gives, for
# every n >= 1, a source that also draws on the harmonics above n:
#   f_n = C_n sum_{m >= 1} p_m (p_{n-m} + 2 conj(p_{m-n})),  p_j = 0 for j <= 0,
# truncated at the highest harmonic kept, N_h.  The weakly nonlinear cascade (Eq. 2.6)
# is the same sum without the conjugate products.

def source_term_full(n: int, fields: Sequence[np.ndarray], f0: float, medium) -> np.ndarray:
    """Eq. 2.5 source of harmonic n from ``fields[m-1]`` = p_m, m = 1..N_h (same grid)."""
    nh = len(fields)
    if not 1 <= n <= nh:
        raise ValueError("harmonic outside 1..N_h")
    p = [None] + [np.asarray(v, dtype=np.complex128) for v in fields]
    acc = np.zeros_like(p[1])
    for m in range(1, nh + 1):
        if 1 <= n - m:
            acc = acc + p[m] * p[n - m]
        if 1 <= m - n:
            acc = acc + 2.0 * p[m] * np.conj(p[m - n])
    return physics.source_coefficient(n, f0, medium) * acc


def full_cascade(p_inc: np.ndarray, nh: int, h: float, f0: float, medium, iters: int,
                 start=None):
    """Jacobi fixed-point iteration of Eq. 2.5 on one grid:
    p_1 <- p_inc + V_{k_1}[f_1(p)],  p_n <- V_{k_n}[f_n(p)] for n = 2..N_h,
    starting from ``start`` (default: the weakly nonlinear cascade of Eq. 2.6).
    Returns the list of iterates' fields after ``iters`` sweeps."""
    if start is None:
        p = [np.asarray(p_inc, dtype=np.complex128)]
        for n in range(2, nh + 1):
            p.append(harmonic(n, p[:n - 1], h, f0, medium))
    else:
        p = [np.asarray(v, dtype=np.complex128) for v in start]
    for _ in range(iters):
        new = []
        for n in range(1, nh + 1):
            u = potential.apply_fft(source_term_full(n, p, f0, medium), h, physics.wavenumber(n, f0, medium))
            new.append(p_inc + u if n == 1 else u)
        p = new
    return p
