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


def nested_run(p1_on_first: np.ndarray, grids: Dict[int, object], f0: float, medium) -> Dict[int, np.ndarray]:
    """Section 6 loop for harmonics 2..max(grids).

    ``grids[n]`` is the grid of harmonic n (objects with .n, .origin, .h);
    ``p1_on_first`` is p1 evaluated on grids[2].  Every p_m with m >= 2 lives on
    grids[m]; p1 lives on grids[2].  Returns {n: p_n on grids[n]}.
    """
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
                lower.append(interp.restrict_trilinear(fields[m], src_grid, g))
        fields[n] = harmonic(n, lower, g.h, f0, medium)
        home[n] = g
    return {n: v for n, v in fields.items() if n >= 2}
