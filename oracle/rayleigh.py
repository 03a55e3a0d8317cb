"""Incident field p1 of a bowl transducer as a monopole sum (Section 3.2, Eq. 3.10).

Eq. 3.10 gives the unnormalised field (A / n_p) sum_i G_k(x, r_i) with A the bowl
area.  The paper normalises to a radiated power; the workloads prescribe a surface
pressure p0 instead.  Reading: uniform normal surface velocity v0 = p0 / (rho0 c0)
in the Rayleigh integral p(x) = -i omega rho0 v0 / (2 pi) int exp(i k R)/R dS, i.e.
p(x) = -2 i k p0 int G_k(x, y) dS(y), discretised by Eq. 3.10's equal-weight sum:
p1(x) = -2 i k1 p0 (A / n_p) sum_i G_k1(x - r_i).

The bowl is the spherical cap of radius l about the focus with aperture radius R;
its area is A = 2 pi l (l - sqrt(l^2 - R^2)).
"""
from __future__ import annotations

import math

import numpy as np

from . import physics


def cap_area(l: float, R: float) -> float:
    return 2.0 * math.pi * l * (l - math.sqrt(l * l - R * R))


def incident_field_at(points_xyz: np.ndarray, bowl_points: np.ndarray, bowl, medium) -> np.ndarray:
    """p1 at arbitrary (T, 3) coordinates from the (n_p, 3) bowl points (Eq. 3.10)."""
    k = physics.wavenumber(1, bowl.f0, medium)
    A = cap_area(bowl.l, bowl.R)
    scale = -2j * k * bowl.p0 * A / len(bowl_points)
    x = np.asarray(points_xyz, dtype=np.float64).reshape(-1, 3)
    out = np.empty(len(x), dtype=np.complex128)
    chunk = max(1, 2_000_000 // max(1, len(bowl_points)))
    for s in range(0, len(x), chunk):
        d = x[s:s + chunk, None, :] - bowl_points[None, :, :]
        r = np.sqrt(np.sum(d * d, axis=2))
        out[s:s + chunk] = scale * np.sum(np.exp(1j * k * r) / (4.0 * math.pi * r), axis=1)
    return out


def incident_field(grid, bowl_points: np.ndarray, bowl, medium) -> np.ndarray:
    """p1 on every voxel centre of ``grid`` (shape grid.n)."""
    ax = [grid.origin[a] + grid.h * np.arange(grid.n[a], dtype=np.float64) for a in range(3)]
    X, Y, Z = np.meshgrid(*ax, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    return incident_field_at(xyz, bowl_points, bowl, medium).reshape(tuple(grid.n))
