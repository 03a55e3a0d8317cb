"""Linear (trilinear) and quadratic interpolation of a field from one voxel grid onto a
nested one (Section 6; test infrastructure only).

The paper interpolates each lower harmonic from the mesh it was computed on onto
the voxel centres of the next mesh with linear interpolation on a regular grid.
Reading where the paper is silent: the target centres must lie inside the box
spanned by the source centres (no extrapolation); the oracle raises otherwise.

For a target coordinate x on one axis, t = (x - o_src) / h_src; i0 = floor(t),
clamped to [0, N-2]; weight w = t - i0; the value is the tensor product of the
1-D linear interpolants (1 - w) v[i0] + w v[i0 + 1] over the three axes.

Quadratic (the higher-order option Section 6 mentions): per axis the Lagrange
polynomial through the three nearest source centres c - 1, c, c + 1 with
c = floor(t + 1/2) clamped to [1, N-2], evaluated at u = t - c.  At a half-integer t
two stencils are equally near and the paper does not say which to take; both are
valid.  Two ways of locating the targets are offered:
- positions="float": t from the plain FP64 formula; at a target within TIE_TOL of a
  half-integer the caller picks the stencil below (tie="down") or above (tie="up");
- positions="fixed" (default): t held as an exact 40-bit fixed-point number (the
  positions the C interface defines), so that a cascade compared voxel by voxel sees
  the same stencil decision on both sides.  The pins check that the fixed positions
  give the float positions' stencil and weights away from ties, and one of the two
  valid stencils at a tie.
"""
from __future__ import annotations

import math

import numpy as np

TOL = 1.0e-9


def _axis_weights(src_origin: float, src_h: float, src_n: int, dst_coords: np.ndarray):
    t = (dst_coords - src_origin) / src_h
    if src_n == 1:
        if np.any(np.abs(t) > TOL):
            raise ValueError("target outside the source grid")
        return np.zeros(len(t), dtype=np.int64), np.zeros(len(t)), True
    if np.any(t < -TOL) or np.any(t > (src_n - 1) + TOL):
        raise ValueError("target outside the source grid")
    t = np.clip(t, 0.0, src_n - 1.0)
    i0 = np.minimum(np.floor(t).astype(np.int64), src_n - 2)
    w = t - i0
    return i0, w, False


def restrict_trilinear(src: np.ndarray, src_grid, dst_grid) -> np.ndarray:
    """Values of the trilinear interpolant of ``src`` (on src_grid) at dst_grid's voxel centres."""
    src = np.asarray(src, dtype=np.complex128)
    idx, wts, single = [], [], []
    for a in range(3):
        coords = dst_grid.origin[a] + dst_grid.h * np.arange(dst_grid.n[a], dtype=np.float64)
        i0, w, s = _axis_weights(src_grid.origin[a], src_grid.h, src_grid.n[a], coords)
        idx.append(i0)
        wts.append(w)
        single.append(s)
    out = np.zeros(tuple(dst_grid.n), dtype=np.complex128)
    for cx in (0, 1):
        if single[0] and cx:
            continue
        wx = (1.0 - wts[0]) if cx == 0 else wts[0]
        ix = idx[0] + cx
        for cy in (0, 1):
            if single[1] and cy:
                continue
            wy = (1.0 - wts[1]) if cy == 0 else wts[1]
            iy = idx[1] + cy
            for cz in (0, 1):
                if single[2] and cz:
                    continue
                wz = (1.0 - wts[2]) if cz == 0 else wts[2]
                iz = idx[2] + cz
                w = wx[:, None, None] * wy[None, :, None] * wz[None, None, :]
                out += w * src[np.ix_(ix, iy, iz)]
    return out


FIX_BITS = 40


def _round_half_away(x: float) -> int:
    return int(math.floor(x + 0.5)) if x >= 0 else -int(math.floor(-x + 0.5))


def _fixed_positions(src_origin: float, src_h: float, dst_origin: float, dst_h: float, count: int) -> np.ndarray:
    """Target positions in source-voxel units as exact integers with FIX_BITS fractional
    bits: T_i = round(a 2^F) + i round(b 2^F), a = (o_dst - o_src) / h_src, b = h_dst / h_src.
    The quadratic stencil's centre is a discontinuous function of t (at half-integers),
    so it is decided on these exact positions, as the header of the C interface defines."""
    a = (dst_origin - src_origin) / src_h
    b = dst_h / src_h
    A = _round_half_away(a * 2.0 ** FIX_BITS)
    B = _round_half_away(b * 2.0 ** FIX_BITS)
    return np.array([A + i * B for i in range(count)], dtype=object)


TIE_TOL = 1.0e-9


def _axis_quadratic(src_origin: float, src_h: float, src_n: int, dst_coords: np.ndarray, T=None, tie="down"):
    """Indices (k, 3) and weights (k, 3) of the quadratic Lagrange interpolant through the
    three source centres nearest to each target; a two-centre axis stays linear and a
    one-centre axis takes its only value.  T: exact fixed-point positions (optional);
    without them, t within TIE_TOL of a half-integer takes the stencil ``tie`` names."""
    t = (dst_coords - src_origin) / src_h
    k = len(t)
    if src_n < 3:
        i0, w, single = _axis_weights(src_origin, src_h, src_n, dst_coords)
        idx = np.stack([i0, i0 + (0 if single else 1), i0 + (0 if single else 1)], axis=1)
        wts = np.stack([1.0 - w if not single else np.ones(k), w if not single else np.zeros(k), np.zeros(k)], axis=1)
        return idx, wts
    if np.any(t < -TOL) or np.any(t > (src_n - 1) + TOL):
        raise ValueError("target outside the source grid")
    if T is None:
        lo = np.floor(t).astype(np.int64)
        at_tie = np.abs(t - lo - 0.5) <= TIE_TOL
        c = np.where(at_tie, lo + (1 if tie == "up" else 0), np.floor(t + 0.5).astype(np.int64))
        c = np.clip(c, 1, src_n - 2)
        u = t - c
    else:
        half = 1 << (FIX_BITS - 1)
        c = np.array([min(max((int(v) + half) >> FIX_BITS, 1), src_n - 2) for v in T], dtype=np.int64)
        u = np.array([(int(v) - (int(ci) << FIX_BITS)) / 2.0 ** FIX_BITS for v, ci in zip(T, c)])
    # Lagrange basis on the nodes -1, 0, 1
    l_m = u * (u - 1.0) / 2.0
    l_0 = (1.0 - u) * (1.0 + u)
    l_p = u * (u + 1.0) / 2.0
    return np.stack([c - 1, c, c + 1], axis=1), np.stack([l_m, l_0, l_p], axis=1)


def tie_axes(src_grid, dst_grid):
    """Per axis, a boolean mask of the targets within TIE_TOL of a half-integer source
    position (where two quadratic stencils are equally near)."""
    out = []
    for a in range(3):
        coords = dst_grid.origin[a] + dst_grid.h * np.arange(dst_grid.n[a], dtype=np.float64)
        t = (coords - src_grid.origin[a]) / src_grid.h
        out.append(np.abs(t - np.floor(t) - 0.5) <= TIE_TOL if src_grid.n[a] >= 3 else np.zeros(len(t), bool))
    return out


def restrict_quadratic(src: np.ndarray, src_grid, dst_grid, positions: str = "fixed", tie=("down",) * 3) -> np.ndarray:
    """Values of the tensor-product quadratic interpolant of ``src`` at dst_grid's centres.

    positions="fixed": the stencil centres from the exact fixed-point positions;
    positions="float": from the FP64 positions, with tie[a] ("down" or "up") choosing the
    stencil on axis a at half-integer positions."""
    src = np.asarray(src, dtype=np.complex128)
    if positions not in ("fixed", "float"):
        raise ValueError("positions must be 'fixed' or 'float'")
    idx, wts = [], []
    for a in range(3):
        coords = dst_grid.origin[a] + dst_grid.h * np.arange(dst_grid.n[a], dtype=np.float64)
        T = None
        if positions == "fixed":
            T = _fixed_positions(src_grid.origin[a], src_grid.h, dst_grid.origin[a], dst_grid.h, dst_grid.n[a])
        i, w = _axis_quadratic(src_grid.origin[a], src_grid.h, src_grid.n[a], coords, T, tie[a])
        idx.append(i)
        wts.append(w)
    out = np.zeros(tuple(dst_grid.n), dtype=np.complex128)
    for p in range(3):
        for q in range(3):
            for r in range(3):
                w = wts[0][:, p][:, None, None] * wts[1][:, q][None, :, None] * wts[2][:, r][None, None, :]
                out += w * src[np.ix_(idx[0][:, p], idx[1][:, q], idx[2][:, r])]
    return out
