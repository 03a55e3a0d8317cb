"""Linear (trilinear) interpolation of a field from one voxel grid onto a nested one (Section 6).

The paper interpolates each lower harmonic from the mesh it was computed on onto
the voxel centres of the next mesh with linear interpolation on a regular grid.
Reading where the paper is silent: the target centres must lie inside the box
spanned by the source centres (no extrapolation); the oracle raises otherwise.

For a target coordinate x on one axis, t = (x - o_src) / h_src; i0 = floor(t),
clamped to [0, N-2]; weight w = t - i0; the value is the tensor product of the
1-D linear interpolants (1 - w) v[i0] + w v[i0 + 1] over the three axes.
"""
from __future__ import annotations

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
