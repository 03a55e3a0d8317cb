"""Integration-domain selection for the harmonics (Section 5) through the C ABI.

Two pieces:
- the rule of thumb for nested domains: with D_2 = [L + d, w, w] (L before the focus,
  d beyond it, w across), harmonic i gets [(lambda_i/lambda_2) L + d,
  (lambda_i/lambda_2) w, (lambda_i/lambda_2) w], meshed at lambda_i / 6;
- the Q0 study: for a harmonic's source f on a reference grid, the smallest box D with
  log10(|f| / max|f|) < Q0 outside it (vp_q0_box), the harmonic recomputed with the
  source restricted to D, and its error against the reference on the voxel line
  nearest the axis, relative to the fundamental there (the error measure of Section 5).
Every field operation runs in libvp.so; this module chooses grids and orders calls.
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence

import numpy as np
import torch

from . import synth, vp


def rule_of_thumb_grids(bowl: synth.Bowl, L: float, d: float, w: float, harmonics: Sequence[int],
                        medium=synth.WATER) -> Dict[int, synth.Grid]:
    """Grids of the rule of thumb: x in [l - s L, l + d], y, z in [-s w / 2, s w / 2] with
    s = lambda_i / lambda_2, spacing lambda_i / 6 (voxel centres inside the box)."""
    lam2 = synth.wavelength(medium.c0, bowl.f0, 2)
    out = {}
    for i in harmonics:
        lam = synth.wavelength(medium.c0, bowl.f0, i)
        s = lam / lam2
        h = lam / 6
        x0, x1 = bowl.l - s * L, bowl.l + d
        nx = max(1, int(math.floor((x1 - x0) / h)) + 1)
        nt = max(1, int(math.floor(s * w / h)) + 1)
        origin = (x0, -0.5 * (nt - 1) * h, -0.5 * (nt - 1) * h)
        out[i] = synth.Grid((nx, nt, nt), origin, h)
    return out


def box_grid(g: synth.Grid, lo, hi) -> synth.Grid:
    """Sub-grid of g with voxel index bounds lo..hi (inclusive); centres coincide with g's."""
    n = tuple(int(hi[a] - lo[a] + 1) for a in range(3))
    origin = tuple(g.origin[a] + lo[a] * g.h for a in range(3))
    return synth.Grid(n, origin, g.h)


def axis_line(g: synth.Grid):
    """(iy, iz) of the voxel line nearest the x axis (y = z = 0)."""
    iy = int(round(-g.origin[1] / g.h))
    iz = int(round(-g.origin[2] / g.h))
    return min(max(iy, 0), g.n[1] - 1), min(max(iz, 0), g.n[2] - 1)


def q0_study(g: synth.Grid, harmonic: int, f0: float, f: torch.Tensor, p1: torch.Tensor,
             q0_values: Sequence[float], medium=synth.WATER) -> List[dict]:
    """Error of p_n computed from the source restricted to the Q0 box, per Q0.

    g: reference grid of harmonic n; f: the source f_n on g (complex64, device);
    p1: the fundamental on g (for the error's denominator)."""
    ref_plan = vp.vp_plan(g, harmonic, f0, medium)
    ref_plan.kernel_fft()
    p_ref = torch.empty_like(f)
    ref_plan.apply(f, p_ref)
    ref_plan.close()
    iy, iz = axis_line(g)
    rows = []
    for q0 in q0_values:
        lo, hi, _ = vp.vp_q0_box(f, q0)
        d = box_grid(g, lo, hi)
        f_d = torch.empty(d.n, dtype=torch.complex64, device=f.device)
        vp.vp_restrict_to_nested_box(g, f, d, f_d)  # coincident centres: an exact copy
        plan = vp.vp_plan(d, harmonic, f0, medium)
        plan.kernel_fft()
        p_d = torch.empty_like(f_d)
        plan.apply(f_d, p_d)
        plan.close()
        row = {"q0": q0, "box_lo": list(lo), "box_hi": list(hi), "box_n": list(d.n),
               "volume_fraction": float(np.prod(d.n) / np.prod(g.n))}
        if lo[1] <= iy <= hi[1] and lo[2] <= iz <= hi[2]:
            a = p_d[:, iy - lo[1], iz - lo[2]].cpu().numpy().astype(np.complex128)
            r = p_ref[lo[0]:hi[0] + 1, iy, iz].cpu().numpy().astype(np.complex128)
            den = p1[lo[0]:hi[0] + 1, iy, iz].cpu().numpy().astype(np.complex128)
            row["axis_error_pct"] = float(100.0 * np.linalg.norm(a - r) / np.linalg.norm(den))
        else:
            row["axis_error_pct"] = None
        rows.append(row)
    return rows
