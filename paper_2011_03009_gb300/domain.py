"""Integration-domain selection for the harmonics (Section 5) through the C ABI.

Two pieces:
- the rule of thumb for nested domains: with D_2 = [L + d, w, w] (L before the focus,
  d beyond it, w across), harmonic i gets [(lambda_i/lambda_2) L + d,
  (lambda_i/lambda_2) w, (lambda_i/lambda_2) w], meshed at lambda_i / 6;
- the Q0 study: for a harmonic's source f on a reference grid, the smallest box D with
  log10(|f| / max|f|) < Q0 outside it (vp_q0_box), the harmonic recomputed with the
  source restricted to D, and its error against the reference on the voxel line
  nearest the axis, relative to the fundamental there (the error measure of Section 5).
- the mesh-refinement study (Section 3, "how many points per wavelength"): the second
  harmonic on meshes of h = lambda / (2 n_w) over one fixed box, against a finely meshed
  reference, with its error along the x axis and the fitted convergence order.
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


def nw_grid(bowl: synth.Bowl, medium: synth.Medium, n_w: int, q: Sequence[int], x_start: float) -> synth.Grid:
    """Mesh of the box [x_start, x_start + q_x lambda / 2] x [-q_y lambda / 4, q_y lambda / 4]
    x [-q_z lambda / 4, q_z lambda / 4] (lambda the fundamental wavelength) at
    h = lambda / (2 n_w): n = n_w q voxels, so every n_w covers exactly the same box, and
    with n_w, q_y, q_z odd the x axis is a voxel line."""
    lam = synth.wavelength(medium.c0, bowl.f0, 1)
    h = lam / (2 * n_w)
    n = tuple(int(n_w) * int(v) for v in q)
    origin = (x_start + 0.5 * h, -0.5 * (n[1] - 1) * h, -0.5 * (n[2] - 1) * h)
    return synth.Grid(n, origin, h)


def second_harmonic(g: synth.Grid, bowl: synth.Bowl, pts: torch.Tensor, medium: synth.Medium):
    """p1 on g from the bowl points (Eq. 3.10) and p2 = V_{k2}[C_2 p1^2] (Eq. 3.5)."""
    p1 = torch.empty(g.n, dtype=torch.complex64, device=pts.device)
    vp.vp_incident_field(g, pts, bowl, medium, p1)
    plan = vp.vp_plan(g, 2, bowl.f0, medium)
    plan.kernel_fft()
    p2 = torch.empty_like(p1)
    plan.source_assemble([p1])
    plan.apply(None, p2)
    plan.close()
    return p1, p2


def nw_study(bowl: synth.Bowl, medium: synth.Medium, n_ws: Sequence[int], n_w_ref: int, q: Sequence[int],
             x_start: float, n_points: int = 4096) -> dict:
    """Relative L2 error (%) of p2 along the x axis for each n_w against the n_w_ref mesh.

    The monopoles sit at Deserno-spaced points of the bowl.  The reference axis line is
    interpolated by a cubic spline to each mesh's own axis nodes (interpolation error
    ~ (k h_ref)^4, far below the errors measured), and the error is the discrete L2 norm
    over those nodes (the midpoint rule along x).  The fitted order is the least-squares
    slope of -log(error) against log(n_w)."""
    from scipy.interpolate import CubicSpline
    dev = torch.device("cuda", torch.cuda.current_device())
    pts = torch.from_numpy(synth.deserno_cap_points(bowl, n_points)).to(dev)
    for v in (n_w_ref, *n_ws):
        if v % 2 == 0:
            raise ValueError("n_w must be odd, so that the x axis is a voxel line")
    if q[1] % 2 == 0 or q[2] % 2 == 0:
        raise ValueError("q_y and q_z must be odd")

    def axis_values(g, p2):
        return p2[:, (g.n[1] - 1) // 2, (g.n[2] - 1) // 2].cpu().numpy().astype(np.complex128)

    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    g_ref = nw_grid(bowl, medium, n_w_ref, q, x_start)
    t0.record()
    _, p2_ref = second_harmonic(g_ref, bowl, pts, medium)
    t1.record()
    torch.cuda.synchronize()
    ref_ms = t0.elapsed_time(t1)
    spline = CubicSpline(g_ref.axis(0), axis_values(g_ref, p2_ref))
    del p2_ref
    rows = []
    for n_w in n_ws:
        g = nw_grid(bowl, medium, n_w, q, x_start)
        t0.record()
        _, p2 = second_harmonic(g, bowl, pts, medium)
        t1.record()
        torch.cuda.synchronize()
        got = axis_values(g, p2)
        ref = spline(g.axis(0))
        err = 100.0 * float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        rows.append({"n_w": int(n_w), "h_um": 1e6 * g.h, "grid": list(g.n), "error_pct": err,
                     "ms": t0.elapsed_time(t1)})
    def fit(sel):
        if len(sel) < 2:
            return None
        x = np.log(np.array([r["n_w"] for r in sel], dtype=np.float64))
        y = np.log(np.array([r["error_pct"] for r in sel], dtype=np.float64))
        return float(-np.polyfit(x, y, 1)[0])

    # the reference's own error flattens the finest meshes' errors away from the trend;
    # the order over meshes at most half as fine as the reference is the cleaner estimate
    return {"rows": rows, "order": fit(rows), "order_coarse": fit([r for r in rows if 2 * r["n_w"] <= n_w_ref]),
            "n_w_ref": int(n_w_ref), "ref_grid": list(g_ref.n), "ref_ms": ref_ms, "points": int(pts.shape[0])}
