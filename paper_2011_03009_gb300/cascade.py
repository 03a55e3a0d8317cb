"""Harmonic cascades through the C ABI (include/vp.h).

NestedCascade: the weakly nonlinear cascade of Section 6 on nested per-harmonic grids.

FullCascade: the full harmonic cascade with conjugate terms (Eq. 2.5) by fixed-point
iteration, on one grid.

The weakly nonlinear cascade (Eq. 2.6) keeps only the products p_m p_{n-m}, m < n;
Eq. 2.5 also keeps 2 p_m conj(p_{m-n}) for m > n, so every harmonic, the fundamental
included, depends on the ones above it.  The system is solved by Jacobi iteration:
    p_1 <- p_inc + V_{k_1}[f_1(p)],   p_n <- V_{k_n}[f_n(p)]  (n = 2..N_h),
started from the weakly nonlinear solution.  Every step runs in libvp.so's kernels
(vp_source_assemble with VP_SRC_CONJ, vp_apply, vp_vec_*); this module orders calls.
"""
from __future__ import annotations

from typing import Dict, List

import torch

from . import vp


class NestedCascade:
    """Section 6's loop: p1 on the grid of harmonic 2, then for n = 2..N each p_n on its
    own grid from the source of the lower harmonics (Eq. 2.6), every p_m restricted from
    its grid to grid n inside the source kernel (vp_source_from_nested) where it lives
    elsewhere, and the volume potential (vp_apply).

    grids: {n: grid of harmonic n} for n = 2..N.  One plan per harmonic, its kernel
    spectrum built once; run() reuses them for any p1 on grids[2]."""

    def __init__(self, grids: Dict[int, object], f0: float, medium, quadratic: bool = False, device="cuda"):
        self.grids = {int(n): g for n, g in grids.items()}
        if not self.grids or min(self.grids) != 2 or sorted(self.grids) != list(range(2, max(self.grids) + 1)):
            raise ValueError("grids must hold harmonics 2..N")
        self.quadratic = quadratic
        self.plans = {n: vp.vp_plan(g, n, f0, medium) for n, g in self.grids.items()}
        for p in self.plans.values():
            p.kernel_fft()
        self.out = {n: torch.empty(tuple(int(v) for v in g.n), dtype=torch.complex64, device=device)
                    for n, g in self.grids.items()}

    def run(self, p1: torch.Tensor, stream=None) -> Dict[int, torch.Tensor]:
        """p_n on grids[n] for n = 2..N from p1 on grids[2] (the returned tensors are the
        cascade's own buffers, overwritten by the next run)."""
        fields = {1: (p1, self.grids[2])}
        for n in sorted(self.grids):
            g, plan = self.grids[n], self.plans[n]
            lower = [fields[m] for m in range(1, n)]
            if all(h is g for _, h in lower):  # all on grid n: no restriction
                plan.source_assemble([f for f, _ in lower], stream=stream)
            else:
                plan.source_from_nested([h for _, h in lower], [f for f, _ in lower], quadratic=self.quadratic,
                                        stream=stream)
            plan.apply(None, self.out[n], stream=stream)
            fields[n] = (self.out[n], g)
        return self.out

    def close(self):
        for p in self.plans.values():
            p.close()


class FullCascade:
    def __init__(self, grid, nh: int, f0: float, medium, device="cuda"):
        if not 2 <= nh <= vp.MAX_LOWER:
            raise ValueError("N_h must be in 2..8")
        self.nh = nh
        self.grid = grid
        self.plans = [vp.vp_plan(grid, n, f0, medium) for n in range(1, nh + 1)]
        for p in self.plans:
            p.kernel_fft()
        shape = tuple(int(v) for v in grid.n)
        mk = lambda: torch.zeros(shape, dtype=torch.complex64, device=device)
        self.p: List[torch.Tensor] = [mk() for _ in range(nh)]
        self.q: List[torch.Tensor] = [mk() for _ in range(nh)]
        self.tmp = mk()

    def weakly_nonlinear(self, p_inc: torch.Tensor) -> List[torch.Tensor]:
        """The Eq. 2.6 cascade: p_1 = p_inc, p_n = V[C_n sum_{m<n} p_m p_{n-m}]."""
        vp.vp_vec_axpby(1.0, p_inc, 0.0, None, self.p[0])
        for n in range(2, self.nh + 1):
            plan = self.plans[n - 1]
            plan.source_assemble(self.p[:n - 1])
            plan.apply(None, self.p[n - 1])
        return self.p

    def sweep(self, p_inc: torch.Tensor) -> float:
        """One Jacobi sweep of Eq. 2.5; returns max_n ||p_n^new - p_n|| / ||p_n^new||."""
        for n in range(1, self.nh + 1):
            plan = self.plans[n - 1]
            plan.source_assemble(self.p, conj=True)
            plan.apply(None, self.q[n - 1])
        vp.vp_vec_axpby(1.0, self.q[0], 1.0, p_inc, self.q[0])
        change = 0.0
        for n in range(self.nh):
            vp.vp_vec_axpby(1.0, self.q[n], -1.0, self.p[n], self.tmp)
            d = vp.vp_vec_dot(self.tmp, self.tmp).real
            s = vp.vp_vec_dot(self.q[n], self.q[n]).real
            change = max(change, (d / s) ** 0.5 if s > 0 else 0.0)
        self.p, self.q = self.q, self.p
        return change

    def run(self, p_inc: torch.Tensor, max_iter: int = 50, tol: float = 1e-6, start: bool = True):
        """Iterate from the weakly nonlinear solution until the relative change < tol."""
        if start:
            self.weakly_nonlinear(p_inc)
        hist = []
        for _ in range(max_iter):
            hist.append(self.sweep(p_inc))
            if hist[-1] < tol:
                break
        return self.p, hist

    def close(self):
        for p in self.plans:
            p.close()
