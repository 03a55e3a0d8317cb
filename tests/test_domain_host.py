"""Host logic of the domain driver: the rule of thumb for nested domains (Section 5)
and the sub-grid bookkeeping of the Q0 study."""
import math

import pytest

pytest.importorskip("torch")

from paper_2011_03009_gb300 import synth  # noqa: E402


def _domain():
    import importlib
    try:
        return importlib.import_module("paper_2011_03009_gb300.domain")
    except ImportError as e:  # the library must be built for the module to import
        pytest.skip(str(e))


def test_rule_of_thumb_keeps_voxel_counts_nearly_equal():
    domain = _domain()
    bowl = synth.Bowl(l=0.06, R=0.03, f0=1.1e6, p0=1e6)
    L, d, w = 0.03, 0.01, 0.02
    g = domain.rule_of_thumb_grids(bowl, L, d, w, [2, 3, 4, 5])
    lam = {i: synth.wavelength(1500.0, bowl.f0, i) for i in g}
    counts = {i: g[i].n[0] * g[i].n[1] * g[i].n[2] for i in g}
    for i in g:
        s = lam[i] / lam[2]
        assert g[i].h == pytest.approx(lam[i] / 6)
        # x from l - s L to at most l + d; transverse extent s w
        assert g[i].origin[0] == pytest.approx(bowl.l - s * L)
        assert g[i].origin[0] + (g[i].n[0] - 1) * g[i].h <= bowl.l + d + 1e-12
        assert (g[i].n[1] - 1) * g[i].h <= s * w + 1e-12
    # only the unscaled length d makes the counts grow with i (Section 5)
    assert all(counts[i + 1] >= counts[i] * 0.98 for i in (2, 3, 4))
    assert counts[5] < 1.6 * counts[2]


def test_box_grid_and_axis_line():
    domain = _domain()
    g = synth.Grid((20, 11, 9), (0.01, -5e-4, -4e-4), 1e-4)
    sub = domain.box_grid(g, (3, 2, 1), (10, 8, 7))
    assert sub.n == (8, 7, 7)
    assert sub.origin[0] == pytest.approx(0.01 + 3e-4) and sub.origin[1] == pytest.approx(-3e-4)
    assert domain.axis_line(g) == (5, 4)


def test_refinement_meshes_cover_one_box():
    """Every n_w mesh of the refinement study covers the same box, with the x axis on a
    voxel line (host logic, no GPU)."""
    domain = _domain()
    bowl, med = synth.H131, synth.LIVER
    lam = synth.wavelength(med.c0, bowl.f0, 1)
    x0 = bowl.l - 2 * lam
    for n_w in (5, 9, 21, 35):
        g = domain.nw_grid(bowl, med, n_w, (6, 3, 3), x0)
        assert g.n == (6 * n_w, 3 * n_w, 3 * n_w)
        assert math.isclose(g.h, lam / (2 * n_w), rel_tol=1e-15)
        lo = [g.origin[a] - 0.5 * g.h for a in range(3)]
        hi = [g.origin[a] + (g.n[a] - 0.5) * g.h for a in range(3)]
        assert math.isclose(lo[0], x0, abs_tol=1e-12) and math.isclose(hi[0], x0 + 3 * lam, rel_tol=1e-12)
        assert math.isclose(hi[1], 0.75 * lam, rel_tol=1e-12) and math.isclose(lo[1], -0.75 * lam, rel_tol=1e-12)
        assert abs(g.origin[1] + (g.n[1] - 1) // 2 * g.h) < 1e-15  # the axis is a voxel line
