"""Evenly spaced monopole points on the bowl (Section 3, after Deserno's construction):
host checks of the point set, no GPU."""
import math

import numpy as np
import pytest

from paper_2011_03009_gb300 import synth


@pytest.mark.parametrize("bowl", [synth.H131, synth.H101, synth.Bowl(l=0.02, R=0.01, f0=1.0e6, p0=0.5e6)])
@pytest.mark.parametrize("n", [500, 2000, 4096, 20000])
def test_cap_points_lie_on_the_cap_and_match_the_count(bowl, n):
    p = synth.deserno_cap_points(bowl, n)
    assert abs(len(p) - n) <= 0.02 * n
    r = np.linalg.norm(p - np.array([bowl.l, 0.0, 0.0]), axis=1)
    assert np.allclose(r, bowl.l, rtol=1e-12, atol=0.0)
    # inside the cap: polar angle from the focus at most asin(R / l)
    theta = np.arccos(np.clip((bowl.l - p[:, 0]) / bowl.l, -1.0, 1.0))
    assert theta.max() <= math.asin(bowl.R / bowl.l) + 1e-12
    # rings of equally spaced points: the set is symmetric about the axis
    assert abs(p[:, 1].mean()) < 1e-12 * bowl.l and abs(p[:, 2].mean()) < 1e-12 * bowl.l


def test_cap_points_are_evenly_spaced():
    from scipy.spatial import cKDTree
    bowl = synth.H131
    n = 4096
    p = synth.deserno_cap_points(bowl, n)
    d, _ = cKDTree(p).query(p, k=2)
    nn = d[:, 1]
    # the spacing the construction aims at: sqrt of the cap area per point
    area = 2.0 * math.pi * bowl.l ** 2 * (1.0 - math.sqrt(1.0 - (bowl.R / bowl.l) ** 2))
    target = math.sqrt(area / n)
    med = np.median(nn)
    assert 0.7 * target < med < 1.2 * target
    assert nn.min() > 0.45 * med and nn.max() < 1.6 * med
