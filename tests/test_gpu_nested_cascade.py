"""Section 6's nested loop through the product driver (cascade.NestedCascade: restriction
fused with the source products, then the volume potential) against the oracle's loop,
harmonics 2-4 on nested focal grids, with linear and quadratic inter-mesh interpolation."""
import numpy as np
import pytest
import torch

from oracle import cascade as ocascade, interp, rayleigh
from paper_2011_03009_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cascade(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_03009_gb300 import cascade as cmod
    return cmod


@pytest.mark.parametrize("quadratic", [False, True])
def test_nested_cascade_matches_oracle_loop(cascade, quadratic):
    bowl = synth.Bowl(l=0.02, R=0.01, f0=1.0e6, p0=0.5e6)
    grids = {n: synth.focus_grid(bowl, (s, s + 3, s - 2), n) for n, s in ((2, 24), (3, 28), (4, 32))}
    pts = synth.sample_bowl_points(bowl, 400, seed=9)
    p1 = rayleigh.incident_field(grids[2], pts, bowl, synth.WATER)
    restrict = interp.restrict_quadratic if quadratic else interp.restrict_trilinear
    ref = ocascade.nested_run(p1, grids, bowl.f0, synth.WATER, restrict=restrict)
    run = cascade.NestedCascade(grids, bowl.f0, synth.WATER, quadratic=quadratic)
    out = run.run(torch.from_numpy(p1.astype(np.complex64)).cuda())
    torch.cuda.synchronize()
    for n, want in ref.items():
        got = out[n].cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-5, n
    run.close()


def test_nested_cascade_rejects_a_gap_in_the_harmonics(cascade):
    bowl = synth.Bowl(l=0.02, R=0.01, f0=1.0e6, p0=0.5e6)
    grids = {2: synth.focus_grid(bowl, (8, 8, 8), 2), 4: synth.focus_grid(bowl, (8, 8, 8), 4)}
    with pytest.raises(ValueError):
        cascade.NestedCascade(grids, bowl.f0, synth.WATER)
