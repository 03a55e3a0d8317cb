"""Parity at the full sizes of the 5-harmonic nested run, in the launch configuration
bench.py times: the 600 x 600 x 640 fundamental grid (embedding 1200 x 1200 x 1280: the
8-column column sweeps at L = 1200 and the pair-split z sweep at L = 1280) and the
320^3 ... 512^3 focal boxes of harmonics 2-5 (embeddings 640 ... 1024: the 8-line
pipelined z sweeps).

At these sizes the oracle's dense FFT route does not fit a test's budget, so the checks
are the ones that hold at any size:
- a sparse source (a seeded 16^3 block and the two far corners) applied by the plan on
  the whole grid, against the oracle's direct sum of Eq. 3.9 at sampled targets;
- the nested source of harmonic 5 (restriction of p1..p4 from their own grids fused with
  the products of Eq. 2.6), against the oracle's trilinear restriction and source term
  at sampled target voxels.
"""
import numpy as np
import pytest
import torch

from oracle import cascade, interp, physics, potential
from paper_2011_03009_gb300 import synth

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5


@pytest.fixture(scope="module")
def vp(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_03009_gb300 import vp as vpmod
    return vpmod


def _grid(harmonic):
    w = synth.WORKLOADS["nested5"]()
    if harmonic == 1:
        return w, w.v1_grid
    return w, {st.harmonic: st.grid for st in w.steps}[harmonic]


@pytest.mark.parametrize("harmonic", [1, 2, 3, 4, 5])
def test_sparse_source_at_full_size(vp, harmonic):
    w, g = _grid(harmonic)
    plan = vp.vp_plan(g, harmonic, w.bowl.f0, w.medium)
    plan.kernel_fft()
    m = tuple(plan.info().m)
    assert m == tuple(2 * v for v in g.n)  # the bench's embeddings
    idx, val = synth.sparse_block_source(g.n, 16, seed=300 + harmonic)
    val32 = val.astype(np.complex64)
    f = torch.zeros(g.n, dtype=torch.complex64, device="cuda")
    it = torch.from_numpy(idx).cuda()
    f[it[:, 0], it[:, 1], it[:, 2]] = torch.from_numpy(val32).cuda()
    u = torch.empty_like(f)
    plan.apply(f, u)
    tg = synth.sample_targets(g.n, idx, 1500, seed=400 + harmonic)
    tt = torch.from_numpy(tg).cuda()
    got = u[tt[:, 0], tt[:, 1], tt[:, 2]].cpu().numpy().astype(np.complex128)
    del f, u
    plan.close()
    torch.cuda.empty_cache()
    k = physics.wavenumber(harmonic, w.bowl.f0, w.medium)
    ref = potential.apply_sparse(idx, val32.astype(np.complex128), g.h, k, tg)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= REL_L2, rel
    assert np.max(np.abs(got - ref)) <= 2 * REL_L2 * np.max(np.abs(ref))


def _point_grid(g, v):
    """The one-voxel grid at voxel v of g (its centre, spacing kept)."""
    return synth.Grid((1, 1, 1), tuple(g.origin[a] + g.h * int(v[a]) for a in range(3)), g.h)


def test_harmonic5_nested_source_at_full_size(vp):
    """f5 = C5 (2 p1 p4 + 2 p2 p3) on the 512^3 grid from p1, p2 on the 320^3 grid of
    harmonic 2, p3 on 384^3 and p4 on 432^3, linear interpolation (Section 6)."""
    w = synth.WORKLOADS["nested5"]()
    grids = {st.harmonic: st.grid for st in w.steps}
    homes = [grids[2], grids[2], grids[3], grids[4]]  # p1, p2, p3, p4
    fields = [synth.random_field(g.n, seed=500 + i).astype(np.complex64) for i, g in enumerate(homes)]
    plan = vp.vp_plan(grids[5], 5, w.bowl.f0, w.medium)
    f5 = torch.empty(grids[5].n, dtype=torch.complex64, device="cuda")
    plan.source_from_nested(homes, [torch.from_numpy(a).cuda() for a in fields], f_out=f5)
    rng = np.random.default_rng(7)
    n5 = grids[5].n
    tg = np.concatenate([np.stack([rng.integers(0, n5[a], size=400) for a in range(3)], axis=1),
                         np.array([(x, y, z) for x in (0, n5[0] - 1) for y in (0, n5[1] - 1) for z in (0, n5[2] - 1)])])
    tt = torch.from_numpy(tg).cuda()
    got = f5[tt[:, 0], tt[:, 1], tt[:, 2]].cpu().numpy().astype(np.complex128)
    plan.close()
    ref = np.empty(len(tg), dtype=np.complex128)
    for i, v in enumerate(tg):
        pg = _point_grid(grids[5], v)
        lower = [interp.restrict_trilinear(fields[m].astype(np.complex128), homes[m], pg) for m in range(4)]
        ref[i] = cascade.source_term(5, lower, w.bowl.f0, w.medium)[0, 0, 0]
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= REL_L2, rel
    assert np.max(np.abs(got - ref)) <= 4 * REL_L2 * np.max(np.abs(ref))
