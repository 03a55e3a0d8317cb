"""Parity at the benchmark's full sizes, in the launch configuration bench.py times
(nested 128^3 / 192^3 / 256^3 grids, default embeddings, two-level engine).

The oracle's dense FFT route at these sizes (a 512^3 complex128 padded cube) takes
seconds on the GPU machine's host cores, so a dense smooth source is compared with it
element by element; besides, two checks that hold at any size are used:
- sparse sources: f = a few weighted point sources, whose potential at any voxel is the
  quadrature sum of Eq. 3.9 written out (h^3 G_k at the offset, the self-cell integral
  on the source voxel), evaluated by the oracle at sampled targets (including the
  sources themselves, their neighbours and the grid's far corners);
- homogeneity of the cascade (Eq. 2.6): scaling p1 by s scales p_n by s^n exactly.
"""
import numpy as np
import pytest
import torch

from oracle import greens, physics, potential
from paper_2011_03009_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vp(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_03009_gb300 import vp as vpmod
    return vpmod


def _targets(n, sources, rng, count=150):
    t = [tuple(int(rng.integers(0, n[a])) for a in range(3)) for _ in range(count)]
    corners = [(x, y, z) for x in (0, n[0] - 1) for y in (0, n[1] - 1) for z in (0, n[2] - 1)]
    near = []
    for s in sources:
        near.append(tuple(s))
        for a in range(3):
            for d in (-1, 1):
                q = list(s)
                q[a] = min(max(q[a] + d, 0), n[a] - 1)
                near.append(tuple(q))
    return np.array(t + corners + near)


@pytest.mark.parametrize("harmonic", [1, 2, 3])
def test_point_sources_at_full_size(vp, harmonic):
    wl = synth.WORKLOADS["nested3"]()
    g = wl.v1_grid if harmonic == 1 else [s.grid for s in wl.steps if s.harmonic == harmonic][0]
    n = g.n
    rng = np.random.default_rng(harmonic)
    src = np.array([[int(rng.integers(0, n[a])) for a in range(3)] for _ in range(5)])
    src[0] = (0, 0, 0)
    src[1] = (n[0] - 1, n[1] - 1, n[2] - 1)
    w = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    f = torch.zeros(n, dtype=torch.complex64, device="cuda")
    for (i, j, k), c in zip(src, w):
        f[i, j, k] = complex(c)
    plan = vp.vp_plan(g, harmonic, wl.bowl.f0, wl.medium)
    plan.kernel_fft()
    u = torch.empty_like(f)
    plan.apply(f, u)
    tg = _targets(n, src, rng)
    got = u[tg[:, 0], tg[:, 1], tg[:, 2]].cpu().numpy().astype(np.complex128)
    kn = physics.wavenumber(harmonic, wl.bowl.f0, wl.medium)
    w32 = w.astype(np.complex64).astype(np.complex128)
    ref = np.zeros(len(tg), dtype=np.complex128)
    for s, c in zip(src, w32):
        r = g.h * np.sqrt(np.sum((tg - s) ** 2, axis=1).astype(np.float64))
        same = r == 0
        val = np.where(same, greens.self_cell(kn, g.h), g.h ** 3 * greens.green(kn, np.where(same, 1.0, r)))
        ref += c * val
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, err
    # every sample individually, relative to the largest contribution of one source
    scale = np.max(np.abs(w32)) * abs(greens.self_cell(kn, g.h))
    assert np.max(np.abs(got - ref)) <= 2e-5 * scale
    plan.close()


def test_cascade_homogeneity_at_full_size(vp):
    """p1 -> 2 p1 gives p2 -> 4 p2 and p3 -> 8 p3 on the 192^3 / 256^3 grids, through
    restriction, the fused source and the apply (Eq. 2.6)."""
    wl = synth.WORKLOADS["nested3"]()
    g2 = wl.steps[0].grid
    g3 = wl.steps[1].grid
    pts = torch.from_numpy(synth.sample_bowl_points(wl.bowl, wl.n_points, wl.seed)).cuda()
    p1 = torch.empty(g2.n, dtype=torch.complex64, device="cuda")
    vp.vp_incident_field(g2, pts, wl.bowl, wl.medium, p1)
    plans = {2: vp.vp_plan(g2, 2, wl.bowl.f0, wl.medium), 3: vp.vp_plan(g3, 3, wl.bowl.f0, wl.medium)}
    for p in plans.values():
        p.kernel_fft()

    def chain(q1):
        p2 = torch.empty_like(q1)
        plans[2].source_assemble([q1])
        plans[2].apply(None, p2)
        r1 = torch.empty(g3.n, dtype=torch.complex64, device="cuda")
        r2 = torch.empty_like(r1)
        vp.vp_restrict_to_nested_box(g2, q1, g3, r1)
        vp.vp_restrict_to_nested_box(g2, p2, g3, r2)
        p3 = torch.empty_like(r1)
        plans[3].source_assemble([r1, r2])
        plans[3].apply(None, p3)
        return p2, p3

    a2, a3 = chain(p1)
    b2, b3 = chain(2 * p1)
    for a, b, s in ((a2, b2, 4.0), (a3, b3, 8.0)):
        rel = float((b - s * a).norm() / (s * a).norm())
        assert rel <= 1e-6, rel
    for p in plans.values():
        p.close()


@pytest.mark.parametrize("harmonic", [2, 3])
def test_dense_source_at_full_size_matches_oracle(vp, harmonic):
    """A dense smooth source on the full 192^3 / 256^3 grid (default embedding, the
    bench's launch configuration), every voxel against the oracle's FFT route."""
    w = synth.WORKLOADS["nested3"]()
    g = {st.harmonic: st.grid for st in w.steps}[harmonic]
    k = physics.wavenumber(harmonic, w.bowl.f0, w.medium)
    f = synth.smooth_blob_field(g, (w.bowl.l, 0.0, 0.0), 20 * g.h, k.real)
    ref = potential.apply_fft(f, g.h, k)
    plan = vp.vp_plan(g, harmonic, w.bowl.f0, w.medium)
    vp.vp_kernel_fft(plan)
    fd = torch.from_numpy(np.ascontiguousarray(f).astype(np.complex64)).cuda()
    u = torch.empty_like(fd)
    vp.vp_apply(plan, fd, u)
    got = u.cpu().numpy().astype(np.complex128)
    plan.close()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
