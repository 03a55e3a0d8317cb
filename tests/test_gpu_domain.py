"""Domain selection on the GPU (vp_q0_box) against the oracle, bit for bit: the same
FP64 decision on exact squares of the FP32 parts."""
import numpy as np
import pytest
import torch

from oracle import domain
from paper_2011_03009_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vp(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_03009_gb300 import vp as vpmod
    return vpmod


def _blob(n, seed):
    rng = np.random.default_rng(seed)
    axes = [np.arange(k) for k in n]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    c = [rng.uniform(0.3, 0.7) * k for k in n]
    w = [rng.uniform(0.1, 0.3) * k for k in n]
    env = np.exp(-((X - c[0]) ** 2 / w[0] ** 2 + (Y - c[1]) ** 2 / w[1] ** 2 + (Z - c[2]) ** 2 / w[2] ** 2))
    noise = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return (env * noise).astype(np.complex64)


@pytest.mark.parametrize("n", [(37, 29, 41), (1, 5, 3), (64, 64, 64), (150, 40, 33)])
def test_q0_box_matches_oracle(vp, n):
    f = _blob(n, sum(n))
    ft = torch.from_numpy(f).cuda()
    for q0 in (0.0, -0.5, -1.0, -2.0, -3.5, -8.0):
        lo, hi, m = vp.vp_q0_box(ft, q0)
        assert (lo, hi) == domain.q0_box(f, q0), (n, q0)
        assert abs(m - np.abs(f.astype(np.complex128)).max()) <= 1e-6 * m


def test_q0_box_zero_field_and_errors(vp):
    z = torch.zeros((4, 5, 6), dtype=torch.complex64, device="cuda")
    assert vp.vp_q0_box(z, -1.0)[:2] == ((0, 0, 0), (3, 4, 5))
    with pytest.raises(vp.VpError):
        vp.vp_q0_box(z, 0.5)


def test_q0_study_error_shrinks_with_the_box(vp):
    """Harmonic 3's source on its grid: a lower Q0 keeps a larger box and gives a smaller
    axis error; a box covering the whole grid reproduces the reference exactly."""
    from paper_2011_03009_gb300 import domain
    bowl = synth.Bowl(l=0.02, R=0.01, f0=1.0e6, p0=1.0e6)
    g2 = synth.focus_grid(bowl, (48, 40, 40), 2)
    g3 = synth.focus_grid(bowl, (48, 40, 40), 3)
    pts = torch.from_numpy(synth.sample_bowl_points(bowl, 1024, 3)).cuda()
    p1 = torch.empty(g2.n, dtype=torch.complex64, device="cuda")
    vp.vp_incident_field(g2, pts, bowl, synth.WATER, p1)
    plan2 = vp.vp_plan(g2, 2, bowl.f0, synth.WATER)
    plan2.kernel_fft()
    p2 = torch.empty_like(p1)
    plan2.source_assemble([p1])
    plan2.apply(None, p2)
    r1 = torch.empty(g3.n, dtype=torch.complex64, device="cuda")
    r2 = torch.empty_like(r1)
    vp.vp_restrict_to_nested_box(g2, p1, g3, r1)
    vp.vp_restrict_to_nested_box(g2, p2, g3, r2)
    plan3 = vp.vp_plan(g3, 3, bowl.f0, synth.WATER)
    f3 = torch.empty_like(r1)
    plan3.source_assemble([r1, r2], f_out=f3)
    rows = domain.q0_study(g3, 3, bowl.f0, f3, r1, [-0.5, -1.0, -2.0, -12.0])
    errs = [r["axis_error_pct"] for r in rows]
    fr = [r["volume_fraction"] for r in rows]
    assert all(e is not None for e in errs)
    assert fr == sorted(fr) and fr[-1] == 1.0
    assert errs[2] <= errs[0] and errs[-1] == 0.0
