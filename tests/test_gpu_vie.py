"""Inhomogeneous-medium VIE (Section 7) solved on the GPU (vp_vie_solve, BiCGStab)
against the FP64 oracle (GMRES on the same discrete operator), and the residual of the
GPU solution measured with the FP64 operator."""
import numpy as np
import pytest
import torch

from oracle import physics, vie
from paper_2011_03009_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vp(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_03009_gb300 import vp as vpmod
    return vpmod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("n,harmonic", [((32, 28, 24), 1), ((20, 20, 20), 2)])
def test_vie_matches_oracle(vp, n, harmonic):
    f0 = 1.0e6
    h = synth.wavelength(synth.WATER.c0, f0, harmonic) / 6
    g = synth.centred_grid(n, h, (0.0, 0.0, 0.0))
    kk = vie.sphere_wavenumber(g, (0.3 * h, -0.2 * h, 0.0), 0.3 * min(n) * h, harmonic, f0, synth.WATER,
                               synth.TISSUE)
    kb = physics.wavenumber(harmonic, f0, synth.WATER)
    q = vie.contrast(kk, kb)
    b = synth.random_field(n, 21)
    q32, b32 = q.astype(np.complex64).astype(np.complex128), b.astype(np.complex64).astype(np.complex128)
    ref = vie.solve(q32, b32, g.h, kb)
    plan = vp.vp_plan(g, harmonic, f0, synth.WATER)
    plan.kernel_fft()
    x = torch.zeros(n, dtype=torch.complex64, device="cuda")
    it, res = plan.vie_solve(dev(q), dev(b), x, tol=1e-7, max_iter=300)
    got = host(x)
    assert res <= 1e-6 and it >= 1
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    # FP64 residual of the GPU solution
    r = b32.reshape(-1) - vie.operator(q32, g.h, kb)(got)
    assert np.linalg.norm(r) / np.linalg.norm(b32) <= 2e-6
    # zero contrast: x = b in one step
    it0, res0 = plan.vie_solve(dev(np.zeros(n)), dev(b), x, tol=1e-7)
    assert np.linalg.norm(host(x) - b32) / np.linalg.norm(b32) <= 1e-6
    plan.close()


def test_vie_zero_right_hand_side_and_bad_arguments(vp):
    g = synth.centred_grid((12, 10, 8), 2e-4, (0.0, 0.0, 0.0))
    plan = vp.vp_plan(g, 1, 1.0e6, synth.WATER)
    q = torch.ones(g.n, dtype=torch.complex64, device="cuda") * 1e4
    b = torch.zeros(g.n, dtype=torch.complex64, device="cuda")
    x = torch.ones_like(b)
    with pytest.raises(vp.VpError):       # spectrum not built
        plan.vie_solve(q, b, x)
    plan.kernel_fft()
    it, res = plan.vie_solve(q, b, x)
    torch.cuda.synchronize()
    assert it == 0 and res == 0.0 and float(x.abs().max()) == 0.0
    with pytest.raises(vp.VpError):
        plan.vie_solve(q, b, x, tol=0.0)
    plan.close()
