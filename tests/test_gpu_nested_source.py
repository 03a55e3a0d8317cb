"""The source of harmonic n from lower harmonics on their own nested grids, against the
oracle: each p_m restricted to the plan's grid (Section 6, step 2a) and the products of
Eq. 2.6 formed there, in one kernel (vp_source_from_nested)."""
import numpy as np
import pytest
import torch

from oracle import cascade, interp
from paper_2011_03009_gb300 import synth

pytestmark = pytest.mark.gpu

F0 = 1.1e6


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


def rel_l2(got, ref):
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def oracle_source(harmonic, grids, fields, target, quadratic=False):
    restrict = interp.restrict_quadratic if quadratic else interp.restrict_trilinear
    lower = [restrict(f, g, target) for f, g in zip(fields, grids)]
    return cascade.source_term(harmonic, lower, F0, synth.WATER)


# a coarse p1 box, a finer p2 box inside it, the target (finer still) inside both; the
# target spans several 16 x 64 blocks with ragged ends
G1 = synth.Grid((12, 16, 28), (0.0, 0.0, 0.0), 3.0e-4)
G2 = synth.Grid((14, 20, 38), (0.0002, 0.0003, 0.0004), 2.0e-4)
TARGET = synth.Grid((23, 37, 75), (0.0005, 0.0006, 0.0009), 0.8e-4)


@pytest.mark.parametrize("quadratic", [False, True])
def test_nested_source_matches_oracle(vp, quadratic):
    fields = [synth.random_field(G1.n, seed=41), synth.random_field(G2.n, seed=42)]
    plan = vp.vp_plan(TARGET, 3, F0, synth.WATER)
    f = torch.empty(TARGET.n, dtype=torch.complex64, device="cuda")
    plan.source_from_nested([G1, G2], [dev(x) for x in fields], f_out=f, quadratic=quadratic)
    ref = oracle_source(3, [G1, G2], fields, TARGET, quadratic)
    assert rel_l2(host(f), ref) <= 1e-6
    plan.close()


@pytest.mark.parametrize("harmonic", [2, 4, 5])
def test_nested_source_every_harmonic_with_a_same_grid_field(vp, harmonic):
    """p_1 on the coarse box, the others alternating between the finer box and the
    target grid itself (an identity restriction)."""
    grids = [G1] + [G2 if m % 2 == 0 else TARGET for m in range(2, harmonic)]
    fields = [synth.random_field(g.n, seed=50 + m) for m, g in enumerate(grids)]
    plan = vp.vp_plan(TARGET, harmonic, F0, synth.WATER)
    f = torch.empty(TARGET.n, dtype=torch.complex64, device="cuda")
    plan.source_from_nested(grids, [dev(x) for x in fields], f_out=f)
    ref = oracle_source(harmonic, grids, fields, TARGET)
    assert rel_l2(host(f), ref) <= 1e-6
    plan.close()


@pytest.mark.parametrize("quadratic", [False, True])
def test_nested_source_from_a_one_voxel_axis(vp, quadratic):
    """A source one voxel thick along x (one-point stencils there) takes the tiled kernel
    with per-target stencil sizes; sources with two voxels or more on every axis (the
    other tests, the runs) take the linear kernel without them."""
    src = synth.Grid((1, 16, 28), (0.0005, 0.0, 0.0), 3.0e-4)
    dst = synth.Grid((1, 37, 75), (0.0005, 0.0006, 0.0009), 0.8e-4)
    fields = [synth.random_field(src.n, seed=81)]
    plan = vp.vp_plan(dst, 2, F0, synth.WATER)
    f = torch.empty(dst.n, dtype=torch.complex64, device="cuda")
    plan.source_from_nested([src], [dev(x) for x in fields], f_out=f, quadratic=quadratic)
    ref = oracle_source(2, [src], fields, dst, quadratic)
    assert rel_l2(host(f), ref) <= 1e-6
    plan.close()


def test_nested_source_direct_form_for_a_coarser_target(vp):
    """Target spacing above the source spacing: the per-target gather form."""
    src = synth.Grid((30, 31, 32), (0.0, 0.0, 0.0), 1.0e-4)
    dst = synth.Grid((10, 11, 12), (2.0e-4, 1.0e-4, 3.0e-4), 2.5e-4)
    fields = [synth.random_field(src.n, seed=61), synth.random_field(src.n, seed=62)]
    plan = vp.vp_plan(dst, 3, F0, synth.WATER)
    f = torch.empty(dst.n, dtype=torch.complex64, device="cuda")
    for quadratic in (False, True):
        plan.source_from_nested([src, src], [dev(x) for x in fields], f_out=f, quadratic=quadratic)
        ref = oracle_source(3, [src, src], fields, dst, quadratic)
        assert rel_l2(host(f), ref) <= 1e-6
    plan.close()


def test_staged_nested_source_then_apply(vp):
    """f_out = None stages the source for vp_apply(plan, NULL, u): the potential equals
    the oracle's V[f] of the oracle's source."""
    fields = [synth.random_field(G1.n, seed=71), synth.random_field(G2.n, seed=72)]
    plan = vp.vp_plan(TARGET, 3, F0, synth.WATER)
    vp.vp_kernel_fft(plan)
    u = torch.empty(TARGET.n, dtype=torch.complex64, device="cuda")
    plan.source_from_nested([G1, G2], [dev(x) for x in fields])
    plan.apply(None, u)
    lower = [interp.restrict_trilinear(f, g, TARGET) for f, g in zip(fields, [G1, G2])]
    ref = cascade.harmonic(3, lower, TARGET.h, F0, synth.WATER)
    assert rel_l2(host(u), ref) <= 1e-5
    plan.close()


def test_nested_source_errors(vp):
    plan = vp.vp_plan(TARGET, 3, F0, synth.WATER)
    f = torch.empty(TARGET.n, dtype=torch.complex64, device="cuda")
    a, b = dev(synth.random_field(G1.n, seed=1)), dev(synth.random_field(G2.n, seed=2))
    outside = synth.Grid((10, 10, 10), (0.0015, 0.0015, 0.0015), 1.0e-4)  # too small to hold the target
    with pytest.raises(vp.VpError) as e:
        plan.source_from_nested([G1, outside], [a, b], f_out=f)
    assert e.value.status == vp.VP_ERR_NOT_NESTED
    with pytest.raises(vp.VpError) as e:
        plan.source_from_nested([G1], [a], f_out=f)  # n_lower != n - 1
    assert e.value.status == vp.VP_ERR_ARG
    with pytest.raises(vp.VpError) as e:
        plan.source_from_nested([G1, G2], [a, None], f_out=f)
    assert e.value.status == vp.VP_ERR_ARG
    plan.close()
