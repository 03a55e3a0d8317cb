"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: relative L2 error <= 1e-5 over every output voxel for the FP32 path
(the single-precision target of the method's volume potential), tighter where the
arithmetic allows.  Sizes span several 16-line tiles, ragged tails and odd axes.
"""
import numpy as np
import pytest
import torch

from oracle import cascade, interp, physics, potential, rayleigh
from paper_2011_03009_gb300 import synth

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5


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


def grid(n, h=1.25e-4, origin=(0.0, 0.0, 0.0)):
    return synth.Grid(tuple(n), tuple(origin), h)


def gpu_apply(vp, g, f, harmonic, f0=1.0e6, m=None, radix=None):
    plan = vp.vp_plan(g, harmonic, f0, synth.WATER, m=m, radix=radix)
    vp.vp_kernel_fft(plan)
    u = torch.empty(g.n, dtype=torch.complex64, device="cuda")
    vp.vp_apply(plan, dev(f), u)
    out = host(u)
    plan.close()
    return out


@pytest.mark.parametrize("n", [(8, 8, 8), (12, 9, 7), (16, 16, 16), (33, 20, 17), (1, 5, 3), (40, 48, 36),
                               (2, 1, 1), (1, 1, 1)])
def test_apply_matches_oracle(vp, n):
    g = grid(n)
    k = physics.wavenumber(2, 1.0e6, synth.WATER)
    f = synth.random_field(n, seed=sum(n))
    ref = potential.apply_fft(f, g.h, k)
    got = gpu_apply(vp, g, f, 2)
    assert rel_l2(got, ref) <= REL_L2


@pytest.mark.parametrize("m,radix", [
    ((32, 32, 36), ((2, 16), (4, 8), (4, 3, 3))),
    ((40, 30, 45), ((8, 5), (5, 3, 2), (5, 3, 3))),
    ((48, 45, 50), ((16, 3), (5, 3, 3), (5, 5, 2))),
    ((64, 60, 80), ((4, 4, 4), (3, 4, 5), (16, 5))),
])
def test_every_radix_and_embedding_size(vp, m, radix):
    n = (16, 15, 17)
    g = grid(n, h=9e-5)
    k = physics.wavenumber(3, 1.1e6, synth.WATER)
    f = synth.random_field(n, seed=5)
    ref = potential.apply_fft(f, g.h, k)
    got = gpu_apply(vp, g, f, 3, f0=1.1e6, m=m, radix=radix)
    assert rel_l2(got, ref) <= REL_L2


def test_apply_matches_bruteforce_definition(vp):
    n = (10, 13, 9)
    g = grid(n, h=6e-5)
    k = physics.wavenumber(4, 1.1e6, synth.WATER)
    f = synth.random_field(n, seed=9)
    ref = potential.apply_bruteforce(f, g.h, k)
    got = gpu_apply(vp, g, f, 4, f0=1.1e6)
    assert rel_l2(got, ref) <= REL_L2


def test_kernel_spectrum_octant(vp):
    n = (12, 10, 9)
    g = grid(n)
    plan = vp.vp_plan(g, 2, 1.0e6, synth.WATER)
    vp.vp_kernel_fft(plan)
    inf = plan.info()
    m = tuple(inf.m)
    o = tuple(v // 2 + 1 for v in m)
    buf = torch.empty(o, dtype=torch.complex64, device="cuda")
    plan.kernel_spectrum_get(buf)
    got = host(buf)
    plan.close()
    full = potential.kernel_spectrum(n, g.h, physics.wavenumber(2, 1.0e6, synth.WATER), m)
    ref = full[: o[0], : o[1], : o[2]]
    assert rel_l2(got, ref) <= 1e-6
    # even spectrum: K^(q) = K^(M - q)
    assert np.allclose(full[1:, :, :], full[:0:-1, :, :], rtol=1e-10, atol=1e-10 * np.abs(full).max())


def test_plan_info_constants(vp):
    g = grid((8, 8, 8))
    plan = vp.vp_plan(g, 3, 1.1e6, synth.WATER)
    inf = plan.info()
    k = physics.wavenumber(3, 1.1e6, synth.WATER)
    assert abs(complex(inf.k_re, inf.k_im) - k) <= 1e-12 * abs(k)
    assert abs(inf.c_n - physics.source_coefficient(3, 1.1e6, synth.WATER)) <= 1e-12 * abs(inf.c_n)
    from oracle import greens
    sc = greens.self_cell(k, g.h)
    assert abs(complex(inf.self_re, inf.self_im) - sc) <= 1e-12 * abs(sc)
    assert tuple(inf.m) == (16, 16, 16)
    plan.close()


@pytest.mark.parametrize("harmonic", [2, 3, 4, 5])
def test_source_assembly_matches_oracle(vp, harmonic):
    n = (9, 17, 20)
    g = grid(n)
    lower = [synth.random_field(n, seed=100 + m) for m in range(1, harmonic)]
    plan = vp.vp_plan(g, harmonic, 1.1e6, synth.WATER)
    f = torch.empty(n, dtype=torch.complex64, device="cuda")
    plan.source_assemble([dev(x) for x in lower], f_out=f)
    got = host(f)
    ref = cascade.source_term(harmonic, lower, 1.1e6, synth.WATER)
    assert rel_l2(got, ref) <= 1e-6
    # fused path: assembly straight into the first FFT sweep, then the apply
    vp.vp_kernel_fft(plan)
    u = torch.empty(n, dtype=torch.complex64, device="cuda")
    plan.source_assemble([dev(x) for x in lower])
    plan.apply(None, u)
    got_u = host(u)
    plan.close()
    ref_u = cascade.harmonic(harmonic, lower, g.h, 1.1e6, synth.WATER)
    assert rel_l2(got_u, ref_u) <= REL_L2


def test_call_order_errors(vp):
    g = grid((8, 8, 8))
    plan = vp.vp_plan(g, 2, 1.0e6, synth.WATER)
    u = torch.empty(g.n, dtype=torch.complex64, device="cuda")
    with pytest.raises(vp.VpError) as e:
        plan.apply(dev(np.zeros(g.n)), u)
    assert e.value.status == vp.VP_ERR_STATE
    vp.vp_kernel_fft(plan)
    with pytest.raises(vp.VpError) as e:
        plan.apply(None, u)
    assert e.value.status == vp.VP_ERR_STATE
    with pytest.raises(vp.VpError) as e:
        plan.source_assemble([dev(np.zeros(g.n)), dev(np.zeros(g.n))])
    assert e.value.status == vp.VP_ERR_ARG
    plan.close()


def test_restriction_matches_oracle(vp):
    src = synth.Grid((21, 19, 23), (0.01, -0.003, -0.0032), 3.1e-4)
    dst = synth.centred_grid((30, 27, 33), 1.7e-4, (0.0131, -0.0001, 0.0002))
    f = synth.random_field(src.n, seed=3)
    out = torch.empty(dst.n, dtype=torch.complex64, device="cuda")
    vp.vp_restrict_to_nested_box(src, dev(f), dst, out)
    got = host(out)
    ref = interp.restrict_trilinear(f, src, dst)
    assert rel_l2(got, ref) <= 1e-6
    # identical grids: identity
    same = torch.empty(src.n, dtype=torch.complex64, device="cuda")
    vp.vp_restrict_to_nested_box(src, dev(f), src, same)
    assert rel_l2(host(same), f.astype(np.complex64).astype(np.complex128)) <= 1e-7


@pytest.mark.parametrize("quadratic", [False, True])
@pytest.mark.parametrize("case", ["several_tiles", "coarser_target", "flat_axis", "two_point_axis"])
def test_restriction_tiles_and_direct_form(vp, case, quadratic):
    """Shared-memory tiles (target spacing <= ~source spacing) over several ragged
    8 x 64 blocks, the direct form for a coarser target, and a one-voxel source axis."""
    if case == "several_tiles":
        src = synth.Grid((12, 40, 90), (0.0, 0.0, 0.0), 2.0e-4)
        dst = synth.Grid((9, 53, 130), (1.0e-4, 3.0e-4, 1.1e-4), 1.3e-4)
    elif case == "coarser_target":
        src = synth.Grid((30, 31, 32), (0.0, 0.0, 0.0), 1.0e-4)
        dst = synth.Grid((10, 11, 12), (2.0e-4, 1.0e-4, 3.0e-4), 2.5e-4)
    elif case == "flat_axis":
        src = synth.Grid((1, 20, 70), (0.001, 0.0, 0.0), 2.0e-4)
        dst = synth.Grid((1, 25, 90), (0.001, 1.0e-4, 2.0e-4), 1.4e-4)
    else:
        src = synth.Grid((2, 20, 70), (0.001, 0.0, 0.0), 2.0e-4)
        dst = synth.Grid((2, 25, 90), (0.00105, 1.0e-4, 2.0e-4), 1.4e-4)
    f = synth.random_field(src.n, seed=7)
    out = torch.empty(dst.n, dtype=torch.complex64, device="cuda")
    vp.vp_restrict_to_nested_box(src, dev(f), dst, out, quadratic=quadratic)
    ref = (interp.restrict_quadratic if quadratic else interp.restrict_trilinear)(f, src, dst)
    assert rel_l2(host(out), ref) <= 1e-6


def test_quadratic_restriction_matches_plain_positions_up_to_ties(vp):
    """Against the oracle's plain FP64 target positions: every voxel equals the
    quadratic interpolant for one valid stencil choice per axis (two equally near
    stencils at a half-integer position, one elsewhere).  Spacing ratio 2/3 with even
    voxel counts, as between the nested 192^3 and 256^3 grids: every third target sits
    on a half-integer on each axis."""
    c = (0.06, 0.0, 0.0)
    src = synth.centred_grid((24, 24, 24), 3.0e-4, c)
    dst = synth.centred_grid((28, 28, 28), 2.0e-4, c)
    ties = interp.tie_axes(src, dst)
    assert all(t.sum() >= 9 for t in ties)
    f = synth.random_field(src.n, seed=21)
    out = torch.empty(dst.n, dtype=torch.complex64, device="cuda")
    vp.vp_restrict_to_nested_box(src, dev(f), dst, out, quadratic=True)
    got = host(out)
    err = np.full(dst.n, np.inf)
    for tx in ("down", "up"):
        for ty in ("down", "up"):
            for tz in ("down", "up"):
                ref = interp.restrict_quadratic(f, src, dst, positions="float", tie=(tx, ty, tz))
                err = np.minimum(err, np.abs(got - ref))
    assert np.max(err) <= 2e-6 * np.max(np.abs(f))


def test_quadratic_restriction_exact_on_triquadratic_field(vp):
    src = synth.Grid((21, 19, 23), (0.01, -0.003, -0.0032), 3.1e-4)
    dst = synth.centred_grid((30, 27, 33), 1.7e-4, (0.0131, -0.0001, 0.0002))
    X, Y, Z = np.meshgrid(src.axis(0), src.axis(1), src.axis(2), indexing="ij")
    Xd, Yd, Zd = np.meshgrid(dst.axis(0), dst.axis(1), dst.axis(2), indexing="ij")
    q = lambda x, y, z: (1 + 30 * (x - 0.013) + 900 * (x - 0.013) ** 2) * (2 - 40 * y + 1e3 * y * y) * (1j + 50 * z)
    out = torch.empty(dst.n, dtype=torch.complex64, device="cuda")
    vp.vp_restrict_to_nested_box(src, dev(q(X, Y, Z)), dst, out, quadratic=True)
    assert rel_l2(host(out), q(Xd, Yd, Zd)) <= 1e-6


def test_restriction_not_nested(vp):
    src = synth.Grid((5, 5, 5), (0.0, 0.0, 0.0), 1e-3)
    dst = synth.Grid((3, 3, 3), (0.0, 0.0, 0.0031), 1e-3)
    out = torch.empty(dst.n, dtype=torch.complex64, device="cuda")
    with pytest.raises(vp.VpError) as e:
        vp.vp_restrict_to_nested_box(src, dev(np.ones(src.n)), dst, out)
    assert e.value.status == vp.VP_ERR_NOT_NESTED
    vp.vp_restrict_to_nested_box(src, dev(np.ones(src.n)), dst, out, zero_outside=True)
    got = host(out)
    assert np.all(got[:, :, 1:] == 0) and np.allclose(got[:, :, 0], 1.0)


def test_incident_field_matches_oracle(vp):
    bowl = synth.Bowl(l=0.02, R=0.01, f0=1.0e6, p0=0.5e6)
    g = synth.focus_grid(bowl, (14, 11, 9), 2)
    pts = synth.sample_bowl_points(bowl, 700, seed=4)
    out = torch.empty(g.n, dtype=torch.complex64, device="cuda")
    vp.vp_incident_field(g, torch.from_numpy(pts).cuda(), bowl, synth.WATER, out)
    got = host(out)
    ref = rayleigh.incident_field(g, pts, bowl, synth.WATER)
    assert rel_l2(got, ref) <= 2e-6


def test_incident_field_next_to_the_bowl(vp):
    """A grid straddling the cap: points within a few voxels of the tile take the direct
    FP64 distance, the others the tile-centred expansion; both against the oracle."""
    bowl = synth.Bowl(l=0.02, R=0.01, f0=1.0e6, p0=0.5e6)
    g = synth.Grid((12, 20, 20), (0.0005, -0.005, -0.005), 0.5e-3)
    pts = synth.sample_bowl_points(bowl, 600, seed=5)
    out = torch.empty(g.n, dtype=torch.complex64, device="cuda")
    vp.vp_incident_field(g, torch.from_numpy(pts).cuda(), bowl, synth.WATER, out)
    got = host(out)
    ref = rayleigh.incident_field(g, pts, bowl, synth.WATER)
    assert rel_l2(got, ref) <= 2e-6


def test_small_workload_end_to_end(vp):
    """32^3 second harmonic of the 1 cm / 2 cm / 1 MHz bowl, against oracle and brute force."""
    w = synth.workload_small_p2()
    g = w.steps[0].grid
    pts = synth.sample_bowl_points(w.bowl, w.n_points, w.seed)
    p1 = torch.empty(g.n, dtype=torch.complex64, device="cuda")
    vp.vp_incident_field(g, torch.from_numpy(pts).cuda(), w.bowl, w.medium, p1)
    plan = vp.vp_plan(g, 2, w.bowl.f0, w.medium)
    vp.vp_kernel_fft(plan)
    u = torch.empty(g.n, dtype=torch.complex64, device="cuda")
    vp.vp_source_assemble(plan, [p1])
    vp.vp_apply(plan, None, u)
    got = host(u)
    plan.close()
    p1_ref = rayleigh.incident_field(g, pts, w.bowl, w.medium)
    assert rel_l2(host(p1), p1_ref) <= 2e-6
    ref = cascade.harmonic(2, [p1_ref], g.h, w.bowl.f0, w.medium)
    assert rel_l2(got, ref) <= REL_L2
    f = cascade.source_term(2, [p1_ref], w.bowl.f0, w.medium)
    k2 = physics.wavenumber(2, w.bowl.f0, w.medium)
    rng = np.random.default_rng(0)
    tg = rng.integers(0, 32, size=(12, 3))
    bf = potential.apply_bruteforce(f, g.h, k2, targets=tg)
    sel = got[tg[:, 0], tg[:, 1], tg[:, 2]]
    assert np.linalg.norm(sel - bf) <= REL_L2 * np.linalg.norm(bf) * 3


FAST_SIZES = [32, 64, 128, 192, 256, 320, 384, 512, 640, 768, 864, 1024, 1200, 1280]


@pytest.mark.parametrize("L", FAST_SIZES)
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_two_level_engine_every_size_and_axis(vp, L, axis):
    """Each compiled two-level length on each sweep type (x column, y column, z line),
    with a ragged N = L/2 - 1 along that axis and radix-pass axes elsewhere."""
    n = [5, 6, 7]
    n[axis] = L // 2 - 1
    m = [0, 0, 0]
    m[axis] = L
    g = grid(tuple(n), h=5e-5)
    k = physics.wavenumber(2, 1.1e6, synth.WATER)
    f = synth.random_field(tuple(n), seed=L + axis)
    plan = vp.vp_plan(g, 2, 1.1e6, synth.WATER, m=m)
    assert plan.info().engine[axis] == 1
    vp.vp_kernel_fft(plan)
    u = torch.empty(tuple(n), dtype=torch.complex64, device="cuda")
    vp.vp_apply(plan, dev(f), u)
    got = host(u)
    plan.close()
    ref = potential.apply_fft(f, g.h, k)
    assert rel_l2(got, ref) <= REL_L2


@pytest.mark.parametrize("harmonic", [2, 4, 5])
def test_fused_source_on_two_level_engine(vp, harmonic):
    n = (60, 31, 64)  # M = 128 (two-level), 64 (two-level), 128 (two-level)
    g = grid(n, h=6e-5)
    lower = [synth.random_field(n, seed=200 + m) for m in range(1, harmonic)]
    plan = vp.vp_plan(g, harmonic, 1.1e6, synth.WATER)
    assert list(plan.info().engine) == [1, 1, 1]
    vp.vp_kernel_fft(plan)
    u = torch.empty(n, dtype=torch.complex64, device="cuda")
    plan.source_assemble([dev(x) for x in lower])
    plan.apply(None, u)
    got = host(u)
    plan.close()
    ref = cascade.harmonic(harmonic, lower, g.h, 1.1e6, synth.WATER)
    assert rel_l2(got, ref) <= REL_L2


@pytest.mark.parametrize("n", [(20, 24, 18), (13, 36, 320), (60, 32, 64), (9, 30, 16)])
def test_grouped_and_plain_intermediate_layouts_match_oracle(vp, n):
    """The x sweep writes its output with x rows grouped by 4 y-planes where N_y is a
    multiple of 4 and x, y run on the two-level engine (layout 0), or plain (layout 1);
    with a field and with the fused source of Eq. 2.6 both match the oracle and each
    other bit for bit (the same arithmetic in another order of memory).  N_y = 30 stays
    plain under layout 0."""
    g = grid(n, h=6e-5)
    harmonic = 3
    lower = [synth.random_field(n, seed=300 + m) for m in range(1, harmonic)]
    f = synth.random_field(n, seed=301)
    k = physics.wavenumber(harmonic, 1.1e6, synth.WATER)
    outs = {}
    for layout in (0, 1):
        plan = vp.vp_plan(g, harmonic, 1.1e6, synth.WATER, layout=layout)
        gy = plan.info().group_y
        two_level = list(plan.info().engine)[:2] == [1, 1]
        assert gy == 1 or (layout == 0 and two_level and gy > 1 and n[1] % gy == 0)
        if layout == 0 and two_level and n[1] % 8 == 0:
            assert gy > 1
        vp.vp_kernel_fft(plan)
        u = torch.empty(n, dtype=torch.complex64, device="cuda")
        vp.vp_apply(plan, dev(f), u)
        uf = host(u)
        plan.source_assemble([dev(x) for x in lower])
        plan.apply(None, u)
        outs[layout] = (uf, host(u))
        plan.close()
    assert rel_l2(outs[0][0], potential.apply_fft(f, g.h, k)) <= REL_L2
    assert rel_l2(outs[0][1], cascade.harmonic(harmonic, lower, g.h, 1.1e6, synth.WATER)) <= REL_L2
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_two_level_kernel_spectrum_octant(vp):
    n = (64, 96, 40)  # M = 128, 192, 80 -> 128, 192 two-level; 80 radix passes
    g = grid(n, h=8e-5)
    plan = vp.vp_plan(g, 3, 1.1e6, synth.WATER)
    inf = plan.info()
    m = tuple(inf.m)
    o = tuple(v // 2 + 1 for v in m)
    vp.vp_kernel_fft(plan)
    buf = torch.empty(o, dtype=torch.complex64, device="cuda")
    plan.kernel_spectrum_get(buf)
    got = host(buf)
    plan.close()
    full = potential.kernel_spectrum(n, g.h, physics.wavenumber(3, 1.1e6, synth.WATER), m)
    assert rel_l2(got, full[: o[0], : o[1], : o[2]]) <= 1e-6


def test_retargeted_plan_matches_a_fresh_plan_and_the_oracle(vp):
    """vp_plan_retarget: same N, new spacing/origin/harmonic/f0; K^ rebuilt, result equal
    to a plan created for the new problem, and to the oracle."""
    n = (24, 20, 18)
    g1, g2 = grid(n, h=1.25e-4), grid(n, h=0.9e-4, origin=(0.01, 0.0, 0.002))
    f = synth.random_field(n, seed=11)
    plan = vp.vp_plan(g1, 2, 1.0e6, synth.WATER)
    plan.kernel_fft()
    u = torch.empty(n, dtype=torch.complex64, device="cuda")
    plan.apply(dev(f), u)
    plan.retarget(g2, 3, 1.3e6, synth.WATER)
    assert plan.info().khat_ready == 0
    with pytest.raises(vp.VpError):
        plan.apply(dev(f), u)          # stale spectrum
    plan.kernel_fft()
    plan.apply(dev(f), u)
    got = host(u)
    fresh = gpu_apply(vp, g2, f, 3, f0=1.3e6)
    assert np.array_equal(got, fresh)
    k = physics.wavenumber(3, 1.3e6, synth.WATER)
    assert rel_l2(got, potential.apply_fft(f, g2.h, k)) <= REL_L2
    with pytest.raises(vp.VpError):
        plan.retarget(grid((24, 20, 17)), 3, 1.3e6, synth.WATER)
    plan.close()


@pytest.mark.parametrize("nz", [256, 320, 384, 432, 512, 640])
def test_every_z_sweep_form_matches_oracle(vp, nz):
    """Each form of the pipelined z sweep (16-, 8- and 4-line tiles, the pair-split
    8-line form, the 4-line form with its factors swapped) at the z embeddings of the runs (M_z = 512 ... 1280), with ragged x and
    y axes; a form not compiled for M_z falls back to the automatic choice."""
    n = (7, 5, nz)
    g = grid(n)
    k = physics.wavenumber(3, 1.0e6, synth.WATER)
    f = synth.random_field(n, seed=nz)
    ref = potential.apply_fft(f, g.h, k)
    for form in (vp.VP_ZFORM_TILE16, vp.VP_ZFORM_TILE8, vp.VP_ZFORM_TILE4, vp.VP_ZFORM_PAIR8, vp.VP_ZFORM_TILE4T):
        plan = vp.vp_plan(g, 3, 1.0e6, synth.WATER, zform=form)
        assert plan.info().m[2] == 2 * nz
        vp.vp_kernel_fft(plan)
        u = torch.empty(n, dtype=torch.complex64, device="cuda")
        vp.vp_apply(plan, dev(f), u)
        assert rel_l2(host(u), ref) <= REL_L2, form
        plan.close()


@pytest.mark.parametrize("nz", [256, 320, 432, 640])
def test_bulk_and_element_staging_match_oracle_and_each_other(vp, nz):
    """The 4-line z-sweep forms stage their lines and octant lines by bulk asynchronous
    copies (staging 0) or by per-element cp.async (staging 1): both match the oracle and
    give the same floating-point result, and the plan's device status stays clear."""
    n = (9, 7, nz)
    g = grid(n)
    k = physics.wavenumber(2, 1.1e6, synth.WATER)
    f = synth.random_field(n, seed=nz + 1)
    ref = potential.apply_fft(f, g.h, k)
    form = vp.VP_ZFORM_TILE4T if nz == 640 else vp.VP_ZFORM_TILE4
    outs = []
    for staging in (0, 1):
        plan = vp.vp_plan(g, 2, 1.1e6, synth.WATER, zform=form, staging=staging)
        assert plan.info().staging == staging
        vp.vp_kernel_fft(plan)
        u = torch.empty(n, dtype=torch.complex64, device="cuda")
        vp.vp_apply(plan, dev(f), u)
        assert plan.check() == vp.VP_OK
        outs.append(host(u))
        assert rel_l2(outs[-1], ref) <= REL_L2, staging
        plan.close()
    assert np.array_equal(outs[0], outs[1])


def test_odd_line_length_falls_back_to_element_staging(vp):
    """N_z odd: a line is not a whole number of 16-byte units, so the 4-line form keeps
    cp.async staging; the result matches the oracle and no refusal is recorded."""
    n = (6, 5, 255)
    g = grid(n)
    k = physics.wavenumber(2, 1.0e6, synth.WATER)
    f = synth.random_field(n, seed=255)
    plan = vp.vp_plan(g, 2, 1.0e6, synth.WATER, zform=vp.VP_ZFORM_TILE4)
    assert plan.info().m[2] == 512
    vp.vp_kernel_fft(plan)
    u = torch.empty(n, dtype=torch.complex64, device="cuda")
    vp.vp_apply(plan, dev(f), u)
    assert plan.check() == vp.VP_OK
    assert rel_l2(host(u), potential.apply_fft(f, g.h, k)) <= REL_L2
    plan.close()


def test_expired_bulk_wait_is_reported_and_the_context_stays_usable(vp):
    """Test hook: the bulk-staged z sweep issues none of its first copies, so each CTA's
    bounded wait (about one second) expires; the CTAs record it and return, vp_plan_check
    reports VP_ERR_TIMEOUT once and clears it, and a normal plan then runs and matches the
    oracle on the same context."""
    n = (8, 6, 320)
    g = grid(n)
    k = physics.wavenumber(2, 1.0e6, synth.WATER)
    f = synth.random_field(n, seed=5)
    stalled = vp.vp_plan(g, 2, 1.0e6, synth.WATER, zform=vp.VP_ZFORM_TILE4, test_expire_waits=True)
    vp.vp_kernel_fft(stalled)
    u = torch.empty(n, dtype=torch.complex64, device="cuda")
    vp.vp_apply(stalled, dev(f), u)
    assert stalled.check() == vp.VP_ERR_TIMEOUT
    assert stalled.check() == vp.VP_OK
    stalled.close()
    plan = vp.vp_plan(g, 2, 1.0e6, synth.WATER, zform=vp.VP_ZFORM_TILE4)
    vp.vp_kernel_fft(plan)
    vp.vp_apply(plan, dev(f), u)
    assert plan.check() == vp.VP_OK
    assert rel_l2(host(u), potential.apply_fft(f, g.h, k)) <= REL_L2
    plan.close()


def test_autotuned_z_form_matches_oracle(vp):
    """The autotuner times the z-sweep forms for M_z >= 512 and keeps one; the plan it
    returns reports that form and matches the oracle."""
    n = (9, 6, 320)
    g = grid(n)
    k = physics.wavenumber(2, 1.0e6, synth.WATER)
    f = synth.random_field(n, seed=77)
    plan = vp.vp_plan(g, 2, 1.0e6, synth.WATER, autotune=True)
    inf = plan.info()
    assert inf.m[2] == 640 and vp.VP_ZFORM_TILE16 <= inf.zform <= vp.VP_ZFORM_TILE4T
    vp.vp_kernel_fft(plan)
    u = torch.empty(n, dtype=torch.complex64, device="cuda")
    vp.vp_apply(plan, dev(f), u)
    assert rel_l2(host(u), potential.apply_fft(f, g.h, k)) <= REL_L2
    plan.close()
