"""Full cascade with conjugate terms (Eq. 2.5) on the GPU against the oracle: the
source term for every harmonic (written out and fused with the apply), the vector
operations, and the fixed-point iterates."""
import numpy as np
import pytest
import torch

from oracle import cascade as ocascade
from oracle import physics, potential
from paper_2011_03009_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_03009_gb300 import cascade, vp
    return vp, cascade


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_vector_operations(mods):
    vp, _ = mods
    n = (17, 9, 13)
    x, y = synth.random_field(n, 1), synth.random_field(n, 2)
    xt, yt = dev(x), dev(y)
    out = torch.empty_like(xt)
    a, b = 0.3 - 1.1j, -2.0 + 0.5j
    vp.vp_vec_axpby(a, xt, b, yt, out)
    assert rel(host(out), a * x.astype(np.complex64) + b * y.astype(np.complex64)) <= 1e-6
    vp.vp_vec_mul(xt, yt, out)
    assert rel(host(out), x.astype(np.complex64) * y.astype(np.complex64)) <= 1e-6
    x32, y32 = x.astype(np.complex64).astype(np.complex128), y.astype(np.complex64).astype(np.complex128)
    d = vp.vp_vec_dot(xt, yt)
    assert abs(d - np.vdot(x32, y32)) <= 1e-12 * abs(np.vdot(x32, y32)) * 1e3
    d2 = vp.vp_vec_dot(xt, yt, conj_x=False)
    assert abs(d2 - np.sum(x32 * y32)) <= 1e-9 * np.linalg.norm(x32) * np.linalg.norm(y32)
    # in place: out aliases x
    vp.vp_vec_axpby(2.0, xt, 0.0, None, xt)
    assert rel(host(xt), 2 * x32) <= 1e-7


@pytest.mark.parametrize("nh", [2, 4, 8])
def test_full_source_matches_oracle(mods, nh):
    vp, _ = mods
    g = synth.Grid((20, 18, 22), (0.0, 0.0, 0.0), 1.25e-4)
    fields = [synth.random_field(g.n, 10 + m, scale=1e5 / m) for m in range(1, nh + 1)]
    tf = [dev(f) for f in fields]
    f32 = [f.astype(np.complex64).astype(np.complex128) for f in fields]
    for n in range(1, nh + 1):
        plan = vp.vp_plan(g, n, 1.0e6, synth.WATER)
        plan.kernel_fft()
        out = torch.empty(g.n, dtype=torch.complex64, device="cuda")
        lower = list(tf)
        plan.source_assemble(lower, f_out=out, conj=True)
        ref = ocascade.source_term_full(n, f32, 1.0e6, synth.WATER)
        assert rel(host(out), ref) <= 1e-6, n
        # staged form feeding the apply
        u = torch.empty_like(out)
        plan.source_assemble(lower, conj=True)
        plan.apply(None, u)
        uref = potential.apply_fft(ref, g.h, physics.wavenumber(n, 1.0e6, synth.WATER))
        assert rel(host(u), uref) <= 1e-5, n
        plan.close()


def test_full_cascade_iterates_match_oracle(mods):
    vp, cascade = mods
    g = synth.Grid((24, 20, 16), (0.0, 0.0, 0.0), 2.0e-4)
    p_inc = synth.random_field(g.n, 3, scale=4.0e5)
    fc = cascade.FullCascade(g, 3, 1.0e6, synth.WATER)
    pt = dev(p_inc)
    fc.weakly_nonlinear(pt)
    hist = [fc.sweep(pt) for _ in range(3)]
    ref = ocascade.full_cascade(p_inc.astype(np.complex64).astype(np.complex128), 3, g.h, 1.0e6, synth.WATER,
                                iters=3)
    for n in range(3):
        assert rel(host(fc.p[n]), ref[n]) <= 1e-5, n
    assert hist[-1] < hist[0]
    fc.close()
