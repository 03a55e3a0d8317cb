"""The allocation-free entry point vp_apply_static against the plan-based path.

vp_apply_static serves callers that cannot allocate device memory (work recorded
while a stream is captured into a CUDA graph, device memory owned by another
allocator, loops that cannot afford cudaMalloc's device-wide synchronisation).  It
keeps every intermediate in one fixed device array inside libvp.so, so consecutive
calls reuse the same memory; the test makes two different calls in a row and checks
each against vp_plan + vp_kernel_fft + vp_apply on the same input.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2011_03009_gb300 import synth

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5


@pytest.fixture(scope="module")
def vp(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_03009_gb300 import vp as vpmod
    return vpmod


def _plan_path(vp, g, harmonic, f0, f):
    plan = vp.vp_plan(g, harmonic, f0, synth.WATER)
    vp.vp_kernel_fft(plan)
    u = torch.empty(g.n, dtype=torch.complex64, device="cuda")
    vp.vp_apply(plan, f, u)
    torch.cuda.synchronize()
    out = u.cpu().numpy().astype(np.complex128)
    plan.close()
    return out


def _static_path(vp, g, harmonic, f0, f):
    u = torch.full(g.n, float("nan"), dtype=torch.complex64, device="cuda")
    grid = vp.grid_of(g)
    med = vp.make_medium(synth.WATER)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = vp.lib.vp_apply_static(ctypes.byref(grid), harmonic, f0, ctypes.byref(med),
                                ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()), stream)
    assert st == vp.VP_OK, vp.status_string(st)
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.complex128)


def test_static_entry_point_matches_plan_path_on_consecutive_calls(vp):
    cases = [((40, 33, 64), 2, 1.0e6, 1.25e-4, 7), ((17, 64, 9), 3, 1.1e6, 7.6e-5, 8)]
    for n, harmonic, f0, h, seed in cases:
        g = synth.Grid(n, (0.0, 0.0, 0.0), h)
        f = torch.from_numpy(synth.random_field(n, seed).astype(np.complex64)).cuda()
        ref = _plan_path(vp, g, harmonic, f0, f)
        got = _static_path(vp, g, harmonic, f0, f)
        assert np.all(np.isfinite(got))
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= REL_L2, (n, rel)


def test_static_entry_point_rejects_oversized_grids(vp):
    g = vp.make_grid((8, 65, 8), (0.0, 0.0, 0.0), 1e-4)
    med = vp.make_medium(synth.WATER)
    buf = torch.empty(8, dtype=torch.complex64, device="cuda")
    st = vp.lib.vp_apply_static(ctypes.byref(g), 2, 1.0e6, ctypes.byref(med), ctypes.c_void_p(buf.data_ptr()),
                                ctypes.c_void_p(buf.data_ptr()), None)
    assert st == vp.VP_ERR_SIZE
