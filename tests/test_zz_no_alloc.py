"""The allocation-free entry point vp_apply_static against the plan-based path.

vp_apply_static serves callers that cannot allocate device memory (work recorded
while a stream is captured into a CUDA graph, device memory owned by another
allocator, loops that cannot afford cudaMalloc's device-wide synchronisation).  It
keeps every intermediate in one fixed device array inside libvp.so, so consecutive
calls reuse the same memory; the tests make different calls in a row and check each
against vp_plan + vp_kernel_fft + vp_apply on the same input and against the FP64
oracle's FFT route, including the 64^3 grid that fills the array (M = 128 on every
axis).
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from oracle import physics, potential
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


def test_static_entry_point_matches_oracle_at_the_size_cap(vp):
    """Two calls in a row against the FP64 oracle's zero-padded FFT route: the 64^3 grid
    that fills the fixed array (M = 128 on every axis), then a ragged smaller grid, so
    the second call runs on memory the first one filled."""
    cases = [((64, 64, 64), 2, 1.0e6, 1.25e-4, 11), ((23, 64, 50), 4, 1.1e6, 5.7e-5, 12)]
    for n, harmonic, f0, h, seed in cases:
        g = synth.Grid(n, (0.0, 0.0, 0.0), h)
        f_host = synth.random_field(n, seed).astype(np.complex64)
        ref = potential.apply_fft(f_host.astype(np.complex128), h, physics.wavenumber(harmonic, f0, synth.WATER))
        got = _static_path(vp, g, harmonic, f0, torch.from_numpy(f_host).cuda())
        assert np.all(np.isfinite(got))
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= REL_L2, (n, rel)


def test_static_entry_point_rejects_non_finite_media(vp):
    g = vp.make_grid((8, 8, 8), (0.0, 0.0, 0.0), 1e-4)
    buf = torch.zeros((8, 8, 8), dtype=torch.complex64, device="cuda")
    for field in ("eta", "alpha0", "c0", "beta", "rho0"):
        med = vp.make_medium(synth.WATER)
        setattr(med, field, math.nan if field != "c0" else math.inf)
        st = vp.lib.vp_apply_static(ctypes.byref(g), 2, 1.0e6, ctypes.byref(med), ctypes.c_void_p(buf.data_ptr()),
                                    ctypes.c_void_p(buf.data_ptr()), None)
        assert st == vp.VP_ERR_ARG, field


def test_static_entry_point_rejects_oversized_grids(vp):
    g = vp.make_grid((8, 65, 8), (0.0, 0.0, 0.0), 1e-4)
    med = vp.make_medium(synth.WATER)
    buf = torch.empty(8, dtype=torch.complex64, device="cuda")
    st = vp.lib.vp_apply_static(ctypes.byref(g), 2, 1.0e6, ctypes.byref(med), ctypes.c_void_p(buf.data_ptr()),
                                ctypes.c_void_p(buf.data_ptr()), None)
    assert st == vp.VP_ERR_SIZE
