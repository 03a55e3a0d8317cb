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
