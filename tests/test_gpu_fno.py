"""FNO surrogate kernels against the FP64 reference: forward values, gradients by
central finite differences of the reference loss, and a training step that lowers the
loss.  Parameters are rounded to BF16 on both sides (the kernels use BF16 weights and
activations with FP32 accumulation), so tolerances are a few 1e-2."""
import numpy as np
import pytest
import torch

from oracle import fno as ofno

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_03009_gb300 import fno as fmod
    return fmod


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).bfloat16().float().double().numpy()


def make(F, cfg, seed):
    m = F.Fno(cfg, seed=seed)
    flat = bf16_round(m.init_params(seed))
    m.set_params(flat)
    return m, flat


def test_forward_matches_fp64_reference(F):
    cfg = F.FnoConfig(n=16, width=8, hidden=16, layers=2, modes=(8, 8, 4))
    m, flat = make(F, cfg, 3)
    rng = np.random.default_rng(4)
    x = 0.5 * rng.standard_normal((16, 16, 16, 2))
    xt = torch.from_numpy(x.reshape(-1, 2).astype(np.float32)).cuda()
    y = torch.empty((16 ** 3, 8), dtype=torch.float32, device="cuda")
    m.forward(xt, y)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.float64).reshape(16, 16, 16, 8)
    ref = ofno.forward(m.unpack(flat), bf16_round(x), cfg.modes)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= 3e-2, rel


def test_gradients_match_finite_differences_of_the_reference(F):
    cfg = F.FnoConfig(n=8, width=4, hidden=8, layers=2, modes=(4, 4, 3))
    m, flat = make(F, cfg, 5)
    rng = np.random.default_rng(6)
    x = bf16_round(0.5 * rng.standard_normal((8, 8, 8, 2)))
    t = rng.standard_normal((8, 8, 8, 8))
    xt = torch.from_numpy(x.reshape(-1, 2).astype(np.float32)).cuda()
    tt = torch.from_numpy(t.reshape(-1, 8).astype(np.float32)).cuda()
    m.grads.zero_()
    m.forward(xt)
    m.loss(tt)
    m.backward(xt, tt)
    torch.cuda.synchronize()
    g_gpu = m.grads.cpu().numpy().astype(np.float64)
    # central differences of the FP64 reference loss, every parameter
    eps = 1e-4
    g_fd = np.zeros_like(flat)
    for i in range(len(flat)):
        fp = flat.copy()
        fp[i] += eps
        fm = flat.copy()
        fm[i] -= eps
        g_fd[i] = (ofno.loss(m.unpack(fp), x, t, cfg.modes) - ofno.loss(m.unpack(fm), x, t, cfg.modes)) / (2 * eps)
    for name, (a, b) in m.slices().items():
        ref = g_fd[a:b]
        got = g_gpu[a:b]
        if np.linalg.norm(ref) < 1e-12:
            assert np.linalg.norm(got) < 1e-6, name
            continue
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel <= 5e-2, (name, rel)


def test_training_steps_reduce_the_loss(F):
    cfg = F.FnoConfig(n=16, width=8, hidden=16, layers=2, modes=(8, 8, 4))
    m, _ = make(F, cfg, 7)
    rng = np.random.default_rng(8)
    xs, ts = [], []
    for _ in range(4):
        x = (0.5 * rng.standard_normal((16 ** 3, 2))).astype(np.float32)
        xs.append(torch.from_numpy(x).cuda())
        ts.append(torch.from_numpy(np.tile(x, (1, 4)) * 0.5).cuda())
    order = np.arange(4)
    first = m.train_epoch(xs, ts, lr=3e-3, batch=2, order=order)
    for _ in range(30):
        last = m.train_epoch(xs, ts, lr=3e-3, batch=2, order=order)
    assert last < 0.5 * first, (first, last)


def test_fused_tiles_and_inference_match_fp64_reference(F):
    """N = 64: the spectral inverse rides inside the pointwise GEMM and vp_fno_infer fuses
    the projection; both against the FP64 reference and against each other."""
    cfg = F.FnoConfig(n=64, width=16, hidden=32, layers=2, modes=(8, 8, 4))
    m, flat = make(F, cfg, 9)
    rng = np.random.default_rng(10)
    x = bf16_round(0.5 * rng.standard_normal((64, 64, 64, 2)))
    xt = torch.from_numpy(x.reshape(-1, 2).astype(np.float32)).cuda()
    y_fwd = torch.empty((64 ** 3, 8), dtype=torch.float32, device="cuda")
    y_inf = torch.empty_like(y_fwd)
    m.forward(xt, y_fwd)
    m.infer(xt, y_inf)
    torch.cuda.synchronize()
    ref = ofno.forward(m.unpack(flat), x, cfg.modes).reshape(-1, 8)
    for got in (y_fwd, y_inf):
        g = got.cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
        assert rel <= 3e-2, rel
    d = (y_fwd - y_inf).norm() / y_fwd.norm()
    assert float(d) <= 1e-2, float(d)
