"""The surrogate's runtime judge and fallback (JudgedSurrogate): the plain path computes
p2 for every sample and decides whether the network's harmonics are kept.

- Rejected samples return exactly the plain cascade's fields (same kernels, same order).
- Accepted samples return the exact p2 and the network's p3..p5, decoded from its
  normalised outputs.
- The judge's error is the network's relative L2 error on p2 against the plain path.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_03009_gb300 import fno as fmod
    return fmod


def _model(F, n=64):
    cfg = F.FnoConfig(n=n, width=16, hidden=32, layers=2, modes=(8, 8, 4))
    m = F.Fno(cfg, seed=3)
    m.kappa = torch.tensor([2.0e-7, 5.0e-14, 1.0e-20, 3.0e-27], dtype=torch.float64)
    return m


def test_rejected_sample_equals_the_plain_cascade(F):
    model = _model(F)
    judged = F.JudgedSurrogate(model, threshold=1e-2, n_points=256)
    bowl = F.draw_bowls(1, 11)[0]
    out, info = judged.run(bowl, 5)
    assert info["fallback"] and info["judge_rel_l2"] > 1e-2
    ref = F.PlainCascade(64, 256)
    ref.incident(bowl, 5)
    box = ref.harmonics(bowl)
    torch.cuda.synchronize()
    for h in range(2, 6):
        assert torch.equal(out[h], box[h]), h


def test_accepted_sample_keeps_the_network_output(F):
    model = _model(F)
    judged = F.JudgedSurrogate(model, threshold=float("inf"), n_points=256)
    bowl = F.draw_bowls(1, 12)[0]
    out, info = judged.run(bowl, 6)
    assert not info["fallback"]
    c = judged.casc
    s = float(c.p1_box.abs().max().item())
    y = judged.y.double()
    for h in range(3, 6):
        k = 2 * (h - 2)
        want = (torch.complex(y[:, k], y[:, k + 1]).reshape(c.p1_box.shape) * (s ** h * float(model.kappa[h - 2])))
        got = out[h].to(torch.complex128)
        assert float((got - want).abs().max() / want.abs().max()) <= 1e-6, h
    # the judge's p2 is the plain path's
    ref = F.PlainCascade(64, 256)
    ref.incident(bowl, 6)
    box = ref.harmonics(bowl)
    assert torch.equal(out[2], box[2])


def test_judge_error_is_the_networks_p2_error(F):
    model = _model(F)
    judged = F.JudgedSurrogate(model, threshold=1e-2, n_points=256)
    bowl = F.draw_bowls(1, 13)[0]
    _, info = judged.run(bowl, 7)
    ref = F.PlainCascade(64, 256)
    p1, harm = ref.run(bowl, 7)
    x, t, _ = F.encode(p1, harm, model.kappa)
    e2 = float(model.rel_l2(x, t)[0])
    # inference and the training forward pass round their BF16 activations apart
    assert abs(info["judge_rel_l2"] - e2) <= 1e-2 * e2, (info["judge_rel_l2"], e2)
