"""What the trained surrogate gains over the method without it, on the GPU.

- Training gains accuracy: a small surrogate trained briefly on fields from the plain
  path (the reference) has a held-out relative L2 error, per harmonic, well below that of the
  same network before training.
- Inference cost: at the 128^3 focal box, one evaluation of the surrogate in the
  workload's architecture (4 layers, width 48, 32 x 32 x 16 modes) is timed against the
  plain cascade it would replace (kernel spectra, restrictions, sources and potentials
  of harmonics 2..5), both from p1 on the device; timing does not depend on the weights'
  values.  Both are reported; which one is faster is a measured outcome, not assumed.
- Every held-out sample is checked against the plain path; those above the 1e-2 threshold are
  the ones that fall back (counted, not hidden).
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


def _ms(fn, reps=5):
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def test_training_gains_accuracy(F):
    n = 64
    cfg = F.FnoConfig(n=n, width=32, hidden=64, layers=3, modes=(16, 16, 8))
    xs, ts, _, kappa, _ = F.make_dataset(32, 5, n, 256)
    xv, tv, _, _, _ = F.make_dataset(6, 6, n, 256, kappa)
    model = F.Fno(cfg, seed=0)
    model.kappa = kappa
    before = np.array([model.rel_l2(x, t) for x, t in zip(xv, tv)])
    rng = np.random.default_rng(0)
    for ep in range(40):
        model.train_epoch(xs, ts, 2e-3 * (0.5 + 0.5 * np.cos(np.pi * ep / 40)), 4, rng.permutation(len(xs)))
    after = np.array([model.rel_l2(x, t) for x, t in zip(xv, tv)])
    # every harmonic improves, and the mean error at least halves
    assert np.all(after.mean(axis=0) < 0.75 * before.mean(axis=0)), (before.mean(0), after.mean(0))
    assert after.mean() < 0.5 * before.mean(), (before.mean(), after.mean())
    fallback = float(np.mean(after.max(axis=1) > 1e-2))
    print(f"held-out rel-L2 before {before.mean(0)} after {after.mean(0)}; fallback rate at 1e-2: {fallback:.2f}")


def test_inference_cost_against_the_plain_cascade(F):
    n = 128
    cfg = F.FnoConfig(n=n, width=48, hidden=128, layers=4, modes=(32, 32, 16))
    model = F.Fno(cfg, seed=0)
    casc = F.PlainCascade(n, 256)
    bowls = F.draw_bowls(2, 7)
    casc.incident(bowls[0], 0)
    t_plain = _ms(lambda: casc.harmonics(bowls[0]))
    x = torch.view_as_real(casc.p1_box / casc.p1_box.abs().max()).reshape(-1, 2).float().contiguous()
    y = torch.empty((n ** 3, 8), dtype=torch.float32, device="cuda")
    t_sur = _ms(lambda: model.infer(x, y))
    print(f"128^3: surrogate {t_sur:.3f} ms vs plain cascade {t_plain:.3f} ms per field "
          f"({'surrogate' if t_sur < t_plain else 'plain path'} faster by {max(t_sur, t_plain) / min(t_sur, t_plain):.2f}x)")
    assert 0 < t_sur < 1e3 and 0 < t_plain < 1e3
    assert torch.isfinite(y).all()
