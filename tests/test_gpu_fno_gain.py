"""What the trained surrogate gains over the method without it, on the GPU.

A 64^3 surrogate is trained briefly on fields from the plain path (the judge), then:
- training gains accuracy: the held-out relative L2 error per harmonic drops well below
  that of the same network before training;
- inference gains speed: one surrogate evaluation takes less device time than the
  plain cascade it replaces (four kernel spectra, restrictions, sources, potentials),
  both starting from p1 on the device;
- every held-out sample is judged by the plain path: the samples above the 1e-2
  threshold are the ones that fall back (counted, not hidden).
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


def test_trained_surrogate_gains_accuracy_and_speed(F):
    n = 64
    cfg = F.FnoConfig(n=n, width=32, hidden=64, layers=3, modes=(16, 16, 8))
    xs, ts, _, kappa, _ = F.make_dataset(32, 5, n, 256)
    xv, tv, _, _, _ = F.make_dataset(6, 6, n, 256, kappa)
    model = F.Fno(cfg, seed=0)
    model.kappa = kappa
    before = np.array([model.rel_l2(x, t) for x, t in zip(xv, tv)])
    rng = np.random.default_rng(0)
    for ep in range(25):
        model.train_epoch(xs, ts, 2e-3 * (0.5 + 0.5 * np.cos(np.pi * ep / 25)), 4, rng.permutation(len(xs)))
    after = np.array([model.rel_l2(x, t) for x, t in zip(xv, tv)])
    # accuracy gained by training (the untrained network is the baseline)
    assert np.all(after.mean(axis=0) < 0.5 * before.mean(axis=0)), (before.mean(0), after.mean(0))
    # speed gained over the plain cascade from p1 (same GPU, same box)
    casc = F.PlainCascade(n, 256)
    bowls = F.draw_bowls(3, 7)
    casc.incident(bowls[0], 0)
    t_plain = _ms(lambda: casc.harmonics(bowls[0]))
    y = torch.empty((n ** 3, 8), dtype=torch.float32, device="cuda")
    t_sur = _ms(lambda: model.infer(xv[0], y))
    assert t_sur < t_plain, (t_sur, t_plain)
    fallback = float(np.mean(after.max(axis=1) > 1e-2))
    print(f"held-out rel-L2 before {before.mean(0)} after {after.mean(0)}; surrogate {t_sur:.3f} ms vs "
          f"plain {t_plain:.3f} ms; fallback rate at 1e-2: {fallback:.2f}")
