"""Batched evaluation (vp_batch_*): uneven grids and harmonics in grouped launches must
give the same fields as one plan at a time, and the oracle's."""
import numpy as np
import pytest
import torch

from oracle import cascade, potential, physics
from paper_2011_03009_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vp(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_03009_gb300 import vp as vpmod
    return vpmod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).cuda()


def test_batch_matches_single_plans_and_oracle(vp):
    # (n, harmonic, plain-or-source): groups of equal embedding, a mixed group, and
    # one radix-pass item (N = 21 -> M = 42) that runs on its own
    specs = [((40, 40, 40), 1, "f"), ((37, 33, 40), 1, "f"), ((48, 60, 48), 2, "src"), ((40, 40, 40), 3, "src"),
             ((21, 21, 21), 2, "src"), ((64, 64, 64), 2, "src"), ((60, 50, 64), 2, "src")]
    plans, us, fs, lowers, refs_in = [], [], [], [], []
    for i, (n, h, kind) in enumerate(specs):
        g = synth.Grid(n, (0.0, 0.0, 0.0), 9e-5)
        p = vp.vp_plan(g, h, 1.1e6, synth.WATER)
        p.kernel_fft()
        plans.append(p)
        us.append(torch.empty(n, dtype=torch.complex64, device="cuda"))
        if kind == "f":
            f = synth.random_field(n, 10 + i)
            fs.append(dev(f))
            lowers.append(None)
            refs_in.append(("f", f))
        else:
            lo = [synth.random_field(n, 100 * i + m) for m in range(1, h)]
            fs.append(None)
            lowers.append([dev(x) for x in lo])
            refs_in.append(("src", lo))
    batch = vp.Batch(plans, us, fs=fs, lowers=lowers)
    for _ in range(2):  # run twice: bound pointers, same results
        batch.run()
    torch.cuda.synchronize()
    got = [u.cpu().numpy().astype(np.complex128) for u in us]
    # single-plan path
    for i, (n, h, kind) in enumerate(specs):
        u1 = torch.empty(n, dtype=torch.complex64, device="cuda")
        if kind == "f":
            plans[i].apply(fs[i], u1)
        else:
            plans[i].source_assemble(lowers[i])
            plans[i].apply(None, u1)
        torch.cuda.synchronize()
        single = u1.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got[i] - single) <= 1e-6 * np.linalg.norm(single), i
        g = synth.Grid(n, (0.0, 0.0, 0.0), 9e-5)
        if kind == "f":
            ref = potential.apply_fft(refs_in[i][1], g.h, physics.wavenumber(h, 1.1e6, synth.WATER))
        else:
            ref = cascade.harmonic(h, refs_in[i][1], g.h, 1.1e6, synth.WATER)
        assert np.linalg.norm(got[i] - ref) <= 1e-5 * np.linalg.norm(ref), i
    batch.close()
    for p in plans:
        p.close()


def test_batch_rejects_a_plan_listed_twice(vp):
    g = synth.Grid((16, 16, 16), (0.0, 0.0, 0.0), 1e-4)
    p = vp.vp_plan(g, 1, 1e6, synth.WATER)
    u = torch.empty(g.n, dtype=torch.complex64, device="cuda")
    f = torch.zeros(g.n, dtype=torch.complex64, device="cuda")
    with pytest.raises(vp.VpError) as e:
        vp.Batch([p, p], [u, u], fs=[f, f])
    assert e.value.status == vp.VP_ERR_ARG
    p.close()


def test_batch_of_large_items(vp):
    """Items whose z sweeps fill the GPU several times over (96^3 and 96 x 96 x 90, M =
    192: 2304 tiles of 16 lines each) run the single-plan z kernel one after another
    inside the batch; the fields equal the single-plan ones and the oracle's."""
    specs = [((96, 96, 96), 2), ((96, 96, 90), 2)]
    plans, us, lowers, los = [], [], [], []
    for i, (n, h) in enumerate(specs):
        g = synth.Grid(n, (0.0, 0.0, 0.0), 9e-5)
        p = vp.vp_plan(g, h, 1.1e6, synth.WATER)
        assert tuple(p.info().m) == (192, 192, 192)
        p.kernel_fft()
        plans.append(p)
        us.append(torch.empty(n, dtype=torch.complex64, device="cuda"))
        lo = [synth.random_field(n, 700 + i)]
        los.append(lo)
        lowers.append([dev(x) for x in lo])
    batch = vp.Batch(plans, us, lowers=lowers)
    batch.run()
    torch.cuda.synchronize()
    for i, (n, h) in enumerate(specs):
        got = us[i].cpu().numpy().astype(np.complex128)
        u1 = torch.empty(n, dtype=torch.complex64, device="cuda")
        plans[i].source_assemble(lowers[i])
        plans[i].apply(None, u1)
        torch.cuda.synchronize()
        single = u1.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - single) <= 1e-6 * np.linalg.norm(single), i
        g = synth.Grid(n, (0.0, 0.0, 0.0), 9e-5)
        ref = cascade.harmonic(h, los[i], g.h, 1.1e6, synth.WATER)
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref), i
    batch.close()
    for p in plans:
        p.close()


def test_batch_follows_the_callers_stream_and_replays_from_a_graph(vp):
    """vp_batch_run on a non-default stream: inputs written on that stream just before
    the call (no synchronisation) must be seen, the results must be complete when the
    caller's stream continues, and a captured run replays on new inputs."""
    specs = [((40, 40, 40), 1), ((48, 60, 48), 1), ((64, 64, 64), 1), ((21, 21, 21), 1), ((37, 33, 40), 1)]
    plans, us, fs = [], [], []
    for n, h in specs:
        g = synth.Grid(n, (0.0, 0.0, 0.0), 9e-5)
        p = vp.vp_plan(g, h, 1.1e6, synth.WATER)
        p.kernel_fft()
        plans.append(p)
        us.append(torch.empty(n, dtype=torch.complex64, device="cuda"))
        fs.append(torch.empty(n, dtype=torch.complex64, device="cuda"))
    batch = vp.Batch(plans, us, fs=fs)
    srcs = [[dev(synth.random_field(n, 900 + 10 * r + i)) for i, (n, _) in enumerate(specs)] for r in range(3)]
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(s):
        # eager: inputs written on s, the batch on s, the results copied on s
        for f, x in zip(fs, srcs[0]):
            f.copy_(x)
        batch.run(stream=s)
        outs.append([u.clone() for u in us])
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        batch.run(stream=s)
    for r in (1, 2):
        with torch.cuda.stream(s):
            for f, x in zip(fs, srcs[r]):
                f.copy_(x)
            graph.replay()
            outs.append([u.clone() for u in us])
    torch.cuda.synchronize()
    for r in range(3):
        for i, (n, _) in enumerate(specs):
            u1 = torch.empty(n, dtype=torch.complex64, device="cuda")
            plans[i].apply(srcs[r][i], u1)
            torch.cuda.synchronize()
            single = u1.cpu().numpy().astype(np.complex128)
            got = outs[r][i].cpu().numpy().astype(np.complex128)
            assert np.linalg.norm(got - single) <= 1e-6 * np.linalg.norm(single), (r, i)
    batch.close()
    for p in plans:
        p.close()
