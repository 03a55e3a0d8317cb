"""The bench step with V_{k1} on a side stream gives, bit for bit, what the same calls
give one after another on one stream (the side stream joins back before the step ends)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gw(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    import bench
    from paper_2011_03009_gb300 import synth
    return bench.GpuWorkload(synth.WORKLOADS["nested3"](), torch.device("cuda", 0))


def test_overlapped_step_equals_serial_calls(gw):
    assert gw.w.v1_grid is not None
    gw.step()
    torch.cuda.synchronize()
    got = {n: t.clone() for n, t in gw.outs.items()}
    # the same calls, serially on the current stream
    gw.plans[1].apply(gw.p1_v1, gw.outs[1])
    fields = {1: (gw.p1, gw.w.p1_grid)}
    for st in gw.w.steps:
        n = st.harmonic
        lower = [fields[m] for m in range(1, n)]
        if gw.nested[n]:
            gw.plans[n].source_from_nested([g for _, g in lower], [f for f, _ in lower])
        else:
            gw.plans[n].source_assemble([f for f, _ in lower])
        gw.plans[n].apply(None, gw.outs[n])
        fields[n] = (gw.outs[n], st.grid)
    torch.cuda.synchronize()
    for n, t in gw.outs.items():
        assert torch.equal(t, got[n]), n


def test_step_marks_show_the_first_harmonic_overlapping_v_k1(gw):
    """The events a timed step records: harmonic 2 starts beside V_{k1} (its spans are
    then re-timed alone); the outputs equal those of an unmarked step."""
    import bench
    gw.step()
    torch.cuda.synchronize()
    ref = {n: t.clone() for n, t in gw.outs.items()}
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    marks = {"side_end": ev(), "start": {st.harmonic: ev() for st in gw.w.steps}}
    a = ev()
    a.record()
    gw.step(marks=marks)
    torch.cuda.synchronize()
    side_end = a.elapsed_time(marks["side_end"])
    starts = {n: a.elapsed_time(e) for n, e in marks["start"].items()}
    assert side_end > 0 and all(t >= 0 for t in starts.values())
    assert 2 in bench.contended_harmonics([side_end], [starts])
    for n, t in gw.outs.items():
        assert torch.equal(t, ref[n]), n
