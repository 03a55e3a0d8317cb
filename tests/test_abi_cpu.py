"""C ABI checks that need no GPU: the library loads, exports every declared entry
point, and rejects bad arguments on the host before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")
HEADERS = sorted(os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h"))


def _declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names.update(re.findall(r"VP_API\s+[\w\s\*]+?\b(vp_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def vp():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_03009_gb300 import vp as vpmod
    return vpmod


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("vp_plan", "vp_kernel_fft", "vp_source_assemble", "vp_apply",
                     "vp_restrict_to_nested_box", "vp_destroy", "vp_status_string",
                     "vp_batch_create", "vp_batch_plan", "vp_batch_run", "vp_apply_static", "vp_plan_check",
                     "vp_fno_forward", "vp_fno_backward", "vp_fno_adam"):
        assert required in names


def test_library_exports_every_declared_symbol(vp):
    lib = ctypes.CDLL(vp.LIB_PATH)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(vp):
    assert vp.status_string(0) == "VP_OK"
    for code in range(-8, 0):
        assert vp.status_string(code).startswith("VP_ERR_")
    assert "unknown" in vp.status_string(-99)
    assert "sm_103a" in vp.vp_version()


def _medium(vp):
    return vp.vp_medium(1500.0, 1000.0, 3.5, 0.22, 2.0)


def _plan_status(vp, grid, harmonic=2, f0=1e6, med=None, opts=None):
    h = ctypes.c_void_p(0)
    st = vp.lib.vp_plan(ctypes.byref(grid) if grid is not None else None, harmonic, f0,
                        ctypes.byref(med if med is not None else _medium(vp)),
                        ctypes.byref(opts) if opts is not None else None, None, ctypes.byref(h))
    return st, h


def test_plan_rejects_bad_arguments_on_the_host(vp):
    good = vp.make_grid((8, 8, 8), (0, 0, 0), 1e-4)
    assert _plan_status(vp, None)[0] == vp.VP_ERR_ARG
    assert _plan_status(vp, vp.make_grid((0, 8, 8), (0, 0, 0), 1e-4))[0] == vp.VP_ERR_ARG
    assert _plan_status(vp, vp.make_grid((8, 8, 8), (0, 0, 0), 0.0))[0] == vp.VP_ERR_ARG
    assert _plan_status(vp, vp.make_grid((8, 8, 8), (0, 0, 0), -1e-4))[0] == vp.VP_ERR_ARG
    assert _plan_status(vp, good, harmonic=0)[0] == vp.VP_ERR_ARG
    assert _plan_status(vp, good, f0=0.0)[0] == vp.VP_ERR_ARG
    bad_med = vp.vp_medium(0.0, 1000.0, 3.5, 0.22, 2.0)
    assert _plan_status(vp, good, med=bad_med)[0] == vp.VP_ERR_ARG
    neg_att = vp.vp_medium(1500.0, 1000.0, 3.5, -1.0, 2.0)
    assert _plan_status(vp, good, med=neg_att)[0] == vp.VP_ERR_ARG
    st, h = _plan_status(vp, good, harmonic=99)
    assert st == vp.VP_ERR_UNSUPPORTED and not h.value
    for field in ("staging", "layout"):          # each 0 or 1
        for bad in (-1, 2):
            o = vp.vp_plan_opts()
            setattr(o, field, bad)
            st, h = _plan_status(vp, good, opts=o)
            assert st == vp.VP_ERR_ARG and not h.value, field
    assert vp.lib.vp_plan_check(None, None) == vp.VP_ERR_ARG


def test_plan_rejects_bad_sizes_on_the_host(vp):
    good = vp.make_grid((8, 8, 8), (0, 0, 0), 1e-4)
    o = vp.vp_plan_opts()
    o.m[0], o.m[1], o.m[2] = 14, 16, 16          # M < 2N - 1
    assert _plan_status(vp, good, opts=o)[0] == vp.VP_ERR_SIZE
    o = vp.vp_plan_opts()
    o.m[0], o.m[1], o.m[2] = 22, 16, 16          # 22 = 2 * 11 has no schedule
    assert _plan_status(vp, good, opts=o)[0] == vp.VP_ERR_SIZE
    o = vp.vp_plan_opts()
    o.radix[0][0], o.radix[0][1] = 4, 2          # product 8 != M = 16
    assert _plan_status(vp, good, opts=o)[0] == vp.VP_ERR_SIZE
    o = vp.vp_plan_opts()
    o.radix[0][0], o.radix[0][1] = 7, 2          # radix 7 unsupported
    assert _plan_status(vp, good, opts=o)[0] == vp.VP_ERR_SIZE
    assert _plan_status(vp, vp.make_grid((801, 8, 8), (0, 0, 0), 1e-4))[0] == vp.VP_ERR_SIZE


def test_other_calls_reject_bad_arguments_on_the_host(vp):
    P = ctypes.c_void_p
    assert vp.lib.vp_kernel_fft(None, None) == vp.VP_ERR_ARG
    assert vp.lib.vp_apply(None, None, P(16), None) == vp.VP_ERR_ARG
    assert vp.lib.vp_source_assemble(None, None, 1, 0, None, None) == vp.VP_ERR_ARG
    assert vp.lib.vp_destroy(None) == vp.VP_OK
    assert vp.lib.vp_vie_solve(None, P(64), P(64), P(64), 1e-6, 10, None, None, None) == vp.VP_ERR_ARG
    assert vp.lib.vp_vec_axpby(0, 1.0, 0.0, P(64), 0.0, 0.0, None, P(64), None) == vp.VP_ERR_ARG
    assert vp.lib.vp_vec_mul(4, None, P(64), P(64), None) == vp.VP_ERR_ARG
    d2 = (ctypes.c_double * 2)()
    assert vp.lib.vp_vec_dot(4, P(64), None, 1, d2, None) == vp.VP_ERR_ARG
    assert vp.lib.vp_source_assemble(None, None, 1, 1, None, None) == vp.VP_ERR_ARG
    assert vp.lib.vp_source_assemble(None, None, 1, 4, None, None) == vp.VP_ERR_ARG  # unknown flag
    assert vp.lib.vp_source_from_nested(None, None, None, 2, 0, None, None) == vp.VP_ERR_ARG
    n3 = (ctypes.c_int * 3)(4, 4, 4)
    box = (ctypes.c_int * 6)()
    assert vp.lib.vp_q0_box(n3, None, -1.0, box, None, None) == vp.VP_ERR_ARG
    assert vp.lib.vp_q0_box(n3, P(64), 0.5, box, None, None) == vp.VP_ERR_ARG
    assert vp.lib.vp_q0_box(n3, P(64), float("nan"), box, None, None) == vp.VP_ERR_ARG
    src2 = vp.make_grid((5, 5, 5), (0.0, 0.0, 0.0), 1e-3)
    assert vp.lib.vp_restrict_to_nested_box(ctypes.byref(src2), P(64), ctypes.byref(src2), P(64), 4,
                                            None) == vp.VP_ERR_ARG
    g8 = vp.make_grid((8, 8, 8), (0, 0, 0), 1e-4)
    assert vp.lib.vp_plan_retarget(None, ctypes.byref(g8), 2, 1e6, ctypes.byref(_medium(vp))) == vp.VP_ERR_ARG
    assert vp.lib.vp_profile_enable(None, 1) == vp.VP_ERR_ARG
    src = vp.make_grid((5, 5, 5), (0.0, 0.0, 0.0), 1e-3)
    dst_out = vp.make_grid((3, 3, 3), (0.0, 0.0, 0.0031), 1e-3)
    assert vp.lib.vp_restrict_to_nested_box(ctypes.byref(src), P(64), ctypes.byref(dst_out), P(64), 0,
                                            None) == vp.VP_ERR_NOT_NESTED
    assert vp.lib.vp_restrict_to_nested_box(ctypes.byref(src), None, ctypes.byref(src), P(64), 0,
                                            None) == vp.VP_ERR_ARG
    assert vp.lib.vp_restrict_to_nested_box(ctypes.byref(src), P(64), ctypes.byref(src), P(64), 8,
                                            None) == vp.VP_ERR_ARG
    med = _medium(vp)
    assert vp.lib.vp_incident_field(ctypes.byref(src), P(64), 0, 0.02, 0.01, 1e6, 1e5, ctypes.byref(med), P(64),
                                    None) == vp.VP_ERR_ARG
    assert vp.lib.vp_incident_field(ctypes.byref(src), P(64), 10, 0.02, 0.03, 1e6, 1e5, ctypes.byref(med), P(64),
                                    None) == vp.VP_ERR_ARG


def test_fno_descriptor_checks_on_the_host(vp):
    from paper_2011_03009_gb300 import fno
    P = ctypes.c_void_p
    cfg = fno.FnoConfig(n=16, width=8, hidden=12, layers=2, modes=(4, 6, 3))
    d = cfg.desc()
    W, H, (mx, my, mz) = 8, 12, cfg.modes
    per_layer = mx * my * mz * W * W * 2 + W * W + W
    expect = 10 * W + W + 2 * per_layer + W * H + H + H * 8 + 8
    assert fno.lib.vp_fno_param_count(ctypes.byref(d)) == expect
    offs = (ctypes.c_longlong * (3 * 2 + 7))()
    assert fno.lib.vp_fno_param_offsets(ctypes.byref(d), offs) == vp.VP_OK
    o = list(offs)
    assert o[0] == 0 and o[-1] == expect and all(b > a for a, b in zip(o, o[1:]))
    assert o[3] - o[2] == mx * my * mz * W * W * 2          # R_0
    assert fno.lib.vp_fno_workspace_bytes(ctypes.byref(d)) > 16 ** 3 * (2 + 8) * 4
    for bad in (dict(n=2), dict(width=0), dict(layers=9), dict(modes=(5, 6, 3)), dict(modes=(4, 18, 3)),
                dict(modes=(4, 6, 9)), dict(modes=(4, 6, 0))):
        bd = fno.FnoConfig(**{**dict(n=16, width=8, hidden=12, layers=2, modes=(4, 6, 3)), **bad}).desc()
        assert fno.lib.vp_fno_param_count(ctypes.byref(bd)) == -1, bad
        assert fno.lib.vp_fno_workspace_bytes(ctypes.byref(bd)) == -1, bad
        assert fno.lib.vp_fno_forward(ctypes.byref(bd), P(64), P(64), P(64), None, P(64), None) == vp.VP_ERR_ARG
    assert fno.lib.vp_fno_forward(ctypes.byref(d), None, P(64), P(64), None, P(64), None) == vp.VP_ERR_ARG
    assert fno.lib.vp_fno_adam(-1, P(64), P(64), P(64), P(64), P(64), 1e-3, 0.9, 0.999, 1e-8, 0.1, 0.001, 1.0,
                               None) == vp.VP_ERR_ARG
    assert fno.lib.vp_fno_to_bf16(4, None, P(64), None) == vp.VP_ERR_ARG


def test_binding_refuses_buffers_shorter_than_the_call_uses(vp):
    """The ABI takes bare pointers; the binding checks lengths before any call, so a short
    buffer never reaches a kernel (host-only: the check runs on CPU tensors here)."""
    import torch
    from paper_2011_03009_gb300 import synth
    g = synth.Grid((4, 5, 6), (0.0, 0.0, 0.0), 1e-4)
    assert vp._voxels(g) == 120 and vp._voxels(vp.grid_of(g)) == 120
    vp._need(torch.empty(120, dtype=torch.complex64), 120, "u")
    vp._need(torch.empty(200, dtype=torch.complex64), 120, "u")  # longer is fine
    vp._need(None, 120, "f")
    with pytest.raises(ValueError, match="119 elements"):
        vp._need(torch.empty(119, dtype=torch.complex64), 120, "u")


class _FakeField:
    """Stands in for a contiguous complex64 CUDA tensor (no GPU on the host)."""

    def __init__(self, n, dtype=None, shape=None):
        import torch
        self.dtype = dtype or torch.complex64
        self._n = n
        self.shape = shape or (n,)
        self.is_cuda = True

    def is_contiguous(self):
        return True

    def numel(self):
        return self._n

    def data_ptr(self):
        return 4096

    def dim(self):
        return len(self.shape)


class _FakeLib:
    """Records each ABI call and returns VP_OK (vp_plan_get_info fills m = 2N)."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            self.calls.append(name)
            if name == "vp_plan_get_info":
                info = args[1]._obj
                for a in range(3):
                    info.m[a] = 2 * (a + 4)
            return 0
        return call


def test_binding_marshals_every_call_with_length_checks(vp, monkeypatch):
    """Every binding entry point that takes fields, run against a fake library: correct
    lengths pass through to the ABI, a buffer one element short is refused first."""
    import torch
    from paper_2011_03009_gb300 import synth
    fake = _FakeLib()
    monkeypatch.setattr(vp, "lib", fake)
    monkeypatch.setattr(vp, "_stream", lambda stream: ctypes.c_void_p(0))
    g = synth.Grid((4, 5, 6), (0.0, 0.0, 0.0), 1e-4)
    gl = synth.Grid((3, 3, 3), (0.0, 0.0, 0.0), 2e-4)
    nv, nl = 120, 27
    plan = object.__new__(vp.Plan)
    plan._h, plan._g, plan.n = ctypes.c_void_p(1), vp.grid_of(g), g.n
    F = _FakeField
    batch = None
    try:
        octant = 5 * 6 * 7  # m = 8, 10, 12 from the fake info
        plan.kernel_spectrum_get(F(octant))
        plan.kernel_spectrum_set(F(octant))
        plan.source_assemble([F(nv), F(nv)], f_out=F(nv))
        plan.source_from_nested([gl, g], [F(nl), F(nv)], f_out=F(nv))
        plan.apply(F(nv), F(nv))
        plan.apply(None, F(nv))
        plan.vie_solve(F(nv), F(nv), F(nv))
        vp.vp_restrict_to_nested_box(gl, F(nl), g, F(nv))
        vp.vp_vec_axpby(1, F(nv), 2, F(nv), F(nv))
        vp.vp_vec_mul(F(nv), F(nv), F(nv))
        vp.vp_vec_dot(F(nv), F(nv))
        pts = F(30, dtype=torch.float64, shape=(10, 3))
        bowl = synth.Bowl(l=0.06, R=0.03, f0=1.1e6, p0=1e6)
        vp.vp_incident_field(g, pts, bowl, synth.WATER, F(nv))
        vp.vp_apply_static(g, 2, 1.1e6, synth.WATER, F(nv), F(nv))
        batch = vp.Batch([plan], [F(nv)], fs=[None], lowers=[[F(nv)]])
        batch.run()
        for name in ("vp_kernel_spectrum_get", "vp_source_from_nested", "vp_apply", "vp_vie_solve",
                     "vp_restrict_to_nested_box", "vp_vec_dot", "vp_incident_field", "vp_apply_static",
                     "vp_batch_create", "vp_batch_run"):
            assert name in fake.calls, name
        short = [
            lambda: plan.kernel_spectrum_get(F(octant - 1)),
            lambda: plan.source_assemble([F(nv), F(nv - 1)]),
            lambda: plan.source_from_nested([gl, g], [F(nl - 1), F(nv)]),
            lambda: plan.source_from_nested([gl], [F(nl), F(nv)]),
            lambda: plan.apply(F(nv), F(nv - 1)),
            lambda: plan.vie_solve(F(nv), F(nv - 1), F(nv)),
            lambda: vp.vp_restrict_to_nested_box(gl, F(nl), g, F(nv - 1)),
            lambda: vp.vp_vec_mul(F(nv), F(nv - 1), F(nv)),
            lambda: vp.vp_incident_field(g, F(30, dtype=torch.float64, shape=(30,)), bowl, synth.WATER, F(nv)),
            lambda: vp.vp_apply_static(g, 2, 1.1e6, synth.WATER, F(nv - 1), F(nv)),
            lambda: vp.Batch([plan], [F(nv - 1)], fs=[F(nv)]),
        ]
        for i, bad in enumerate(short):
            before = len(fake.calls)
            with pytest.raises(ValueError):
                bad()
            # refused before the ABI call (only the plan-info query may have run)
            assert set(fake.calls[before:]) <= {"vp_plan_get_info"}, (i, fake.calls[before:])
    finally:
        # the handles are fake: keep the destructors away from the real library
        plan._h = ctypes.c_void_p(0)
        if batch is not None:
            batch._h = ctypes.c_void_p(0)


def test_surrogate_binding_checks_activation_buffers(vp, monkeypatch):
    """The surrogate's forward, loss, backward and inference against a fake library:
    [N^3][2] inputs and [N^3][8] outputs/targets pass, a short or FP64 buffer is refused."""
    import torch
    from paper_2011_03009_gb300 import fno
    fake = _FakeLib()
    monkeypatch.setattr(fno, "lib", fake)
    monkeypatch.setattr(fno, "_s", lambda stream=None: ctypes.c_void_p(0))
    m = object.__new__(fno.Fno)
    m.cfg = fno.FnoConfig(n=4, width=4, hidden=8, layers=1, modes=(2, 2, 2))
    m.d = ctypes.c_int(0)
    m.params = m.params_bf16 = m.ws = m.grads = m.sums = torch.zeros(4)
    x, y = _FakeField(128, dtype=torch.float32), _FakeField(512, dtype=torch.float32)
    m.forward(x, y)
    m.forward(x)
    m.loss(y)
    m.backward(x, y)
    m.infer(x, y)
    assert fake.calls == ["vp_fno_forward", "vp_fno_forward", "vp_fno_loss", "vp_fno_backward", "vp_fno_infer"]
    for bad in (lambda: m.forward(_FakeField(127, dtype=torch.float32)),
                lambda: m.infer(x, _FakeField(511, dtype=torch.float32)),
                lambda: m.loss(_FakeField(512, dtype=torch.float64)),
                lambda: m.backward(x, _FakeField(100, dtype=torch.float32))):
        with pytest.raises(ValueError):
            bad()
    assert len(fake.calls) == 5


def test_batch_plan_refuses_bad_arguments_on_the_host(vp):
    """vp_batch_plan (plans first) validates like vp_batch_create before any device work."""
    P = ctypes.c_void_p
    out = P(0)
    plans = (P * 1)(None)
    us = (P * 1)(None)
    assert vp.lib.vp_batch_plan(plans, 0, None, None, us, ctypes.byref(out)) == vp.VP_ERR_ARG
    assert vp.lib.vp_batch_plan(plans, 1, None, None, us, ctypes.byref(out)) == vp.VP_ERR_ARG
    assert not out.value
