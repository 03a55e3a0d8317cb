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
                     "vp_batch_create", "vp_batch_run", "vp_apply_static",
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
