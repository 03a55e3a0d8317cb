"""Thin Python binding of libvp.so (the C ABI declared in include/vp.h).

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  Fields are torch.complex64 CUDA tensors (contiguous, C order);
torch supplies device memory and streams.  There is no CPU fallback: if libvp.so
is missing or fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libvp.so")

VP_OK = 0
VP_ERR_ARG = -1
VP_ERR_SIZE = -2
VP_ERR_NOMEM = -3
VP_ERR_CUDA = -4
VP_ERR_NOT_NESTED = -5
VP_ERR_STATE = -6
VP_ERR_TIMEOUT = -7
VP_ERR_UNSUPPORTED = -8
VP_RESTRICT_ZERO_OUTSIDE = 1
VP_RESTRICT_QUADRATIC = 2
VP_SRC_CONJ = 1
VP_ZFORM_AUTO, VP_ZFORM_TILE16, VP_ZFORM_TILE8, VP_ZFORM_TILE4, VP_ZFORM_PAIR8, VP_ZFORM_TILE4T = 0, 1, 2, 3, 4, 5
MAX_PASS = 8
MAX_LOWER = 8


class VpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


class vp_grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("origin", ctypes.c_double * 3), ("h", ctypes.c_double)]


class vp_medium(ctypes.Structure):
    _fields_ = [("c0", ctypes.c_double), ("rho0", ctypes.c_double), ("beta", ctypes.c_double),
                ("alpha0", ctypes.c_double), ("eta", ctypes.c_double)]


class vp_plan_opts(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int * 3), ("radix", (ctypes.c_int * MAX_PASS) * 3), ("autotune", ctypes.c_int),
                ("zform", ctypes.c_int), ("staging", ctypes.c_int), ("layout", ctypes.c_int),
                ("test_expire_waits", ctypes.c_int)]


class vp_plan_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("m", ctypes.c_int * 3), ("radix", (ctypes.c_int * MAX_PASS) * 3),
                ("k_re", ctypes.c_double), ("k_im", ctypes.c_double), ("c_n", ctypes.c_double),
                ("self_re", ctypes.c_double), ("self_im", ctypes.c_double),
                ("workspace_bytes", ctypes.c_ulonglong), ("khat_ready", ctypes.c_int), ("engine", ctypes.c_int * 3),
                ("zform", ctypes.c_int), ("staging", ctypes.c_int), ("group_y", ctypes.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libvp.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    sig = {
        "vp_plan": (I, [ctypes.POINTER(vp_grid), I, D, ctypes.POINTER(vp_medium), ctypes.POINTER(vp_plan_opts), P,
                        ctypes.POINTER(P)]),
        "vp_destroy": (I, [P]),
        "vp_plan_retarget": (I, [P, ctypes.POINTER(vp_grid), I, D, ctypes.POINTER(vp_medium)]),
        "vp_plan_get_info": (I, [P, ctypes.POINTER(vp_plan_info)]),
        "vp_plan_check": (I, [P, P]),
        "vp_kernel_fft": (I, [P, P]),
        "vp_kernel_spectrum_get": (I, [P, P, P]),
        "vp_kernel_spectrum_set": (I, [P, P, P]),
        "vp_source_assemble": (I, [P, ctypes.POINTER(P), I, I, P, P]),
        "vp_apply": (I, [P, P, P, P]),
        "vp_restrict_to_nested_box": (I, [ctypes.POINTER(vp_grid), P, ctypes.POINTER(vp_grid), P, I, P]),
        "vp_source_from_nested": (I, [P, ctypes.POINTER(vp_grid), ctypes.POINTER(P), I, I, P, P]),
        "vp_incident_field": (I, [ctypes.POINTER(vp_grid), P, I, D, D, D, D, ctypes.POINTER(vp_medium), P, P]),
        "vp_status_string": (ctypes.c_char_p, [I]),
        "vp_profile_enable": (I, [P, I]),
        "vp_profile_read": (I, [P, ctypes.POINTER(D), ctypes.POINTER(I), I]),
        "vp_version": (ctypes.c_char_p, []),
        "vp_apply_static": (I, [ctypes.POINTER(vp_grid), I, D, ctypes.POINTER(vp_medium), P, P, P]),
        "vp_vie_solve": (I, [P, P, P, P, D, I, ctypes.POINTER(I), ctypes.POINTER(D), P]),
        "vp_vec_axpby": (I, [ctypes.c_longlong, D, D, P, D, D, P, P, P]),
        "vp_vec_mul": (I, [ctypes.c_longlong, P, P, P, P]),
        "vp_vec_dot": (I, [ctypes.c_longlong, P, P, I, ctypes.POINTER(D), P]),
        "vp_q0_box": (I, [ctypes.POINTER(I), P, D, ctypes.POINTER(I), ctypes.POINTER(D), P]),
        "vp_batch_create": (I, [I, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                                ctypes.POINTER(P)]),
        "vp_batch_plan": (I, [ctypes.POINTER(P), I, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                              ctypes.POINTER(P)]),
        "vp_batch_run": (I, [P, P]),
        "vp_batch_destroy": (I, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    # the library must have been built from the sources in this tree
    from . import build as _build
    built = lib.vp_version().decode().rsplit(" ", 1)[-1]
    if built not in (_build.source_digest(False), _build.source_digest(True)):
        raise ImportError(f"libvp.so was built from other sources (digest {built}); run __graft_entry__.build()")
    return lib


lib = _load()


def status_string(status: int) -> str:
    return lib.vp_status_string(int(status)).decode()


def _check(status: int, where: str):
    if status != VP_OK:
        raise VpError(status, where)


def make_grid(n, origin, h) -> vp_grid:
    g = vp_grid()
    for a in range(3):
        g.n[a] = int(n[a])
        g.origin[a] = float(origin[a])
    g.h = float(h)
    return g


def grid_of(obj) -> vp_grid:
    """vp_grid from any object with .n, .origin, .h (e.g. synth.Grid)."""
    return make_grid(obj.n, obj.origin, obj.h)


def make_medium(m) -> vp_medium:
    return vp_medium(float(m.c0), float(m.rho0), float(m.beta), float(m.alpha0), float(m.eta))


def _stream(stream) -> ctypes.c_void_p:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _voxels(grid) -> int:
    """Voxel count of a grid (vp_grid or any object with .n)."""
    c = 1
    for v in grid.n:
        c *= int(v)
    return c


def _need(t, n: int, what: str) -> None:
    """The C ABI takes bare pointers: a buffer shorter than the call reads or writes would
    be accessed out of bounds on the device, so the binding refuses it first."""
    if t is not None and t.numel() < n:
        raise ValueError(f"{what}: {t.numel()} elements, the call uses {n}")


def _ptr(t, n: Optional[int] = None, what: str = "field") -> ctypes.c_void_p:
    import torch
    if t is None:
        return ctypes.c_void_p(0)
    if not (t.is_cuda and t.dtype == torch.complex64 and t.is_contiguous()):
        raise ValueError("fields must be contiguous torch.complex64 CUDA tensors")
    if n is not None:
        _need(t, n, what)
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A vp_plan_t with its grid; methods mirror the C ABI calls."""

    def __init__(self, grid, harmonic: int, f0: float, medium, m: Optional[Sequence[int]] = None,
                 radix: Optional[Sequence[Sequence[int]]] = None, autotune: bool = False, stream=None,
                 zform: int = 0, staging: int = 0, layout: int = 0, test_expire_waits: bool = False):
        self.grid = grid
        self.harmonic = int(harmonic)
        self._h = ctypes.c_void_p(0)
        opts = vp_plan_opts()
        if m is not None:
            for a in range(3):
                opts.m[a] = int(m[a])
        if radix is not None:
            for a in range(3):
                for i, r in enumerate(radix[a] or []):
                    opts.radix[a][i] = int(r)
        opts.autotune = 1 if autotune else 0
        opts.zform = int(zform)
        opts.staging = int(staging)
        opts.layout = int(layout)
        opts.test_expire_waits = 1 if test_expire_waits else 0
        g = grid if isinstance(grid, vp_grid) else grid_of(grid)
        self._g = g
        med = medium if isinstance(medium, vp_medium) else make_medium(medium)
        st = lib.vp_plan(ctypes.byref(g), self.harmonic, float(f0), ctypes.byref(med), ctypes.byref(opts),
                         _stream(stream) if autotune else ctypes.c_void_p(0), ctypes.byref(self._h))
        _check(st, "vp_plan")
        self.n = tuple(int(v) for v in g.n)

    def retarget(self, grid, harmonic: int, f0: float, medium):
        """vp_plan_retarget: same voxel counts, new spacing/origin/harmonic/f0/medium."""
        g = grid if isinstance(grid, vp_grid) else grid_of(grid)
        med = medium if isinstance(medium, vp_medium) else make_medium(medium)
        _check(lib.vp_plan_retarget(self._h, ctypes.byref(g), int(harmonic), float(f0), ctypes.byref(med)),
               "vp_plan_retarget")
        self.grid, self._g, self.harmonic = grid, g, int(harmonic)

    def info(self) -> vp_plan_info:
        inf = vp_plan_info()
        _check(lib.vp_plan_get_info(self._h, ctypes.byref(inf)), "vp_plan_get_info")
        return inf

    def check(self, stream=None) -> int:
        """vp_plan_check: synchronise the stream, read and clear the plan's device status
        word; returns VP_OK, VP_ERR_TIMEOUT (a bounded wait expired) or VP_ERR_STATE (an
        alignment refusal) without raising, since the caller asked for the status."""
        st = lib.vp_plan_check(self._h, _stream(stream))
        if st not in (VP_OK, VP_ERR_TIMEOUT, VP_ERR_STATE):
            _check(st, "vp_plan_check")
        return st

    def kernel_fft(self, stream=None):
        _check(lib.vp_kernel_fft(self._h, _stream(stream)), "vp_kernel_fft")

    def kernel_spectrum_get(self, dst, stream=None):
        _check(lib.vp_kernel_spectrum_get(self._h, _ptr(dst, self._octant(), "dst"), _stream(stream)),
               "vp_kernel_spectrum_get")

    def kernel_spectrum_set(self, src, stream=None):
        _check(lib.vp_kernel_spectrum_set(self._h, _ptr(src, self._octant(), "src"), _stream(stream)),
               "vp_kernel_spectrum_set")

    def _octant(self) -> int:
        m = self.info().m
        return (m[0] // 2 + 1) * (m[1] // 2 + 1) * (m[2] // 2 + 1)

    def source_assemble(self, lower, f_out=None, stream=None, conj: bool = False):
        """Eq. 2.6 from lower = [p_1 .. p_{n-1}], or with conj=True the full source of
        Eq. 2.5 from lower = [p_1 .. p_{N_h}] (all entries are read)."""
        nv = _voxels(self._g)
        arr = (ctypes.c_void_p * max(1, len(lower)))(*[_ptr(t, nv, "lower field").value for t in lower])
        _check(lib.vp_source_assemble(self._h, arr, len(lower), VP_SRC_CONJ if conj else 0, _ptr(f_out, nv, "f_out"),
                                      _stream(stream)), "vp_source_assemble")

    def source_from_nested(self, grids, lower, f_out=None, quadratic: bool = False, stream=None):
        """Eq. 2.6 from lower = [p_1 .. p_{n-1}] given on their own grids (grids[m-1] holds
        p_m): the restriction to this plan's grid and the products in one kernel."""
        if len(grids) != len(lower):
            raise ValueError("source_from_nested: one grid per lower field")
        gl = [g if isinstance(g, vp_grid) else grid_of(g) for g in grids]
        gs = (vp_grid * max(1, len(gl)))(*gl)
        arr = (ctypes.c_void_p * max(1, len(lower)))(
            *[_ptr(t, _voxels(gl[i]), "lower field").value for i, t in enumerate(lower)])
        _check(lib.vp_source_from_nested(self._h, gs, arr, len(lower), VP_RESTRICT_QUADRATIC if quadratic else 0,
                                         _ptr(f_out, _voxels(self._g), "f_out"), _stream(stream)),
               "vp_source_from_nested")

    def apply(self, f, u, stream=None):
        nv = _voxels(self._g)
        _check(lib.vp_apply(self._h, _ptr(f, nv, "f"), _ptr(u, nv, "u"), _stream(stream)), "vp_apply")

    def vie_solve(self, q, b, x, tol: float = 1e-6, max_iter: int = 200, stream=None):
        """Solve x - V[q x] = b (Section 7) by BiCGStab in the library; x holds the initial
        guess and receives the solution.  Returns (iterations, relative residual)."""
        it = ctypes.c_int(0)
        res = ctypes.c_double(0.0)
        nv = _voxels(self._g)
        _check(lib.vp_vie_solve(self._h, _ptr(q, nv, "q"), _ptr(b, nv, "b"), _ptr(x, nv, "x"), float(tol),
                                int(max_iter), ctypes.byref(it),
                                ctypes.byref(res), _stream(stream)), "vp_vie_solve")
        return it.value, res.value

    def profile_enable(self, on: bool = True):
        _check(lib.vp_profile_enable(self._h, 1 if on else 0), "vp_profile_enable")

    def profile_read(self, reset: bool = True):
        ms = (ctypes.c_double * 5)()
        cnt = (ctypes.c_int * 5)()
        _check(lib.vp_profile_read(self._h, ms, cnt, 1 if reset else 0), "vp_profile_read")
        return list(ms), list(cnt)

    def close(self):
        if self._h and self._h.value:
            lib.vp_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """vp_batch_t: items (plan, f or lower fields, u) bound once, run with grouped launches."""

    def __init__(self, plans, us, fs=None, lowers=None):
        count = len(plans)
        self._keep = (list(plans), list(us), fs, lowers)  # keep tensors and plans alive
        P = ctypes.c_void_p
        pa = (P * count)(*[p._h.value for p in plans])
        nv = [_voxels(p._g) for p in plans]
        ua = (P * count)(*[_ptr(t, nv[i], "u").value for i, t in enumerate(us)])
        fa = None
        if fs is not None:
            fa = (P * count)(*[(_ptr(t, nv[i], "f").value if t is not None else None) for i, t in enumerate(fs)])
        la = None
        if lowers is not None:
            flat = []
            for i in range(count):
                row = list(lowers[i] or [])
                flat += [_ptr(t, nv[i], "lower field").value for t in row] + [None] * (MAX_LOWER - len(row))
            la = (P * (count * MAX_LOWER))(*flat)
        self._h = P(0)
        _check(lib.vp_batch_create(count, pa, fa, la, ua, ctypes.byref(self._h)), "vp_batch_create")

    def run(self, stream=None):
        _check(lib.vp_batch_run(self._h, _stream(stream)), "vp_batch_run")

    def close(self):
        if self._h and self._h.value:
            lib.vp_batch_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- module-level calls with the C ABI's names ---------------------------------------

def vp_plan(grid, harmonic: int, f0: float, medium, **kw) -> Plan:
    return Plan(grid, harmonic, f0, medium, **kw)


def vp_kernel_fft(plan: Plan, stream=None):
    plan.kernel_fft(stream)


def vp_source_assemble(plan: Plan, lower, f_out=None, stream=None):
    plan.source_assemble(lower, f_out, stream)


def vp_source_from_nested(plan: Plan, grids, lower, f_out=None, quadratic: bool = False, stream=None):
    plan.source_from_nested(grids, lower, f_out, quadratic, stream)


def vp_apply(plan: Plan, f, u, stream=None):
    plan.apply(f, u, stream)


def vp_restrict_to_nested_box(src_grid, src, dst_grid, dst, zero_outside: bool = False, quadratic: bool = False,
                              stream=None):
    gs = src_grid if isinstance(src_grid, vp_grid) else grid_of(src_grid)
    gd = dst_grid if isinstance(dst_grid, vp_grid) else grid_of(dst_grid)
    flags = (VP_RESTRICT_ZERO_OUTSIDE if zero_outside else 0) | (VP_RESTRICT_QUADRATIC if quadratic else 0)
    _check(lib.vp_restrict_to_nested_box(ctypes.byref(gs), _ptr(src, _voxels(gs), "src"), ctypes.byref(gd),
                                         _ptr(dst, _voxels(gd), "dst"), flags,
                                         _stream(stream)), "vp_restrict_to_nested_box")


def vp_vec_axpby(a, x, b, y, out, stream=None):
    """out = a x + b y (complex scalars; y may be None)."""
    a, b = complex(a), complex(b)
    n = x.numel()
    _check(lib.vp_vec_axpby(n, a.real, a.imag, _ptr(x), b.real, b.imag, _ptr(y, n, "y"), _ptr(out, n, "out"),
                            _stream(stream)),
           "vp_vec_axpby")


def vp_vec_mul(x, y, out, stream=None):
    n = x.numel()
    _check(lib.vp_vec_mul(n, _ptr(x), _ptr(y, n, "y"), _ptr(out, n, "out"), _stream(stream)), "vp_vec_mul")


def vp_vec_dot(x, y, conj_x: bool = True, stream=None) -> complex:
    """sum conj(x) y (or sum x y), accumulated in FP64."""
    out = (ctypes.c_double * 2)()
    n = x.numel()
    _check(lib.vp_vec_dot(n, _ptr(x), _ptr(y, n, "y"), 1 if conj_x else 0, out, _stream(stream)), "vp_vec_dot")
    return complex(out[0], out[1])


def vp_q0_box(field, q0: float, stream=None):
    """Smallest index box holding every voxel with log10(|f| / max|f|) >= q0 (Section 5).
    Returns (lo, hi, max_abs) with inclusive bounds per axis."""
    n = (ctypes.c_int * 3)(*field.shape)
    box = (ctypes.c_int * 6)()
    m = ctypes.c_double(0.0)
    _check(lib.vp_q0_box(n, _ptr(field), float(q0), box, ctypes.byref(m), _stream(stream)), "vp_q0_box")
    return tuple(box[0:3]), tuple(box[3:6]), m.value


def vp_incident_field(grid, points, bowl, medium, out, stream=None):
    """p1 on `grid` (Eq. 3.10); points: (n_p, 3) float64 CUDA tensor."""
    import torch
    if not (points.is_cuda and points.dtype == torch.float64 and points.is_contiguous()
            and points.dim() == 2 and points.shape[1] == 3):
        raise ValueError("points must be a contiguous float64 CUDA tensor of shape (n_p, 3)")
    g = grid if isinstance(grid, vp_grid) else grid_of(grid)
    med = medium if isinstance(medium, vp_medium) else make_medium(medium)
    _check(lib.vp_incident_field(ctypes.byref(g), ctypes.c_void_p(points.data_ptr()), int(points.shape[0]),
                                 float(bowl.l), float(bowl.R), float(bowl.f0), float(bowl.p0), ctypes.byref(med),
                                 _ptr(out, _voxels(g), "out"), _stream(stream)), "vp_incident_field")


VP_STATIC_MAX_N = 64


def vp_apply_static(grid, harmonic: int, f0: float, medium, f, u, stream=None):
    """u = V_{k_n}[f] without any device allocation (grids up to 64 voxels per axis).

    For callers that cannot allocate device memory (stream capture, memory owned by
    another allocator); shares one fixed device array across calls, so calls must
    not overlap on the GPU."""
    g = grid if isinstance(grid, vp_grid) else grid_of(grid)
    med = medium if isinstance(medium, vp_medium) else make_medium(medium)
    nv = _voxels(g)
    _check(lib.vp_apply_static(ctypes.byref(g), int(harmonic), float(f0), ctypes.byref(med), _ptr(f, nv, "f"),
                               _ptr(u, nv, "u"),
                               _stream(stream)), "vp_apply_static")


def vp_version() -> str:
    return lib.vp_version().decode()
