#!/usr/bin/env python3
"""Benchmark of the nested-mesh harmonic volume-potential path on GB300.

One step = one pass of the hot path over the workload's harmonics, through the
C ABI: V_{k1}[p1] on the fundamental grid, and for each harmonic n >= 2 the
restriction of the lower harmonics onto grid n fused with the source products (one
kernel), and the volume potential.  V_{k1}[p1] depends on nothing else in the step, so
it runs on a side stream overlapped with the harmonic chain.  Kernel spectra are built before timing (cached per plan, timed
separately); the incident field p1 is an input and is generated before timing.

Default workload: the full nested-mesh run, harmonics 1-5 of a 7.5 cm / 15 cm /
1.1 MHz / 2 MPa bowl in water: V_{k1}[p1] on the 600 x 600 x 640 fundamental grid and
harmonics 2-5 on 320^3, 384^3, 432^3 and 512^3 focal boxes at lambda_n / 6 (the
largest configuration; --workload nested3 runs the 128^3 / 192^3 / 256^3 one).

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "voxel-potentials/s"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="nested5",
                    choices=["small", "nested3", "nested5", "batch64", "vie", "fullcascade", "q0", "nw", "restrict",
                             "fno", "apply"])
    ap.add_argument("--grid", default="128,128,640", help="voxels per axis for --workload apply")
    ap.add_argument("--harmonic", type=int, default=2, help="harmonic for --workload apply")
    ap.add_argument("--zform", type=int, default=0, help="z-sweep form for --workload apply (VP_ZFORM_*)")
    ap.add_argument("--staging", type=int, default=0,
                    help="z-sweep staging for --workload apply: 0 bulk copies (4-line forms), 1 cp.async")
    ap.add_argument("--layout", type=int, default=0,
                    help="x-sweep output layout for --workload apply: 0 grouped by 4 y-planes, 1 plain")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT comparison timing")
    ap.add_argument("--fno-checkpoint", default=None, help="trained surrogate weights (--workload fno)")
    return ap.parse_args()


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------- distributed

def dist_init(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)  # one GPU per rank before any collective
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def max_over_ranks(value: float, world: int) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(voxels: int, steps: int, world: int, total_ms: float) -> float:
    """Whole-job throughput: voxels of every rank's steps over the slowest rank's time."""
    return voxels * steps * world / (total_ms / 1e3)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# --------------------------------------------------------------------------- workload on GPU

def sweep_bytes(n, m, harmonic, fused_source: bool):
    """Algorithmic bytes of each of the five sweeps of one volume-potential evaluation."""
    Nx, Ny, Nz = n
    Mx, My, Mz = m
    W = 8
    nvox = Nx * Ny * Nz
    src_fields = (harmonic - 1) if fused_source else 1
    octant = (Mx // 2 + 1) * (My // 2 + 1) * (Mz // 2 + 1)
    return [
        W * (src_fields * nvox + Mx * Ny * Nz),
        W * (Mx * Ny * Nz + Mx * My * Nz),
        W * (2 * Mx * My * Nz + octant),
        W * (Mx * My * Nz + Mx * Ny * Nz),
        W * (Mx * Ny * Nz + nvox),
    ]


SWEEP_NAMES = ["x_forward_source", "y_forward", "z_conv", "y_inverse", "x_inverse"]


# device code of the z-sweep kernels (the bench's dominant kernels): the register DFTs and
# shared helpers they are built from, the pipelined kernel's section of sweeps2.cuh and,
# for the pair-split form, its own header
SWEEP_SOURCES = ("fft_engine.cuh", "regfft.cuh", "vp_internal.cuh")
ZSWEEP_SECTION = "// Persistent, software-pipelined form of line2_kernel<kConv>"


def csrc_digest(kernel: str = "") -> str:
    """Short digest of a z-sweep kernel's device code; a stored ncu traffic figure is
    used only while it matches (a change of that kernel invalidates it)."""
    import hashlib
    d = os.path.join(ROOT, "paper_2011_03009_gb300", "csrc")
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    with open(os.path.join(d, "sweeps2.cuh"), "rb") as fh:
        text = fh.read()
    i = text.find(ZSWEEP_SECTION.encode())
    h.update(b"sweeps2.cuh\0" + (text[i:] if i >= 0 else text))
    if kernel.startswith("line2_conv_pair8_kernel"):
        with open(os.path.join(d, "sweeps2_pair.cuh"), "rb") as fh:
            h.update(b"sweeps2_pair.cuh\0" + fh.read())
    return h.hexdigest()[:12]


def stored_traffic(kernel: str):
    """DRAM bytes per launch (read + write) of `kernel` from profiles/dram_traffic.txt, or None.

    Each line: <kernel label with spaces replaced by _> <csrc digest> <read bytes> <write bytes>.
    """
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    key, dig = kernel.replace(" ", "_"), csrc_digest(kernel)
    with open(path) as fh:
        for line in fh:
            f = line.split()
            if len(f) == 4 and not line.startswith("#") and f[0] == key and f[1] == dig:
                return int(float(f[2])) + int(float(f[3]))
    return None


def contended_harmonics(side_end_ms, start_ms):
    """Harmonics of the chain that began, in some timed step, before the side stream's
    work had finished: their per-sweep event spans include waits for the GPU that the
    side stream held, so they are timed again alone.

    side_end_ms[i]: time from step i's start to the end of the side stream's work;
    start_ms[i][n]: time from step i's start to the start of harmonic n."""
    out = set()
    for end, starts in zip(side_end_ms, start_ms):
        out.update(n for n, t in starts.items() if t < end)
    return out


def kernel_name(sweep: int, m, engine, fused_source: bool = True) -> str:
    """Name of the CUDA kernel that runs one sweep (two-level or radix-pass engine)."""
    axis = (0, 1, 2, 1, 0)[sweep]
    L = m[axis]
    if engine[axis]:
        if sweep == 2:
            # the pipelined z sweep (its lines are always half-padded here: N <= M / 2 on
            # every axis); at L = 1280 its 4-line form with the factors swapped (40 x 32)
            return f"line2_conv_pipe_kernel (L={L})"
        kind = ("forward, source" if sweep == 0 and fused_source else "forward") if sweep < 2 else "inverse"
        return f"col2_kernel {kind} (L={L})"
    if sweep == 2:
        return f"line_sweep_kernel<conv> (L={L})"
    return f"col_sweep_kernel (L={L})"


class GpuWorkload:
    def __init__(self, w, device):
        import torch
        from paper_2011_03009_gb300 import synth
        from paper_2011_03009_gb300 import vp
        self.w, self.vp, self.torch, self.dev = w, vp, torch, device
        # default priority: a high-priority side stream ends V_{k1} inside harmonic 2 but
        # measured 1.7% slower per step (1.569 against 1.542 ms at 128/192/256^3)
        self.side = torch.cuda.Stream(device)
        pts = synth.sample_bowl_points(w.bowl, w.n_points, w.seed)
        self.pts = torch.from_numpy(pts).to(device)
        c64 = torch.complex64
        # inputs: p1 on the grid of harmonic 2 (and on the fundamental grid for V_{k1}),
        # from the Rayleigh sum (input generator, timed separately with CUDA events)
        self.p1 = torch.empty(w.p1_grid.n, dtype=c64, device=device)
        self.p1_v1 = None
        if w.v1_grid is not None:
            self.p1_v1 = torch.empty(w.v1_grid.n, dtype=c64, device=device)
        vp.vp_incident_field(w.p1_grid, self.pts, w.bowl, w.medium, self.p1)  # warm-up
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        vp.vp_incident_field(w.p1_grid, self.pts, w.bowl, w.medium, self.p1)
        if w.v1_grid is not None:
            vp.vp_incident_field(w.v1_grid, self.pts, w.bowl, w.medium, self.p1_v1)
        ev1.record()
        torch.cuda.synchronize()
        pairs = (w.p1_grid.voxels + (w.v1_grid.voxels if w.v1_grid is not None else 0)) * w.n_points
        self.incident = {"ms": round(ev0.elapsed_time(ev1), 3), "voxel_point_pairs": pairs,
                         "pairs_per_s": pairs / (ev0.elapsed_time(ev1) * 1e-3)}
        self.plans, self.outs = {}, {}
        if w.v1_grid is not None:
            self.plans[1] = vp.vp_plan(w.v1_grid, 1, w.bowl.f0, w.medium)
            self.outs[1] = torch.empty(w.v1_grid.n, dtype=c64, device=device)
        home = {1: w.p1_grid}
        # harmonics whose lower fields live on other grids: restriction and products in
        # one kernel (vp_source_from_nested); the others fuse the products into the
        # first sweep (vp_source_assemble)
        self.nested = {}
        for st in w.steps:
            n = st.harmonic
            self.plans[n] = vp.vp_plan(st.grid, n, w.bowl.f0, w.medium)
            self.outs[n] = torch.empty(st.grid.n, dtype=c64, device=device)
            self.nested[n] = any(home[m] is not st.grid for m in range(1, n))
            home[n] = st.grid
        self.grids = {st.harmonic: st.grid for st in w.steps}
        if w.v1_grid is not None:
            self.grids_v1 = w.v1_grid
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for p in self.plans.values():
            p.kernel_fft()
        torch.cuda.synchronize()
        self.khat_build_ms = 1e3 * (time.perf_counter() - t0)

    def launches_per_step(self) -> int:
        n = 0
        if 1 in self.plans and self.p1_v1 is not None:
            n += 5
        for st in self.w.steps:
            n += 5 + (1 if self.nested[st.harmonic] else 0)
        return n

    def step(self, p1=None, p1_v1=None, marks=None):
        """One pass of the hot path.  `marks` (optional): {"side_end": event, "start":
        {n: event}} recorded at the end of the side stream's work and before each
        harmonic of the chain, which tells afterwards which harmonics overlapped it."""
        w = self.w
        p1 = self.p1 if p1 is None else p1
        p1_v1 = self.p1_v1 if p1_v1 is None else p1_v1
        main = self.torch.cuda.current_stream()
        if w.v1_grid is not None:
            # V_{k1}[p1] on the fundamental grid depends on nothing else in the step: it
            # runs on a side stream, overlapped with the harmonic chain on the caller's
            self.side.wait_stream(main)
            self.plans[1].apply(p1_v1, self.outs[1], stream=self.side)
            if marks is not None:
                marks["side_end"].record(self.side)
        for st in w.steps:
            if marks is not None:
                marks["start"][st.harmonic].record(main)
            self.run_harmonic(st.harmonic, p1)
        if w.v1_grid is not None:
            main.wait_stream(self.side)

    def run_harmonic(self, n, p1=None):
        """Source and potential of harmonic n of the chain, from p1 and the lower
        harmonics' latest outputs."""
        w = self.w
        fields = {1: (self.p1 if p1 is None else p1, w.p1_grid)}
        for st in w.steps:
            if st.harmonic < n:
                fields[st.harmonic] = (self.outs[st.harmonic], st.grid)
        plan = self.plans[n]
        if self.nested[n]:
            plan.source_from_nested([fields[m][1] for m in range(1, n)], [fields[m][0] for m in range(1, n)])
        else:
            plan.source_assemble([fields[m][0] for m in range(1, n)])
        plan.apply(None, self.outs[n])

    def time_nested_sources(self, flush, reps: int = 20):
        """CUDA-event time of each nested-source kernel (restriction of every lower field
        and the products, one launch) with its algorithmic bytes: the lower fields read
        once, the source written once.  Outside the timed step; L2 flushed before each."""
        import numpy as np
        import torch
        out = []
        fields = {1: (self.p1, self.w.p1_grid)}
        for st in self.w.steps:
            n = st.harmonic
            if self.nested[n]:
                plan = self.plans[n]
                grids = [fields[m][1] for m in range(1, n)]
                lower = [fields[m][0] for m in range(1, n)]
                f = torch.empty(st.grid.n, dtype=torch.complex64, device=self.p1.device)
                ms = 0.0
                for _ in range(reps):
                    flush.zero_()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    plan.source_from_nested(grids, lower, f_out=f)
                    b.record()
                    torch.cuda.synchronize()
                    ms += a.elapsed_time(b)
                ms /= reps
                by = 8 * (sum(int(np.prod(g.n)) for g in grids) + int(np.prod(st.grid.n)))
                out.append({"harmonic": n, "kernel": "source_nested_tiled_kernel",
                            "sources": [list(g.n) for g in grids], "n": list(st.grid.n),
                            "ms_per_launch": round(ms, 5), "bytes_per_launch": by,
                            "gbs": round(by / (ms * 1e-3) / 1e9, 1)})
            fields[n] = (self.outs[n], st.grid)
        return out

    def plan_geometry(self):
        out = {}
        for n, p in self.plans.items():
            inf = p.info()
            out[n] = (tuple(inf.n), tuple(inf.m), tuple(inf.engine))
        return out


def run_ours(args, world, rank, local):
    import numpy as np  # noqa: F401
    import torch
    from paper_2011_03009_gb300 import synth

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    w = synth.WORKLOADS[args.workload]()
    gw = GpuWorkload(w, device)
    voxels = w.voxels_per_step
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream()

    for _ in range(max(3, args.warmup)):
        gw.step()
    torch.cuda.synchronize()

    # per-sweep events inside the timed steps for the harmonic chain; the overlapped
    # V_{k1} of the side stream is timed on its own afterwards (its spans there would
    # include the chain's kernels), and so is any chain harmonic that began before V_{k1}
    # ended
    overlapped = 1 if gw.w.v1_grid is not None else None
    for n, p in gw.plans.items():
        p.profile_read(reset=True)
        p.profile_enable(n != overlapped)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    marks = [None] * args.steps
    if overlapped is not None:
        marks = [{"side_end": torch.cuda.Event(enable_timing=True),
                  "start": {st.harmonic: torch.cuda.Event(enable_timing=True) for st in gw.w.steps}}
                 for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()  # evict the previous step's data from L2 (outside the timed events)
        ev[i][0].record(stream)
        gw.step(marks=marks[i])
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    # outside the timed region: no bounded device wait expired and no buffer was refused
    for n, p in gw.plans.items():
        if p.check() != 0:
            raise RuntimeError(f"harmonic {n}: the plan's device status reports an expired wait or a refused buffer")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), world)
    ms_per_step = total_ms / args.steps
    value = aggregate_value(voxels, args.steps, world, total_ms)

    alone = set()
    if overlapped is not None:
        p = gw.plans[overlapped]
        p.profile_enable(True)
        for _ in range(min(args.steps, 50)):
            flush.zero_()
            p.apply(gw.p1_v1, gw.outs[overlapped])
        torch.cuda.synchronize()
        alone.add(overlapped)
        # chain harmonics that overlapped V_{k1}: their in-step spans are discarded and
        # their sweeps timed alone in the same way
        side_end = [a.elapsed_time(m["side_end"]) for (a, _), m in zip(ev, marks)]
        starts = [{n: a.elapsed_time(e) for n, e in m["start"].items()} for (a, _), m in zip(ev, marks)]
        for n in sorted(contended_harmonics(side_end, starts)):
            p = gw.plans[n]
            p.profile_read(reset=True)
            for _ in range(min(args.steps, 50)):
                flush.zero_()
                gw.run_harmonic(n)
            torch.cuda.synchronize()
            alone.add(n)

    # per-sweep kernel timing (events on the launching stream; the harmonic chain inside
    # the timed region, the overlapped V_{k1} alone after it)
    geo = gw.plan_geometry()
    sweeps = []
    for n, p in gw.plans.items():
        p.profile_enable(False)
        ms, cnt = p.profile_read(reset=True)
        nn, mm, eng = geo[n]
        fused = n >= 2 and not gw.nested.get(n, False)
        by = sweep_bytes(nn, mm, n, fused)
        for s in range(5):
            if cnt[s] == 0:
                continue
            per_launch_ms = ms[s] / cnt[s]
            name = SWEEP_NAMES[s] if s or fused else "x_forward"
            sweeps.append({"harmonic": n, "sweep": name, "kernel": kernel_name(s, mm, eng, fused),
                           "n": list(nn), "m": list(mm), "timed": "alone" if n in alone else "in step",
                           "launches": cnt[s], "ms_per_launch": per_launch_ms, "bytes_per_launch": by[s],
                           "gbs": by[s] / (per_launch_ms * 1e-3) / 1e9, "total_ms": ms[s]})
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    # each sweep launches once per step: the dominant kernel has the longest launch
    dom = max(sweeps, key=lambda r: r["ms_per_launch"]) if sweeps else None
    roofline = None
    if dom:
        roofline = {"bound": "hbm", "kernel": f"{dom['kernel']}, harmonic {dom['harmonic']}",
                    "achieved": round(dom["gbs"], 1), "peak": hbm_peak, "peak_source": peak_src,
                    "unit": "GB/s", "frac": round(dom["gbs"] / hbm_peak, 4), "traffic": stored_traffic(dom["kernel"]),
                    "bytes_per_launch": dom["bytes_per_launch"], "ms_per_launch": round(dom["ms_per_launch"], 5),
                    "timed": dom["timed"]}
    # whole-apply model bytes ((25 + n) words per voxel for M = 2N) per harmonic
    per_h = {}
    for n, p in gw.plans.items():
        rows = [r for r in sweeps if r["harmonic"] == n]
        t = sum(r["ms_per_launch"] for r in rows)
        by = sum(r["bytes_per_launch"] for r in rows)
        vox = int(np.prod(geo[n][0]))
        per_h[str(n)] = {"voxels": vox, "apply_ms": round(t, 4), "voxels_per_s": vox / (t * 1e-3),
                         "model_gbs": round(by / (t * 1e-3) / 1e9, 1), "hbm_frac": round(by / (t * 1e-3) / 1e9 / hbm_peak, 4)}

    nested_sources = gw.time_nested_sources(flush)

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(gw, args, world, voxels, flush)

    cufft = None
    if rank == 0 and world == 1 and not args.no_cufft:
        cufft = cufft_comparison(gw, flush)

    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, gw)
        parity = sampled_parity(gw)


    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": {"workload": w.name, "harmonics": ([1] if w.v1_grid is not None else []) + [s.harmonic for s in w.steps],
                   "grids": {str(n): list(geo[n][0]) for n in geo}, "embedding": {str(n): list(geo[n][1]) for n in geo},
                   "engine": {str(n): list(geo[n][2]) for n in geo},
                   "voxels_per_step": voxels, "bowl_points": w.n_points, "parallelism": f"replicas x{world}",
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "streams": ("V_k1 on a side stream, overlapped with the harmonic chain; its per-sweep "
                               "times, and those of chain harmonics that began before it ended, measured "
                               "alone after the timed steps") if w.v1_grid is not None else "one",
                   "khat_build_ms": round(gw.khat_build_ms, 2), "incident_field": gw.incident},
        "roofline": roofline, "per_harmonic": per_h, "sweeps": sweeps, "nested_sources": nested_sources,
        "e2e": e2e, "cpu_baseline": cpu, "rel_l2_per_harmonic": parity, "cufft_comparison": cufft, "clocks": clk,
        "gpu_launches": gw.launches_per_step() * args.steps, "wall_s_timed": round(t_wall, 4),
    }
    if rank == 0:
        print(json.dumps(line))


def cufft_comparison(gw, flush):
    """cuFFT (through torch.fft), timed as a comparison only: the same zero-padded
    circulant convolution per harmonic (pad f into an M^3 cube, 3-D FFT, multiply by a
    full M^3 spectrum, inverse 3-D FFT, crop), unpruned, outside the metric.  The
    spectrum's values do not change the work; a random cube stands in for it."""
    import torch
    out = {}
    for n, p in gw.plans.items():
        inf = p.info()
        N, M = tuple(inf.n), tuple(inf.m)
        # spectrum, padded cube, transform output and cuFFT's work area: ~5 cubes
        need = 5 * 8 * M[0] * M[1] * M[2]
        free, _ = torch.cuda.mem_get_info(gw.dev)
        if need > 0.8 * free:
            out[str(n)] = {"n": list(N), "m": list(M), "skipped": f"needs ~{need / 2**30:.0f} GiB of device memory"}
            continue
        f = torch.randn(N, dtype=torch.complex64, device=gw.dev)
        K = torch.randn(M, dtype=torch.complex64, device=gw.dev)
        cube = torch.zeros(M, dtype=torch.complex64, device=gw.dev)
        u = torch.empty(N, dtype=torch.complex64, device=gw.dev)

        def conv():
            cube.zero_()
            cube[:N[0], :N[1], :N[2]] = f
            F = torch.fft.fftn(cube)
            F *= K
            u.copy_(torch.fft.ifftn(F)[:N[0], :N[1], :N[2]])

        for _ in range(3):
            conv()
        torch.cuda.synchronize()
        ts = []
        for _ in range(5):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            conv()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        ms = sorted(ts)[len(ts) // 2]
        vox = N[0] * N[1] * N[2]
        out[str(n)] = {"n": list(N), "m": list(M), "ms": round(ms, 4), "voxels_per_s": vox / (ms * 1e-3)}
        del f, K, cube, u
    torch.cuda.empty_cache()
    return out


def gpu_local_cpus(dev_index: int):
    """(NUMA node, set of CPUs) the GPU is attached to, from sysfs; None if unknown."""
    try:
        import torch
        pr = torch.cuda.get_device_properties(dev_index)
        base = f"/sys/bus/pci/devices/{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
        with open(base + "/numa_node") as fh:
            node = int(fh.read().strip())
        if node < 0:
            return None
        with open(f"/sys/devices/system/node/node{node}/cpulist") as fh:
            text = fh.read().strip()
        cpus = set()
        for part in text.split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        return node, cpus
    except (OSError, ValueError, AttributeError, RuntimeError):
        return None


def measure_e2e(gw, args, world, voxels, flush):
    """Same metric through the public API with pinned host inputs/outputs, copies inside.

    Steps are independent, so they are pipelined the way a serving loop would run them:
    the host->device copy of step k+1's inputs and the device->host copy of step k's
    results run on their own streams while step k+1 computes (inputs and outputs are
    double-buffered; events order each buffer's reuse).  The timed region runs from
    before the first input copy to after the last result has reached host memory, so
    every step's copies are inside it."""
    import torch
    # the pinned host buffers are allocated (and their pages placed) from the CPUs of the
    # GPU's own NUMA node, and the copies are issued from there
    local = gpu_local_cpus(gw.dev.index if gw.dev.index is not None else 0)
    old_affinity = None
    if local is not None and hasattr(os, "sched_setaffinity"):
        try:
            old_affinity = os.sched_getaffinity(0)
            os.sched_setaffinity(0, local[1] & old_affinity or local[1])
        except OSError:
            old_affinity = None
    h2d_s, comp_s, d2h_s = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    nb = 2
    h_p1 = [gw.p1.cpu().pin_memory() for _ in range(nb)]
    h_v1 = [gw.p1_v1.cpu().pin_memory() for _ in range(nb)] if gw.p1_v1 is not None else None
    d_p1 = [torch.empty_like(gw.p1) for _ in range(nb)]
    d_v1 = [torch.empty_like(gw.p1_v1) for _ in range(nb)] if gw.p1_v1 is not None else None
    outs = [{n: torch.empty_like(o) for n, o in gw.outs.items()} for _ in range(nb)]
    h_out = [{n: torch.empty(o.shape, dtype=o.dtype).pin_memory() for n, o in gw.outs.items()} for _ in range(nb)]
    bi = gw.p1.numel() * 8 + (gw.p1_v1.numel() * 8 if gw.p1_v1 is not None else 0)
    bo = sum(o.numel() * 8 for o in gw.outs.values())
    K = max(3, min(args.steps, 16))
    ev = lambda: torch.cuda.Event()
    in_ready = [ev() for _ in range(nb)]
    in_free = [ev() for _ in range(nb)]
    out_ready = [ev() for _ in range(nb)]
    out_free = [ev() for _ in range(nb)]
    for e in in_free + out_free:
        e.record(torch.cuda.current_stream())
    saved = gw.outs

    def run(steps):
        for k in range(steps):
            i = k % nb
            with torch.cuda.stream(h2d_s):
                h2d_s.wait_event(in_free[i])
                d_p1[i].copy_(h_p1[i], non_blocking=True)
                if d_v1 is not None:
                    d_v1[i].copy_(h_v1[i], non_blocking=True)
                in_ready[i].record(h2d_s)
            with torch.cuda.stream(comp_s):
                comp_s.wait_event(in_ready[i])
                comp_s.wait_event(out_free[i])
                gw.outs = outs[i]
                gw.step(p1=d_p1[i], p1_v1=d_v1[i] if d_v1 is not None else None)
                in_free[i].record(comp_s)
                out_ready[i].record(comp_s)
            with torch.cuda.stream(d2h_s):
                d2h_s.wait_event(out_ready[i])
                for n, o in outs[i].items():
                    h_out[i][n].copy_(o, non_blocking=True)
                out_free[i].record(d2h_s)

    # warm-up: the first two uses of each pinned host buffer ran at a fraction of the
    # copy engines' rate (30-70 GB/s against 190-210 GB/s from the third on)
    run(3 * nb)
    torch.cuda.synchronize()
    barrier(world)
    # three timed runs of K steps (the host copies' rate varies between runs); the median
    reps = []
    for _ in range(3):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(h2d_s)
        run(K)
        # the end event waits for the last results on the host-copy stream
        b.record(d2h_s)
        torch.cuda.synchronize()
        reps.append(max_over_ranks(a.elapsed_time(b), world))
    ms = statistics.median(reps)
    gw.outs = saved
    if old_affinity is not None:
        os.sched_setaffinity(0, old_affinity)
    return {"value": voxels * K * world / (ms / 1e3), "unit": METRIC, "h2d_bytes_per_step": bi,
            "host_numa_node": local[0] if local is not None else None,
            "d2h_bytes_per_step": bo, "steps": K, "repeats_ms_per_step": [round(r / K, 3) for r in reps],
            "pipelined": "inputs/outputs double-buffered on copy streams; median of three timed runs"}


# --------------------------------------------------------------------------- CPU oracle legs

ORACLE_SAMPLE_MAX_M3 = 640 ** 3  # padded cube of the oracle's timed sample (complex128: 4.2 GB)


def oracle_grid(w):
    """(harmonic, grid) of the oracle's bounded sample: the first grid of the run, in the
    order V_{k1}, harmonic 2, 3, ..., whose padded cube (M = 2N) is at most 640^3."""
    cands = ([(1, w.v1_grid)] if w.v1_grid is not None else []) + [(st.harmonic, st.grid) for st in w.steps]
    for n_h, g in cands:
        if 8 * g.n[0] * g.n[1] * g.n[2] <= ORACLE_SAMPLE_MAX_M3:
            return n_h, g
    return cands[-1]


def oracle_sample(w):
    """Bounded sample of the workload for the FP64 oracle: one volume potential of the
    run on the grid oracle_grid names (kernel spectrum prepared outside the timing)."""
    import numpy as np
    from oracle import physics, potential
    from paper_2011_03009_gb300 import synth
    n_h, g = oracle_grid(w)
    k = physics.wavenumber(n_h, w.bowl.f0, w.medium)
    f = synth.smooth_blob_field(g, (w.bowl.l, 0.0, 0.0), 20 * g.h, k.real)
    khat = potential.kernel_spectrum(g.n, g.h, k)
    return g, f, k, khat, np.prod(g.n)


def cpu_baseline(w, gw=None):
    """The FP64 oracle timed on the host cores; with the GPU workload given, the same
    apply on the same synthetic input through the C ABI is compared with it (rel-L2)."""
    import numpy as np
    from oracle import potential
    g, f, k, khat, vox = oracle_sample(w)
    reps, t_total = 0, 0.0
    u_ref = None
    while t_total < 10.0 and reps < 20:
        t0 = time.perf_counter()
        u_ref = potential.apply_fft(f, g.h, k, khat=khat)
        t_total += time.perf_counter() - t0
        reps += 1
    n_h = oracle_grid(w)[0]
    out = {"value": vox * reps / t_total, "unit": METRIC, "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"FP64 oracle apply_fft (zero-padded FFT convolution, spectrum precomputed) on the "
                     f"{'x'.join(map(str, g.n))} grid of harmonic {n_h}, {reps} repetitions"}
    if gw is not None:
        import torch
        fd = torch.from_numpy(np.ascontiguousarray(f).astype(np.complex64)).to(gw.dev)
        ud = torch.empty_like(fd)
        gw.plans[n_h].apply(fd, ud)
        got = ud.cpu().numpy().astype(np.complex128)
        out["rel_l2_vs_oracle"] = {"harmonic": n_h, "grid": list(g.n),
                                   "value": float(np.linalg.norm(got - u_ref) / np.linalg.norm(u_ref))}
        # every other harmonic of the run at its full size, where the oracle's padded
        # cube (M^3 complex128) stays within 2 GiB: the plan's apply on a synthetic
        # smooth source against the oracle's (not timed)
        from oracle import physics
        from paper_2011_03009_gb300 import synth
        per_h = []
        for st in w.steps:
            n, gs = st.harmonic, st.grid
            if np.prod([2 * v for v in gs.n]) > 512 ** 3:
                continue
            kn = physics.wavenumber(n, w.bowl.f0, w.medium)
            fs = synth.smooth_blob_field(gs, (w.bowl.l, 0.0, 0.0), 20 * gs.h, kn.real)
            ref = potential.apply_fft(fs, gs.h, kn)
            fd = torch.from_numpy(np.ascontiguousarray(fs).astype(np.complex64)).to(gw.dev)
            ud = torch.empty_like(fd)
            gw.plans[n].apply(fd, ud)
            got = ud.cpu().numpy().astype(np.complex128)
            per_h.append({"harmonic": n, "grid": list(gs.n),
                          "value": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))})
        if per_h:
            out["rel_l2_vs_oracle_per_harmonic"] = per_h
    return out


def sampled_parity(gw, count=2048):
    """Rel-L2 of every harmonic's volume potential against the FP64 oracle at the run's
    full sizes, in the timed launch configuration: a seeded source that is non-zero on a
    16^3 block and the two far corners, applied by the plan on the whole grid, and the
    oracle's direct sum of Eq. 3.9 (apply_sparse) at `count` uniform targets, the 8
    corners and 256 voxels among and next to the block.  Not timed."""
    import numpy as np
    import torch
    from oracle import physics, potential
    from paper_2011_03009_gb300 import synth
    out = []
    for n, p in gw.plans.items():
        inf = p.info()
        N = tuple(inf.n)
        idx, val = synth.sparse_block_source(N, 16, seed=100 + n)
        val32 = val.astype(np.complex64)
        tg = synth.sample_targets(N, idx, count, seed=200 + n)
        f = torch.zeros(N, dtype=torch.complex64, device=gw.dev)
        it = torch.from_numpy(idx).to(gw.dev)
        f[it[:, 0], it[:, 1], it[:, 2]] = torch.from_numpy(val32).to(gw.dev)
        u = torch.empty_like(f)
        p.apply(f, u)
        tt = torch.from_numpy(tg).to(gw.dev)
        got = u[tt[:, 0], tt[:, 1], tt[:, 2]].cpu().numpy().astype(np.complex128)
        del f, u
        k = physics.wavenumber(n, gw.w.bowl.f0, gw.w.medium)
        g = gw.w.v1_grid if (n == 1 and gw.w.v1_grid is not None) else gw.grids[n]
        ref = potential.apply_sparse(idx, val32.astype(np.complex128), g.h, k, tg)
        out.append({"harmonic": n, "grid": list(N), "m": list(inf.m), "targets": len(tg), "sources": len(idx),
                    "rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                    "max_abs_err_over_max_abs": float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))})
    torch.cuda.empty_cache()
    return {"method": "plan applied to a sparse seeded source on the full grid; FP64 oracle direct sum of "
                      "Eq. 3.9 at sampled target voxels", "rows": out}


def run_reference(args, world, rank):
    from paper_2011_03009_gb300 import synth
    from oracle import potential
    if rank != 0:
        return
    w = synth.WORKLOADS[args.workload]()
    g, f, k, khat, vox = oracle_sample(w)
    for _ in range(max(1, args.warmup)):
        potential.apply_fft(f, g.h, k, khat=khat)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        potential.apply_fft(f, g.h, k, khat=khat)
    dt = time.perf_counter() - t0
    value = vox * args.steps / dt
    sample = (f"FP64 oracle apply_fft on the {'x'.join(map(str, g.n))} grid of {w.name} "
              f"(spectrum precomputed), one evaluation per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": w.name, "sample_grid": list(g.n)},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# --------------------------------------------------------------------------- batched workload

def run_batch(args, world, rank, local):
    """64 seeded transducer configurations x harmonics 1-3 on uneven nested grids:
    a loop of single-instance calls versus grouped batched launches replayed from a
    CUDA graph.  Metric: harmonic fields per second."""
    import torch
    from paper_2011_03009_gb300 import synth
    from paper_2011_03009_gb300 import vp

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    count = 64
    inst = synth.draw_batch_instances(count, seed=4)
    c64 = torch.complex64
    n_points = 512  # bowl points per instance (input generator only)
    items = []
    t0 = time.perf_counter()
    for i, b in enumerate(inst):
        pts = torch.from_numpy(synth.sample_bowl_points(b.bowl, n_points, 4000 + i)).to(dev)
        g1, g2, g3 = b.grids
        it = {"grids": b.grids, "bowl": b.bowl}
        it["p1_g1"] = torch.empty(g1.n, dtype=c64, device=dev)
        it["p1_g2"] = torch.empty(g2.n, dtype=c64, device=dev)
        vp.vp_incident_field(g1, pts, b.bowl, synth.WATER, it["p1_g1"])
        vp.vp_incident_field(g2, pts, b.bowl, synth.WATER, it["p1_g2"])
        it["plans"] = [vp.vp_plan(g, n, b.bowl.f0, synth.WATER, autotune=True) for n, g in ((1, g1), (2, g2), (3, g3))]
        for p in it["plans"]:
            p.kernel_fft()
        it["u"] = [torch.empty(g.n, dtype=c64, device=dev) for g in (g1, g2, g3)]
        it["f3"] = torch.empty(g3.n, dtype=c64, device=dev)
        items.append(it)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0

    # harmonic 3's source from p1 and p2 on grid 2: restriction and products in one
    # kernel per instance (vp_source_from_nested), in both forms
    def nested_all():
        for it in items:
            g1, g2, g3 = it["grids"]
            it["plans"][2].source_from_nested([g2, g2], [it["p1_g2"], it["u"][1]], f_out=it["f3"])

    def plain_step():
        for it in items:
            p1, p2, p3 = it["plans"]
            g1, g2, g3 = it["grids"]
            p1.apply(it["p1_g1"], it["u"][0])
            p2.source_assemble([it["p1_g2"]])
            p2.apply(None, it["u"][1])
            p3.source_from_nested([g2, g2], [it["p1_g2"], it["u"][1]])
            p3.apply(None, it["u"][2])

    b1 = vp.Batch([it["plans"][0] for it in items], [it["u"][0] for it in items], fs=[it["p1_g1"] for it in items])
    b2 = vp.Batch([it["plans"][1] for it in items], [it["u"][1] for it in items],
                  lowers=[[it["p1_g2"]] for it in items])
    b3 = vp.Batch([it["plans"][2] for it in items], [it["u"][2] for it in items], fs=[it["f3"] for it in items])

    def batched_step():
        b1.run()
        b2.run()
        nested_all()
        b3.run()

    def timeit(fn, reps, repeats=5):
        """Per-step milliseconds of `repeats` timings of `reps` steps each (after warm-up)."""
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        out = []
        for _ in range(repeats):
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                fn()
            z.record()
            torch.cuda.synchronize()
            out.append(a.elapsed_time(z) / reps)
        return out

    def summary(ts):
        med = statistics.median(ts)
        return {"fields_per_s": fields / (med / 1e3), "ms_per_step": med, "ms_min": min(ts), "ms_max": max(ts),
                "repeats": len(ts)}

    fields = 3 * count
    reps = max(3, min(args.steps, 20))
    t_plain = timeit(plain_step, reps)
    t_batched = timeit(batched_step, reps)
    # graph of the batched step
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        batched_step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batched_step()
    t_graph = timeit(graph.replay, reps)
    graph_p = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph_p):
        plain_step()
    t_plain_graph = timeit(graph_p.replay, reps)
    ms_graph = statistics.median(t_graph)
    groups = {"h1": len(set(tuple(it["plans"][0].info().m) for it in items)),
              "h2": len(set(tuple(it["plans"][1].info().m) for it in items)),
              "h3": len(set(tuple(it["plans"][2].info().m) for it in items))}
    voxels = sum(g.voxels for it in items for g in it["grids"])
    line = {"metric": "fields/s", "value": fields / (ms_graph / 1e3), "unit": "fields/s", "n_gpus": 1,
            "steps": reps, "warmup": max(3, args.warmup), "ms_per_step": ms_graph, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "batch64_h1-3_uneven_96-256cube", "instances": count, "fields_per_step": fields,
                       "voxels_per_step": voxels, "bowl_points": n_points, "embedding_groups": groups,
                       "setup_s": round(setup_s, 2)},
            "plain_loop": summary(t_plain), "plain_loop_graph": summary(t_plain_graph),
            "batched": summary(t_batched), "batched_graph": summary(t_graph),
            "voxel_potentials_per_s": voxels / (ms_graph / 1e3)}
    if rank == 0:
        print(json.dumps(line))


def _dev_timeit(fn, reps, warmup):
    import torch
    for _ in range(max(1, warmup)):
        fn()
    torch.cuda.synchronize()
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    z.record()
    torch.cuda.synchronize()
    return a.elapsed_time(z) / reps


def _line(metric, value, unit, ms, steps, warmup, higher, config, **extra):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": steps, "warmup": warmup,
         "ms_per_step": ms, "higher_is_better": higher, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
         "data": "synthetic", "config": config}
    d.update(extra)
    print(json.dumps(d))


def _focal_setup(n, harmonic_spacing, n_points=4096, seed=2):
    """128^3-class focal grid of the 3 cm / 6 cm / 1.1 MHz bowl and p1 on it."""
    import torch
    from paper_2011_03009_gb300 import synth, vp
    bowl = synth.Bowl(l=0.06, R=0.03, f0=1.1e6, p0=1.0e6)
    g = synth.focus_grid(bowl, (n, n, n), harmonic_spacing)
    pts = torch.from_numpy(synth.sample_bowl_points(bowl, n_points, seed)).cuda()
    p1 = torch.empty(g.n, dtype=torch.complex64, device="cuda")
    vp.vp_incident_field(g, pts, bowl, synth.WATER, p1)
    return bowl, g, p1


def run_vie(args):
    """Inhomogeneous medium (Section 7): tissue sphere (r = 4 mm) at the focus of the
    nested3 bowl, harmonic 1 on a 128^3 grid at lambda_1/6; b = p_inc; BiCGStab to 1e-6."""
    import numpy as np
    import torch
    from paper_2011_03009_gb300 import synth, vp
    bowl, g, p_inc = _focal_setup(128, 1)
    X, Y, Z = np.meshgrid(g.axis(0), g.axis(1), g.axis(2), indexing="ij")
    inside = (X - bowl.l - 1e-3) ** 2 + (Y - 5e-4) ** 2 + Z ** 2 <= 4e-3 ** 2
    # wavenumbers (with attenuation) from the library's own plan constants
    plan = vp.vp_plan(g, 1, bowl.f0, synth.WATER)
    inf = plan.info()
    kbg = complex(inf.k_re, inf.k_im)
    tplan = vp.vp_plan(synth.Grid((1, 1, 1), (0, 0, 0), g.h), 1, bowl.f0, synth.TISSUE)
    kin = complex(tplan.info().k_re, tplan.info().k_im)
    tplan.close()
    q = torch.from_numpy(np.where(inside, kin * kin - kbg * kbg, 0.0).astype(np.complex64)).cuda()
    plan.kernel_fft()
    x = torch.zeros_like(p_inc)
    stats = {}

    def solve():
        x.zero_()
        stats["it"], stats["res"] = plan.vie_solve(q, p_inc, x, tol=1e-6, max_iter=200)

    reps = max(1, min(args.steps, 5))
    ms = _dev_timeit(solve, reps, min(args.warmup, 2))
    applies = 2 * stats["it"] + 1
    cpu = None if args.no_cpu_baseline else _vie_cpu_baseline(bowl)
    _line("VIE solves/s", 1e3 / ms, "solves/s", ms, reps, min(args.warmup, 2), True,
          {"workload": "vie_tissue_sphere_r4mm_128cube_h1_R3cm_l6cm_1.1MHz", "grid": list(g.n),
           "solver": "BiCGStab", "tol": 1e-6, "inclusion_voxels": int(inside.sum())},
          iterations=stats["it"], relres=stats["res"], ms_per_iteration=ms / max(1, stats["it"]),
          operator_applies=applies, voxel_potentials_per_s=applies * g.voxels / (ms / 1e3), cpu_baseline=cpu)


def _vie_cpu_baseline(bowl):
    """FP64 oracle (GMRES on the same discrete operator) on a 32^3 grid of the same
    recipe: voxel-potentials/s of its operator applications."""
    import numpy as np
    from oracle import physics, potential, vie
    from paper_2011_03009_gb300 import synth
    g = synth.focus_grid(bowl, (32, 32, 32), 1)
    kk = vie.sphere_wavenumber(g, (bowl.l + 1e-3, 5e-4, 0.0), 4e-3, 1, bowl.f0, synth.WATER, synth.TISSUE)
    kb = physics.wavenumber(1, bowl.f0, synth.WATER)
    q = vie.contrast(kk, kb)
    b = synth.random_field(g.n, 1)
    count = {"n": 0}
    op = vie.operator(q, g.h, kb)

    def counted(x):
        count["n"] += 1
        return op(x)
    import scipy.sparse.linalg as sla
    import inspect
    A = sla.LinearOperator((q.size, q.size), matvec=counted, dtype=np.complex128)
    kw = {"rtol": 1e-6} if "rtol" in inspect.signature(sla.gmres).parameters else {"tol": 1e-6}
    t0 = time.perf_counter()
    sla.gmres(A, b.reshape(-1), atol=0.0, restart=60, maxiter=50, **kw)
    dt = time.perf_counter() - t0
    return {"value": count["n"] * g.voxels / dt, "unit": "voxel-potentials/s", "cores": os.cpu_count(),
            "kind": "oracle", "sample": f"FP64 oracle GMRES to 1e-6 on a 32^3 grid of the same recipe "
                                        f"({count['n']} operator applications, {dt:.2f} s)"}


def run_fullcascade(args):
    """Eq. 2.5 with N_h = 5 on one 128^3 focal grid at lambda_5/6 (Jacobi from Eq. 2.6)."""
    import torch
    from paper_2011_03009_gb300 import cascade, synth
    bowl, g, p_inc = _focal_setup(128, 5)
    fc = cascade.FullCascade(g, 5, bowl.f0, synth.WATER)
    stats = {}

    def solve():
        _, hist = fc.run(p_inc, max_iter=30, tol=1e-6)
        stats["hist"] = hist

    reps = max(1, min(args.steps, 3))
    ms = _dev_timeit(solve, reps, min(args.warmup, 1))
    sweeps = len(stats["hist"])
    cpu = None
    if not args.no_cpu_baseline:
        import numpy as np
        from oracle import cascade as ocascade
        gs = synth.focus_grid(bowl, (32, 32, 32), 5)
        p_inc_s = synth.random_field(gs.n, 3, scale=4.0e5)  # synthetic input of the oracle's own
        t0 = time.perf_counter()
        ocascade.full_cascade(p_inc_s, 5, gs.h, bowl.f0, synth.WATER, iters=3)
        dt = time.perf_counter() - t0
        applies = 4 + 3 * 5  # weakly nonlinear start + 3 sweeps of 5 harmonics
        cpu = {"value": applies * gs.voxels / dt, "unit": "voxel-potentials/s", "cores": os.cpu_count(),
               "kind": "oracle", "sample": f"FP64 oracle full cascade, 3 Jacobi sweeps of N_h = 5 on a 32^3 grid "
                                           f"({dt:.2f} s)"}
    _line("full-cascade solves/s", 1e3 / ms, "solves/s", ms, reps, min(args.warmup, 1), True,
          {"workload": "fullcascade_Nh5_128cube_h5spacing_R3cm_l6cm_1.1MHz", "grid": list(g.n), "harmonics": 5,
           "tol": 1e-6},
          sweeps=sweeps, change_history=stats["hist"], ms_per_sweep=ms / max(1, sweeps),
          voxel_potentials_per_s=(5 * (sweeps + 1)) * g.voxels / (ms / 1e3), cpu_baseline=cpu)
    fc.close()


def run_q0(args):
    """Section 5 domain study on the nested3 harmonic-3 source (256^3 at lambda_3/6)."""
    import torch
    from paper_2011_03009_gb300 import domain, synth, vp
    wl = synth.WORKLOADS["nested3"]()
    g2, g3 = wl.steps[0].grid, wl.steps[1].grid
    pts = torch.from_numpy(synth.sample_bowl_points(wl.bowl, wl.n_points, wl.seed)).cuda()
    p1 = torch.empty(g2.n, dtype=torch.complex64, device="cuda")
    vp.vp_incident_field(g2, pts, wl.bowl, wl.medium, p1)
    plan2 = vp.vp_plan(g2, 2, wl.bowl.f0, wl.medium)
    plan2.kernel_fft()
    p2 = torch.empty_like(p1)
    plan2.source_assemble([p1])
    plan2.apply(None, p2)
    r1 = torch.empty(g3.n, dtype=torch.complex64, device="cuda")
    r2 = torch.empty_like(r1)
    vp.vp_restrict_to_nested_box(g2, p1, g3, r1)
    vp.vp_restrict_to_nested_box(g2, p2, g3, r2)
    plan3 = vp.vp_plan(g3, 3, wl.bowl.f0, wl.medium)
    f3 = torch.empty_like(r1)
    plan3.source_assemble([r1, r2], f_out=f3)
    q0s = [-0.5, -1.0, -1.5, -2.0, -3.0, -4.0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rows = domain.q0_study(g3, 3, wl.bowl.f0, f3, r1, q0s, wl.medium)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import domain as odomain
        # the oracle times its own synthetic field of the same size (no input from the GPU path)
        f_host = synth.smooth_blob_field(g3, (wl.bowl.l, 0.0, 0.0), 20 * g3.h, 1.0).astype("complex64")
        t0 = time.perf_counter()
        for q0 in q0s:
            odomain.q0_box(f_host, q0)
        dt = time.perf_counter() - t0
        t1 = time.perf_counter()
        for q0 in q0s:
            vp.vp_q0_box(f3, q0)
        dt_gpu = time.perf_counter() - t1
        cpu = {"value": dt, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"FP64 oracle Q0 boxes of the same 256^3 source for the {len(q0s)} thresholds "
                         f"(the GPU's vp_q0_box for the same: {dt_gpu:.4f} s including host sync)"}
    _line("Q0 study time", sec, "s", sec * 1e3, 1, 0, False,
          {"workload": "q0_study_h3_256cube_nested3", "q0": q0s, "grid": list(g3.n)}, rows=rows, cpu_baseline=cpu)


def run_restrict(args):
    """The standalone restriction (Section 6, step 2a) of the default workload: a field on
    the 192^3 grid of harmonic 2 onto the 256^3 grid of harmonic 3, linear and quadratic;
    CUDA events, L2 flushed before each launch."""
    import numpy as np
    import torch
    from paper_2011_03009_gb300 import synth, vp
    wl = synth.WORKLOADS["nested3"]()
    g2, g3 = wl.steps[0].grid, wl.steps[1].grid
    f = torch.from_numpy(synth.random_field(g2.n, seed=1).astype(np.complex64)).cuda()
    out = torch.empty(g3.n, dtype=torch.complex64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    reps = max(3, min(args.steps, 50))
    rows = {}
    for quad in (False, True):
        for _ in range(max(3, args.warmup)):
            vp.vp_restrict_to_nested_box(g2, f, g3, out, quadratic=quad)
        ms = 0.0
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            vp.vp_restrict_to_nested_box(g2, f, g3, out, quadratic=quad)
            b.record()
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
        ms /= reps
        by = 8 * (g2.voxels + g3.voxels)
        rows["quadratic" if quad else "linear"] = {"ms": round(ms, 5), "model_gbs": round(by / (ms * 1e-3) / 1e9, 1)}
    _line("restricted voxels/s", g3.voxels / (rows["linear"]["ms"] * 1e-3), "voxels/s", rows["linear"]["ms"], reps,
          max(3, args.warmup), True, {"workload": "restrict_192to256_nested3", "src": list(g2.n), "dst": list(g3.n)},
          orders=rows)


def run_fno(args):
    """Surrogate inference (4 layers, width 48, projection 128, 32 x 32 x 16 modes) on the
    128^3 focal box against the plain cascade it would replace (kernel spectra, nested
    sources and potentials of harmonics 2..5 from p1 on the device); CUDA events.  The
    inference time does not depend on the weights' values (random initialisation unless
    --fno-checkpoint names trained weights).  Then the judged route per bowl: incident
    fields, inference, the plain path's p2 as judge, the plain cascade as fallback,
    against the plain route from the bowl; with the fallback rate."""
    import torch
    from paper_2011_03009_gb300 import fno as F
    n = 128
    cfg = F.FnoConfig(n=n, width=48, hidden=128, layers=4, modes=(32, 32, 16))
    model = F.Fno(cfg, seed=0)
    if args.fno_checkpoint:
        model.load_state(torch.load(args.fno_checkpoint))
    casc = F.PlainCascade(n, 512)
    bowl = F.draw_bowls(1, 7)[0]
    casc.incident(bowl, 0)
    x = torch.view_as_real(casc.p1_box / casc.p1_box.abs().max()).reshape(-1, 2).float().contiguous()
    y = torch.empty((n ** 3, 8), dtype=torch.float32, device="cuda")
    reps = max(3, min(args.steps, 20))
    t_inf = _dev_timeit(lambda: model.infer(x, y), reps, args.warmup)
    t_plain = _dev_timeit(lambda: casc.harmonics(bowl), reps, args.warmup)
    bowls = F.draw_bowls(8, 8)
    judged = F.JudgedSurrogate(model, threshold=1e-2, n_points=512)
    plain = F.PlainCascade(n, 512)
    verdicts = []

    def judged_all():
        verdicts.clear()
        for i, b in enumerate(bowls):
            verdicts.append(judged.run(b, i)[1])

    def plain_all():
        for i, b in enumerate(bowls):
            plain.run(b, i)

    t_judged = _dev_timeit(judged_all, 2, 1) / len(bowls)
    t_plain_route = _dev_timeit(plain_all, 2, 1) / len(bowls)
    fb = sum(v["fallback"] for v in verdicts) / len(verdicts)
    locality = _box_locality(F, plain, bowls)
    _line("surrogate fields/s", 1e3 / t_inf, "fields/s", t_inf, reps, max(1, args.warmup), True,
          {"workload": "fno_infer_128cube_w48_l4_m32x32x16", "params": model.count,
           "weights": args.fno_checkpoint or "random initialisation"},
          plain_cascade={"fields_per_s": 1e3 / t_plain, "ms": t_plain},
          judged_route={"fields_per_s": 1e3 / t_judged, "ms_per_bowl": t_judged, "fallback_rate": fb,
                        "threshold": 1e-2, "judge_rel_l2": [v["judge_rel_l2"] for v in verdicts],
                        "bowls": len(bowls)},
          plain_route={"fields_per_s": 1e3 / t_plain_route, "ms_per_bowl": t_plain_route},
          box_locality=locality)


def _box_locality(F, casc, bowls):
    """How much of p2 on the focal box comes from sources outside the box: p2 from the
    source restricted to the box's extent (zero elsewhere on the grid of harmonic 2)
    against p2 from the whole source, relative L2 on the box.  The surrogate sees p1 on
    the box only, so this part of p2 is outside what its input determines."""
    import math
    import torch
    from paper_2011_03009_gb300 import vp
    out = []
    for i, b in enumerate(bowls):
        casc.incident(b, i)
        casc.harmonic(b, 2)
        full = casc.to_box(b, 2).clone()
        g = F.harmonic_grids(b, casc.n, casc.medium)
        g2, g5 = g[2], g[5]
        src = torch.empty_like(casc.f[1])
        plan = casc.plans[2]
        plan.source_assemble([casc.f[1]], f_out=src)
        keep = torch.zeros_like(src)
        sl = []
        for a in range(3):
            lo = max(0, math.ceil((g5.origin[a] - g2.origin[a]) / g2.h - 1e-9))
            hi = min(g2.n[a] - 1, math.floor((g5.origin[a] + (g5.n[a] - 1) * g5.h - g2.origin[a]) / g2.h + 1e-9))
            sl.append(slice(lo, hi + 1))
        keep[sl[0], sl[1], sl[2]] = src[sl[0], sl[1], sl[2]]
        local = torch.empty_like(src)
        plan.apply(keep, local)
        local_box = torch.empty_like(full)
        vp.vp_restrict_to_nested_box(g2, local, g5, local_box)
        out.append(float(((local_box - full).abs().pow(2).sum() / full.abs().pow(2).sum()).sqrt().item()))
    return {"what": "rel-L2 on the box between p2 from the source inside the box only and p2 from the whole "
                    "source (grid of harmonic 2)", "per_bowl": out, "median": sorted(out)[len(out) // 2]}


def run_apply(args):
    """One plan on one grid (--grid, --harmonic, --zform, --staging, --layout; 1.1 MHz water, 227 um voxels):
    the kernel spectrum, then --warmup and --steps applications of a random field, each
    after an L2 flush; per-sweep CUDA-event times.  The small single-sweep cases of the
    ncu captures under profiles/ run through this workload."""
    import torch
    from paper_2011_03009_gb300 import synth, vp
    n = tuple(int(v) for v in args.grid.split(","))
    g = synth.Grid(n, (0.0, 0.0, 0.0), 2.27e-4)
    plan = vp.vp_plan(g, args.harmonic, 1.1e6, synth.WATER, zform=args.zform, staging=args.staging,
                      layout=args.layout)
    plan.kernel_fft()
    f = torch.randn(n, dtype=torch.complex64, device="cuda")
    u = torch.empty_like(f)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        plan.apply(f, u)
    torch.cuda.synchronize()
    plan.profile_enable(True)
    for _ in range(args.steps):
        flush.zero_()
        plan.apply(f, u)
    ms, cnt = plan.profile_read()
    if plan.check() != vp.VP_OK:
        raise RuntimeError("the plan's device status reports an expired wait or a refused buffer")
    inf = plan.info()
    by = sweep_bytes(tuple(inf.n), tuple(inf.m), args.harmonic, False)
    rows = [{"sweep": SWEEP_NAMES[i] if i else "x_forward", "ms": ms[i] / max(1, cnt[i]),
             "gbs": by[i] / (ms[i] / max(1, cnt[i]) * 1e-3) / 1e9} for i in range(5)]
    t = sum(r["ms"] for r in rows)
    _line(METRIC, g.voxels / (t * 1e-3), METRIC, t, args.steps, args.warmup, True,
          {"workload": f"apply_{'x'.join(map(str, n))}_h{args.harmonic}", "m": list(inf.m), "zform": args.zform,
           "staging": args.staging, "group_y": inf.group_y},
          sweeps=rows)


def run_nw(args):
    """Section 3's mesh refinement: p2 of the H131 transducer in liver on meshes of
    h = lambda / (2 n_w), n_w = 5..25 (odd), over one box around the focus, against
    n_w = 35; Deserno-spaced monopoles (4096)."""
    import numpy as np
    import torch
    from paper_2011_03009_gb300 import domain, synth
    bowl, med = synth.H131, synth.LIVER
    lam = synth.wavelength(med.c0, bowl.f0, 1)
    q = (12, 5, 5)  # box: 6 x 2.5 x 2.5 fundamental wavelengths
    x0 = bowl.l - 4 * lam
    n_ws = tuple(range(5, 26, 2))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = domain.nw_study(bowl, med, n_ws, 35, q, x0, n_points=4096)
    sec = time.perf_counter() - t0
    voxels = sum(int(np.prod(r["grid"])) for r in res["rows"]) + int(np.prod(res["ref_grid"]))
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import cascade, rayleigh
        # the oracle's p1 and p2 on the n_w = 5 mesh of the same box, from its own call
        g = domain.nw_grid(bowl, med, 5, q, x0)
        pts = synth.deserno_cap_points(bowl, 4096)
        t1 = time.perf_counter()
        p1 = rayleigh.incident_field(g, pts, bowl, med)
        cascade.harmonic(2, [p1], g.h, bowl.f0, med)
        dt = time.perf_counter() - t1
        cpu = {"value": g.voxels / dt, "unit": "voxels/s (p1 and p2)", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"FP64 oracle p1 (4096 points) and p2 on the n_w = 5 mesh {list(g.n)}, {dt:.2f} s"}
    _line("mesh-refinement study time", sec, "s", sec * 1e3, 1, 0, False,
          {"workload": "nw_study_p2_H131_liver", "q_half_wavelengths": list(q), "n_w": list(n_ws), "n_w_ref": 35,
           "points": res["points"], "voxels": voxels},
          rows=res["rows"], order=res["order"], order_coarse=res["order_coarse"], ref_grid=res["ref_grid"],
          ref_ms=res["ref_ms"], cpu_baseline=cpu)


def main():
    args = parse()
    world, rank, local = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), \
        int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    world, rank, local = dist_init(args)
    if args.workload == "batch64":
        run_batch(args, world, rank, local)
    elif args.workload in ("vie", "fullcascade", "q0", "nw", "restrict", "fno", "apply"):
        import torch
        torch.cuda.set_device(local)
        if rank == 0:
            {"vie": run_vie, "fullcascade": run_fullcascade, "q0": run_q0, "nw": run_nw,
             "restrict": run_restrict, "fno": run_fno, "apply": run_apply}[args.workload](args)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
