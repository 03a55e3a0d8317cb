"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds the workload recipes (medium, bowl transducer, voxel grids) and
seeded random draws (bowl surface points, random complex fields, per-instance
parameter draws).  It holds none of the method's arithmetic: no Green's function,
no wavenumber, no source coefficient, no interpolation.  Both sides of every
parity check compute those themselves from the numbers produced here.

Geometry conventions (Section 2.3, Eq. 3.13): the bowl apex is at the origin, the
transducer axis is +x and the geometric focus is at (l, 0, 0).  A grid is given by
its voxel count per axis n = (nx, ny, nz) (C order, z fastest), the centre of voxel
(0, 0, 0) and the voxel side h; voxel (i, j, k) has centre origin + (i, j, k) * h.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np


@dataclasses.dataclass(frozen=True)
class Medium:
    """Homogeneous propagation medium.

    alpha0 is the power-law attenuation prefactor in dB/m/MHz^eta, eta the exponent
    (Section 2, Table 2).  The workloads use water with c0 = 1500 m/s.
    """

    c0: float = 1500.0
    rho0: float = 1000.0
    beta: float = 3.5
    alpha0: float = 0.22
    eta: float = 2.0


WATER = Medium()
# soft-tissue-like inclusion for the inhomogeneous-medium equations (Section 7)
TISSUE = Medium(c0=1540.0, rho0=1000.0, beta=4.5, alpha0=5.0, eta=1.1)
# liver as listed in Table 2 (alpha0 in dB/m/MHz^eta under the same units reading)
LIVER = Medium(c0=1590.0, rho0=1060.0, beta=4.4, alpha0=90.0, eta=1.1)


@dataclasses.dataclass(frozen=True)
class Bowl:
    """Single-element spherical bowl: focal length l, aperture radius R (Table 1)."""

    l: float
    R: float
    f0: float
    p0: float  # surface pressure amplitude (Pa)


@dataclasses.dataclass(frozen=True)
class Grid:
    n: Tuple[int, int, int]
    origin: Tuple[float, float, float]
    h: float

    @property
    def voxels(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])

    def axis(self, a: int) -> np.ndarray:
        return self.origin[a] + self.h * np.arange(self.n[a], dtype=np.float64)


# Table 1's transducers (f0, focal length l, outer radius R); the surface pressure is
# this module's choice (the paper prescribes a radiated power instead)
H101 = Bowl(l=0.0632, R=0.032, f0=1.1e6, p0=1.0e6)
H131 = Bowl(l=0.035, R=0.0165, f0=1.1e6, p0=1.0e6)


def wavelength(c0: float, f0: float, n: int) -> float:
    """Wavelength of harmonic n: c0 / (n f0)."""
    return c0 / (n * f0)


def centred_grid(n: Sequence[int], h: float, centre: Sequence[float]) -> Grid:
    """Grid of n voxels per axis with spacing h whose box is centred on `centre`."""
    n = tuple(int(v) for v in n)
    origin = tuple(float(centre[a]) - 0.5 * (n[a] - 1) * h for a in range(3))
    return Grid(n, origin, float(h))


def focus_grid(bowl: Bowl, n: Sequence[int], harmonic: int, medium: Medium = WATER,
               ppw: int = 6) -> Grid:
    """Grid centred on the focus with spacing lambda_n / ppw (6 voxels per wavelength)."""
    h = wavelength(medium.c0, bowl.f0, harmonic) / ppw
    return centred_grid(n, h, (bowl.l, 0.0, 0.0))


def sample_bowl_points(bowl: Bowl, n_points: int, seed: int) -> np.ndarray:
    """n_points seeded points uniform in area on the spherical cap of the bowl.

    The cap is the part of the sphere of radius l centred on the focus whose polar
    angle (seen from the focus, measured from the -x direction) is at most
    asin(R / l).  Uniform in area means cos(theta) ~ U[cos(theta_max), 1] and
    phi ~ U[0, 2 pi).  Returns an (n_points, 3) float64 array.
    """
    rng = np.random.default_rng(seed)
    ct_max = math.sqrt(max(0.0, 1.0 - (bowl.R / bowl.l) ** 2))
    ct = rng.uniform(ct_max, 1.0, size=n_points)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=n_points)
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    pts = np.empty((n_points, 3), dtype=np.float64)
    pts[:, 0] = bowl.l * (1.0 - ct)
    pts[:, 1] = bowl.l * st * np.cos(phi)
    pts[:, 2] = bowl.l * st * np.sin(phi)
    return pts


def deserno_cap_points(bowl: Bowl, n_target: int) -> np.ndarray:
    """About n_target evenly spaced points on the bowl's spherical cap (Section 3 places
    the monopoles after Deserno's construction for the sphere).

    On the unit sphere each point is to carry the area a = 2 pi (1 - cos theta_max) /
    n_target, d = sqrt(a).  The polar range [0, theta_max] (seen from the focus,
    measured from -x) is cut into M_theta = round(theta_max / d) rings of width
    d_theta = theta_max / M_theta; ring m sits at theta_m = (m + 1/2) d_theta and holds
    M_phi = round(2 pi sin(theta_m) / d_phi) points at phi = 2 pi k / M_phi, with
    d_phi = a / d_theta.  Deterministic; returns an (n, 3) float64 array, n close to
    n_target.
    """
    th_max = math.asin(min(1.0, bowl.R / bowl.l))
    a = 2.0 * math.pi * (1.0 - math.cos(th_max)) / n_target
    d = math.sqrt(a)
    m_th = max(1, int(round(th_max / d)))
    d_th = th_max / m_th
    d_ph = a / d_th
    rings = []
    for m in range(m_th):
        th = (m + 0.5) * d_th
        m_ph = max(1, int(round(2.0 * math.pi * math.sin(th) / d_ph)))
        ph = 2.0 * math.pi * np.arange(m_ph, dtype=np.float64) / m_ph
        ring = np.empty((m_ph, 3), dtype=np.float64)
        ring[:, 0] = bowl.l * (1.0 - math.cos(th))
        ring[:, 1] = bowl.l * math.sin(th) * np.cos(ph)
        ring[:, 2] = bowl.l * math.sin(th) * np.sin(ph)
        rings.append(ring)
    return np.concatenate(rings, axis=0)


def random_field(n: Sequence[int], seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded complex128 field with standard normal real and imaginary parts."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(v) for v in n)
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def smooth_blob_field(grid: Grid, centre: Sequence[float], width: float, k: float,
                      amp: float = 1.0) -> np.ndarray:
    """Smooth focused-beam-like test field: Gaussian envelope times an axial plane wave."""
    x = grid.axis(0)[:, None, None]
    y = grid.axis(1)[None, :, None]
    z = grid.axis(2)[None, None, :]
    r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2
    return amp * np.exp(-r2 / (width * width)) * np.exp(1j * k * (x - centre[0]))


def sparse_block_source(n: Sequence[int], side: int, seed: int):
    """Seeded source that is non-zero on few voxels of a large grid: a cube of side^3
    voxels (clipped to the grid) at a seeded position with standard normal complex
    values, plus the grid's two opposite corner voxels (the longest offsets the
    embedding holds).  Returns (idx (S, 3) int64, values (S,) complex128)."""
    rng = np.random.default_rng(seed)
    n = tuple(int(v) for v in n)
    lo = [int(rng.integers(0, max(1, n[a] - side + 1))) for a in range(3)]
    ax = [np.arange(lo[a], min(n[a], lo[a] + side)) for a in range(3)]
    block = np.stack(np.meshgrid(*ax, indexing="ij"), axis=-1).reshape(-1, 3)
    corners = np.array([[0, 0, 0], [n[0] - 1, n[1] - 1, n[2] - 1]])
    idx = np.unique(np.concatenate([block, corners]), axis=0).astype(np.int64)
    vals = rng.standard_normal(len(idx)) + 1j * rng.standard_normal(len(idx))
    return idx, vals


def sample_targets(n: Sequence[int], idx: np.ndarray, count: int, seed: int) -> np.ndarray:
    """Seeded target voxels: `count` uniform over the grid, the 8 corners, and up to 256
    voxels among and next to the given source voxels.  (T, 3) int64."""
    rng = np.random.default_rng(seed)
    n = tuple(int(v) for v in n)
    uni = np.stack([rng.integers(0, n[a], size=count) for a in range(3)], axis=1)
    corners = np.array([(x, y, z) for x in (0, n[0] - 1) for y in (0, n[1] - 1) for z in (0, n[2] - 1)])
    pick = idx[rng.choice(len(idx), size=min(256, len(idx)), replace=False)]
    near = np.clip(pick + rng.integers(-2, 3, size=pick.shape), 0, np.array(n) - 1)
    return np.concatenate([uni, corners, near]).astype(np.int64)


# --------------------------------------------------------------------------------------
# Workload recipes (the synthetic bowl-transducer configurations).
# --------------------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class HarmonicStep:
    """One harmonic of a nested-mesh run: its grid and where its inputs come from."""

    harmonic: int
    grid: Grid


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    bowl: Bowl
    medium: Medium
    n_points: int
    seed: int
    steps: Tuple[HarmonicStep, ...]
    # grid on which the incident field p1 is evaluated by the Rayleigh sum
    p1_grid: Grid
    # apply the harmonic-1 operator V_{k1}[p1] on this grid (None: not part of the run)
    v1_grid: Grid | None = None

    @property
    def voxels_per_step(self) -> int:
        v = sum(s.grid.voxels for s in self.steps)
        if self.v1_grid is not None:
            v += self.v1_grid.voxels
        return v


def workload_small_p2() -> Workload:
    """Plain 2nd harmonic on 32^3 (bowl R = 1 cm, l = 2 cm, 1 MHz, 0.5 MPa, 2000 points)."""
    bowl = Bowl(l=0.02, R=0.01, f0=1.0e6, p0=0.5e6)
    g2 = focus_grid(bowl, (32, 32, 32), 2)
    return Workload("p2_32cube_R1cm_l2cm_1MHz", bowl, WATER, 2000, 1,
                    (HarmonicStep(2, g2),), p1_grid=g2)


def workload_nested_h123() -> Workload:
    """Harmonics 1-3 on nested 128^3 / 192^3 / 256^3 focal grids (R = 3 cm, l = 6 cm, 1.1 MHz).

    Harmonic 1: V_{k1}[p1] on the 128^3 grid.  Harmonic 2: p1 evaluated on the
    192^3 grid, f2 from p1^2.  Harmonic 3: p1 and p2 restricted from the 192^3
    grid onto the 256^3 grid, f3 from p1 p2.
    """
    bowl = Bowl(l=0.06, R=0.03, f0=1.1e6, p0=1.0e6)
    g1 = focus_grid(bowl, (128, 128, 128), 1)
    g2 = focus_grid(bowl, (192, 192, 192), 2)
    g3 = focus_grid(bowl, (256, 256, 256), 3)
    return Workload("h1-3_nested_128-192-256cube_R3cm_l6cm_1.1MHz", bowl, WATER, 4096, 2,
                    (HarmonicStep(2, g2), HarmonicStep(3, g3)), p1_grid=g2, v1_grid=g1)


def workload_nested_h1to5() -> Workload:
    """Full 5-harmonic nested run (R = 7.5 cm, l = 15 cm, 1.1 MHz, 2 MPa).

    Fundamental grid 600 x 600 x 640 at lambda_1/6 following the D2 box convention
    (x from just past the rim plane); harmonics 2-5 on 320^3, 384^3, 432^3, 512^3
    focal boxes at lambda_n/6.
    """
    bowl = Bowl(l=0.15, R=0.075, f0=1.1e6, p0=2.0e6)
    h1 = wavelength(WATER.c0, bowl.f0, 1) / 6
    rim = bowl.l - math.sqrt(bowl.l ** 2 - bowl.R ** 2)
    n1 = (600, 600, 640)
    g1 = Grid(n1, (rim + 1.0e-4 + 0.5 * h1, -0.5 * (n1[1] - 1) * h1, -0.5 * (n1[2] - 1) * h1), h1)
    sizes = {2: 320, 3: 384, 4: 432, 5: 512}
    steps = tuple(HarmonicStep(n, focus_grid(bowl, (s, s, s), n)) for n, s in sizes.items())
    return Workload("h1-5_nested_600x600x640_320-512cube_R7.5cm_l15cm", bowl, WATER, 4096, 3,
                    steps, p1_grid=steps[0].grid, v1_grid=g1)


WORKLOADS = {
    "small": workload_small_p2,
    "nested3": workload_nested_h123,
    "nested5": workload_nested_h1to5,
}


@dataclasses.dataclass(frozen=True)
class BatchInstance:
    bowl: Bowl
    grids: Tuple[Grid, ...]  # harmonics 1..3


def draw_batch_instances(count: int, seed: int, nmin: int = 96, nmax: int = 256,
                         harmonics: int = 3) -> List[BatchInstance]:
    """Seeded transducer draws for the batched workload.

    Focal length U[8, 15] cm, aperture radius U[3, 7.5] cm (kept below 0.9 l),
    f0 U[0.8, 1.5] MHz, p0 U[0.5, 3] MPa.  Each harmonic n gets a cubic focal grid
    at lambda_n / 6 whose voxel count is drawn from [nmin, nmax], redrawn so that
    the physical box never grows with n (nested boxes).
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        l = rng.uniform(0.08, 0.15)
        R = min(rng.uniform(0.03, 0.075), 0.9 * l)
        f0 = rng.uniform(0.8e6, 1.5e6)
        p0 = rng.uniform(0.5e6, 3.0e6)
        bowl = Bowl(l=float(l), R=float(R), f0=float(f0), p0=float(p0))
        grids = []
        extent = math.inf
        for n in range(1, harmonics + 1):
            h = wavelength(WATER.c0, f0, n) / 6
            hi = nmax if math.isinf(extent) else min(nmax, int(math.floor(extent / h)))
            lo = min(nmin, hi)
            nv = int(rng.integers(lo, hi + 1))
            extent = nv * h
            grids.append(focus_grid(bowl, (nv, nv, nv), n))
        out.append(BatchInstance(bowl, tuple(grids)))
    return out
