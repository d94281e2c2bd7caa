"""Named workloads and seeded generators (geometry + random draws only).

The workloads mirror the shapes of the paper's optical-diffraction-tomography
experiments (Section 6: spheres/ellipsoids immersed in a homogeneous medium,
plane waves on an illumination cone, complex noisy fields on a detector
plane), at the grid sizes used for parity and measurement.  Units: voxel
h = 1, background wavelength = 4 voxels, so k_b = pi/2 per voxel, except for
the workloads in physical units (the geometry of the paper's simulated 64^3
and real-data 96^3 experiments), where h is the voxel edge in metres and
k_b = 2 pi eta_m / lambda_vacuum.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Tuple

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic reconstruction problem.

    Fields follow the problem min_{x in C} (1/L) sum_l f_l(x) + lam * TV(x)
    of Eq. (1.2) with C = [box_lo, box_hi]^N and the subset split of Eq. (4.1).
    """

    name: str
    config_id: int
    n: int                      # grid edge; N = n^3 voxels
    model: str                  # "ls" (Lippmann-Schwinger) or "born"
    L: int                      # illuminations
    cone_deg: float             # half-angle of the illumination cone
    shape: str                  # "sphere" or "ellipsoid"
    n_objects: int
    size_range: Tuple[float, float]   # radius (sphere) / semi-axis (ellipsoid) range, voxels
    contrast_max: float
    background: Tuple[float, float]   # (amplitude, sigma in voxels); amplitude 0 = none
    snr_db: float
    batch: int                  # mini-batch size b; S = ceil(L / b)
    tv: str                     # "iso" or "aniso"
    lam: float
    box: Tuple[float, float]
    krylov_tol: float
    dual_iters: int
    outer_iters: int
    gamma: float = 0.8
    step: float = 1.0           # a_k (constant)
    margin: int = 2             # voxels kept free of objects at every face
    voxel_m: float = 0.0        # physical units: voxel edge (m); 0 = the lambda/4 voxel convention
    wavelength_m: float = 0.0   # vacuum wavelength (m)
    eta_m: float = 0.0          # refractive index of the medium
    grid: Tuple[int, ...] = ()  # (nz, ny, nx) of a box-shaped grid; () = the cube of edge n

    @property
    def S(self) -> int:
        return int(math.ceil(self.L / self.batch))

    @property
    def dims(self) -> Tuple[int, int, int]:
        """(nz, ny, nx) of the grid."""
        return tuple(self.grid) if self.grid else (self.n, self.n, self.n)

    @property
    def N(self) -> int:
        nz, ny, nx = self.dims
        return nz * ny * nx

    @property
    def M(self) -> int:
        """Detector values: the last z-slice, ny x nx."""
        _, ny, nx = self.dims
        return ny * nx

    @property
    def P(self) -> int:
        return 2 * self.n

    @property
    def kb(self) -> float:
        if self.voxel_m > 0:
            return 2.0 * math.pi * self.eta_m / self.wavelength_m
        return math.pi / 2.0

    @property
    def h(self) -> float:
        return self.voxel_m if self.voxel_m > 0 else 1.0

    def with_(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


WORKLOADS: Dict[str, Workload] = {
    # Plain MQNPM on the nonlinear model, small enough for the FP64 oracle.
    "ls32": Workload(
        name="ls32", config_id=1, n=32, model="ls", L=8, cone_deg=30.0,
        shape="sphere", n_objects=3, size_range=(3.0, 8.0), contrast_max=0.02,
        background=(0.0, 0.0), snr_db=40.0, batch=2, tv="iso", lam=1e-3,
        box=(0.0, 0.05), krylov_tol=1e-6, dual_iters=20, outer_iters=10),
    # First-Born (linear) model at 128^3.
    "born128": Workload(
        name="born128", config_id=2, n=128, model="born", L=60, cone_deg=45.0,
        shape="ellipsoid", n_objects=20, size_range=(128 / 32, 128 / 8),
        contrast_max=0.03, background=(0.005, 128 / 6), snr_db=30.0, batch=8,
        tv="aniso", lam=5e-4, box=(0.0, 0.05), krylov_tol=1e-6, dual_iters=20,
        outer_iters=10),
    # Nonlinear Lippmann-Schwinger at 128^3 (the measured configuration).
    "ls128": Workload(
        name="ls128", config_id=3, n=128, model="ls", L=60, cone_deg=45.0,
        shape="ellipsoid", n_objects=20, size_range=(128 / 32, 128 / 8),
        contrast_max=0.04, background=(0.005, 128 / 6), snr_db=30.0, batch=8,
        tv="iso", lam=1e-3, box=(0.0, 0.06), krylov_tol=1e-4, dual_iters=20,
        outer_iters=10),
    # The paper's simulated strongly scattering experiment in physical units
    # (Section 6): 64^3 voxels of 50 nm, vacuum wavelength 406 nm, medium index
    # 1.333, maximal index 1.43 (contrast (1.43/1.333)^2 - 1), 60 plane waves on
    # a 42-degree cone, S = 4, lambda = 1/64^3.
    "sim64": Workload(
        name="sim64", config_id=6, n=64, model="ls", L=60, cone_deg=42.0,
        shape="ellipsoid", n_objects=8, size_range=(3.0, 12.0),
        contrast_max=(1.43 / 1.333) ** 2 - 1, background=(0.0, 0.0), snr_db=30.0, batch=15,
        tv="iso", lam=1.0 / 64 ** 3, box=(0.0, 0.16), krylov_tol=1e-5, dual_iters=20,
        outer_iters=20, voxel_m=50e-9, wavelength_m=406e-9, eta_m=1.333),
    # Geometry of the paper's real-data experiment (a yeast cell, Section 6):
    # 96^3 voxels of 99 nm, 532 nm, medium 1.338, 60 plane waves on a 35-degree
    # cone, lambda = 2/96^3; the cell is a synthetic ellipsoid cluster (the
    # measured data are not available).
    "yeast96": Workload(
        name="yeast96", config_id=7, n=96, model="ls", L=60, cone_deg=35.0,
        shape="ellipsoid", n_objects=6, size_range=(4.0, 20.0),
        contrast_max=(1.40 / 1.338) ** 2 - 1, background=(0.0, 0.0), snr_db=30.0, batch=15,
        tv="iso", lam=2.0 / 96 ** 3, box=(0.0, 0.1), krylov_tol=1e-5, dual_iters=20,
        outer_iters=20, voxel_m=99e-9, wavelength_m=532e-9, eta_m=1.338),
    # Large strong-scattering case.
    "ls192": Workload(
        name="ls192", config_id=5, n=192, model="ls", L=120, cone_deg=60.0,
        shape="ellipsoid", n_objects=50, size_range=(192 / 32, 192 / 8),
        contrast_max=0.05, background=(0.005, 192 / 6), snr_db=30.0, batch=16,
        tv="iso", lam=2e-3, box=(0.0, 0.07), krylov_tol=1e-4, dual_iters=20,
        outer_iters=50),
}


def workload(name: str, **overrides) -> Workload:
    w = WORKLOADS[name]
    return w.with_(**overrides) if overrides else w


def _rng(w: Workload, offset: int) -> np.random.Generator:
    return np.random.default_rng(1000 * w.config_id + offset)


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation: QR of a Gaussian matrix with sign fix."""
    a = rng.standard_normal((3, 3))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def phantom(w: Workload) -> np.ndarray:
    """Ground-truth contrast x_true, float64 array of shape (nz, ny, nx) = (z, y, x).

    Objects are spheres or randomly rotated ellipsoids with contrast drawn
    uniformly in [0, contrast_max]; overlaps take the maximum.  Every object's
    bounding sphere stays ``margin`` voxels away from each face, so the last
    z-slice (the detector plane) is source-free.  An optional centred Gaussian
    background is tapered to zero inside the same margin.
    """
    rng = _rng(w, 0)
    nz, ny, nx = w.dims
    ext = np.array([nx, ny, nz], dtype=np.float64)           # extents in (x, y, z) order
    Z, Y, X = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    x = np.zeros((nz, ny, nx), dtype=np.float64)
    lo_s, hi_s = w.size_range
    for _ in range(w.n_objects):
        if w.shape == "sphere":
            axes = np.full(3, rng.uniform(lo_s, hi_s))
            rot = np.eye(3)
        else:
            axes = rng.uniform(lo_s, hi_s, size=3)
            rot = _random_rotation(rng)
        room = float(((ext - 1) - 2 * w.margin).min()) / 2.0
        if room <= 0:
            raise ValueError("grid too small for the margin")
        if axes.max() > room:                             # tiny grids: shrink to fit
            axes = axes * (room / axes.max())
        rmax = float(axes.max())
        lo_c = w.margin + rmax
        hi_c = (ext - 1) - w.margin - rmax
        centre = rng.uniform(lo_c, hi_c, size=3)          # (cx, cy, cz)
        value = rng.uniform(0.0, w.contrast_max)
        # only the bounding box of the bounding sphere can be inside
        lo = np.maximum(np.floor(centre - rmax).astype(int), 0)
        hi = np.minimum(np.ceil(centre + rmax).astype(int) + 1, ext.astype(int))
        box = (slice(lo[2], hi[2]), slice(lo[1], hi[1]), slice(lo[0], hi[0]))
        d = np.stack([X[box] - centre[0], Y[box] - centre[1], Z[box] - centre[2]], axis=-1)
        local = d @ rot                                   # coordinates in the body frame
        inside = np.sum((local / axes) ** 2, axis=-1) <= 1.0
        x[box] = np.where(inside, np.maximum(x[box], value), x[box])
    amp, sigma = w.background
    if amp > 0.0:
        mx, my, mz = (ext - 1) / 2.0
        g = amp * np.exp(-((X - mx) ** 2 + (Y - my) ** 2 + (Z - mz) ** 2) / (2.0 * sigma ** 2))

        def inner(m):
            v = np.ones(m, dtype=bool)
            v[: w.margin] = False
            v[m - w.margin:] = False
            return v

        mask = inner(nz)[:, None, None] & inner(ny)[None, :, None] & inner(nx)[None, None, :]
        x = np.maximum(x, np.where(mask, g, 0.0))
    return x


def illumination_dirs(w: Workload) -> np.ndarray:
    """Unit wave-vector directions (L, 3) as (kx, ky, kz) on the cone boundary.

    k_l = (sin t cos phi_l, sin t sin phi_l, cos t), phi_l = 2 pi l / L, t the
    cone half-angle (Section 6: tilted plane waves embedded in a cone).
    """
    t = math.radians(w.cone_deg)
    phi = 2.0 * math.pi * np.arange(w.L) / w.L
    return np.stack([math.sin(t) * np.cos(phi), math.sin(t) * np.sin(phi),
                     np.full(w.L, math.cos(t))], axis=1)


def subsets(w: Workload) -> List[np.ndarray]:
    """Non-overlapping interleaved subsets S_s = {l : l mod S = s} (0-based)."""
    S = w.S
    return [np.arange(s, w.L, S) for s in range(S)]


def noise_draws(w: Workload) -> np.ndarray:
    """Unit-variance circular complex Gaussian draws, shape (L, ny*nx)."""
    rng = _rng(w, 1)
    M = w.M
    re = rng.standard_normal((w.L, M))
    im = rng.standard_normal((w.L, M))
    return (re + 1j * im) / math.sqrt(2.0)


def strategy2_draws(w: Workload, count: int) -> np.ndarray:
    """Uniform subset indices for strategy II (count draws in [0, S))."""
    return _rng(w, 2).integers(0, w.S, size=count)


def power_start(w: Workload) -> np.ndarray:
    """Start vector of the power iteration that estimates alpha_s, shape (nz, ny, nx)."""
    return _rng(w, 3).standard_normal(w.dims)


def uneven_requests(seed: int = 4000, count: int = 16) -> List[Workload]:
    """Uneven multi-volume request mix: grids in {64,96,128,160}, L in {24,48,60},
    mini-batch 4..8, contrast in [0, 0.03], isotropic TV lam = 1e-3, box [0, 0.05]."""
    rng = np.random.default_rng(seed)
    out: List[Workload] = []
    for i in range(count):
        n = int(rng.choice([64, 96, 128, 160]))
        L = int(rng.choice([24, 48, 60]))
        b = int(rng.integers(4, 9))
        out.append(Workload(
            name=f"uneven{i}", config_id=4000 + i, n=n, model="ls", L=L,
            cone_deg=45.0, shape="ellipsoid", n_objects=20,
            size_range=(n / 32, n / 8), contrast_max=0.03,
            background=(0.005, n / 6), snr_db=30.0, batch=b, tv="iso",
            lam=1e-3, box=(0.0, 0.05), krylov_tol=1e-4, dual_iters=20,
            outer_iters=10))
    return out


def small(name: str = "ls32", n: Optional[int] = None, **kw) -> Workload:
    """A workload of the same family at a reduced grid (for parity tests)."""
    w = WORKLOADS[name]
    if n is not None:
        kw.setdefault("size_range", (max(1.0, w.size_range[0] * n / w.n),
                                     max(1.5, w.size_range[1] * n / w.n)))
        if w.background[0] > 0:
            kw.setdefault("background", (w.background[0], n / 6))
        kw["n"] = n
    return w.with_(**kw)
