"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no arithmetic of the reconstruction method (no spherical
harmonics, no projection): it only draws geometries, phantom *fields*
(object masks, fibre directions, zonal amplitudes) and random test arrays.
Turning a phantom field into SH coefficients is done by each side on its own
(the FP64 oracle's ``zonal_to_sh`` for oracle inputs, the library's
``tt_zonal_to_sh`` kernel in the bench).

The synthetic workloads stand in for the paper's measured trabecular-bone
dataset (Table "performance_table": 247 projections of 65x55 pixels, 8
segments), which is not used here.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Setup:
    """Problem description in the paper's terms (Table "h5_format")."""
    shape: tuple            # (nx, ny, nz)
    nj: int
    nk: int
    ell_max: int
    inner_angle: np.ndarray  # alpha_s [rad]
    outer_angle: np.ndarray  # beta_s [rad]
    seg_start: np.ndarray    # phi_c,start [rad]
    seg_end: np.ndarray      # phi_c,end [rad]
    j_offset: np.ndarray
    k_offset: np.ndarray
    two_theta: float = 0.0
    a: float = 1.0
    b: float = 1.0

    @property
    def S(self) -> int:
        return int(self.inner_angle.size)

    @property
    def C(self) -> int:
        return int(self.seg_start.size)

    @property
    def K(self) -> int:
        return (self.ell_max + 1) * (self.ell_max + 2) // 2

    @property
    def volume_shape(self):
        return (*self.shape, self.K)

    @property
    def data_shape(self):
        return (self.S, self.nj, self.nk, self.C)

    def subset(self, proj):
        """The same setup restricted to the projections listed in proj."""
        proj = np.asarray(proj)
        return dataclasses.replace(
            self, inner_angle=self.inner_angle[proj].copy(),
            outer_angle=self.outer_angle[proj].copy(),
            j_offset=self.j_offset[proj].copy(), k_offset=self.k_offset[proj].copy())


def segments(n_seg: int, span: float = math.pi):
    """n_seg evenly spaced azimuthal bins covering [0, span)."""
    edges = np.arange(n_seg + 1, dtype=np.float64) * (span / n_seg)
    return edges[:-1].copy(), edges[1:].copy()


def _setup(n, j, ell_max, alphas_deg, betas_deg, n_seg, offsets=None):
    s0, s1 = segments(n_seg)
    S = len(alphas_deg)
    jo = np.zeros(S) if offsets is None else offsets[0]
    ko = np.zeros(S) if offsets is None else offsets[1]
    return Setup(shape=(n, n, n), nj=j, nk=j, ell_max=ell_max,
                 inner_angle=np.deg2rad(np.asarray(alphas_deg, dtype=np.float64)),
                 outer_angle=np.deg2rad(np.asarray(betas_deg, dtype=np.float64)),
                 seg_start=s0, seg_end=s1, j_offset=jo, k_offset=ko)


def geometry_angles(name: str):
    """(alpha_deg, beta_deg) lists of the five workloads."""
    if name == "cyl16":         # 15 rotations 12 deg apart x tilts {0, 30}
        al = [12.0 * i for t in (0.0, 30.0) for i in range(15)]
        be = [t for t in (0.0, 30.0) for _ in range(15)]
    elif name == "ell64":       # 20 rotations per tilt, 18 deg apart, offset 3 deg per tilt
        tilts = [0.0, 9.0, 18.0, 27.0, 36.0, 45.0]
        al = [18.0 * i + 3.0 * t for t in range(6) for i in range(20)]
        be = [tilts[t] for t in range(6) for _ in range(20)]
    elif name == "ell128":      # 24 rotations 15 deg apart x 10 tilts 0..45 step 5
        al = [15.0 * i for t in range(10) for i in range(24)]
        be = [5.0 * t for t in range(10) for _ in range(24)]
    elif name == "ply100":      # 45 rotations 8 deg apart x tilts {0,15,30,45}
        al = [8.0 * i for t in range(4) for i in range(45)]
        be = [15.0 * t for t in range(4) for _ in range(45)]
    elif name == "paper247":    # 19 rotations (360/19 deg apart, offset 1.5 deg per tilt) x 13 tilts 0..45 deg
        al = [360.0 / 19 * i + 1.5 * t for t in range(13) for i in range(19)]
        be = [3.75 * t for t in range(13) for _ in range(19)]
    else:
        raise KeyError(name)
    return al, be


def workload(name: str) -> Setup:
    """Geometry of the named workload.

    cyl16   16^3, l_max 2, 30 projections of 16x16, 8 segments (FP64 case)
    ell64   64^3, l_max 4, 120 projections of 64x64, 16 segments
    ell128  128^3, l_max 8, 240 projections of 128x128, 8 segments
    ply100  100^3, l_max 6, 180 projections of 100x100, 8 segments
    ell128c16  128^3, l_max 4, ell128 geometry with 16 segments
    paper247_l{2,4,8}  the paper's dataset shape: 247 projections of 65 (j,
               along the rotation axis y) x 55 (k) pixels x 8 segments; the
               volume, 55 x 65 x 55, and the 19 x 13 tilt series are guesses
               (the paper states neither)
    """
    if name.startswith("paper247_l"):
        ell = int(name[len("paper247_l"):])
        s0, s1 = segments(8)
        al, be = geometry_angles("paper247")
        S = len(al)
        return Setup(shape=(55, 65, 55), nj=65, nk=55, ell_max=ell,
                     inner_angle=np.deg2rad(np.asarray(al, dtype=np.float64)),
                     outer_angle=np.deg2rad(np.asarray(be, dtype=np.float64)),
                     seg_start=s0, seg_end=s1, j_offset=np.zeros(S), k_offset=np.zeros(S))
    if name == "cyl16":
        return _setup(16, 16, 2, *geometry_angles("cyl16"), 8)
    if name == "ell64":
        return _setup(64, 64, 4, *geometry_angles("ell64"), 16)
    if name == "ell128":
        return _setup(128, 128, 8, *geometry_angles("ell128"), 8)
    if name == "ply100":
        return _setup(100, 100, 6, *geometry_angles("ply100"), 8)
    if name == "ell128c16":
        return _setup(128, 128, 4, *geometry_angles("ell128"), 16)
    raise KeyError(name)


def small_setup(n=(6, 5, 7), nj=7, nk=6, ell_max=2, n_proj=5, n_seg=4, seed=0,
                offsets=True, two_theta=0.0, a=1.0, b=1.0) -> Setup:
    """A small random geometry (random rotations, tilts up to 60 deg, random
    sub-pixel offsets) for exhaustive parity and identity tests."""
    rng = np.random.default_rng(seed)
    al = rng.uniform(0.0, 2.0 * math.pi, n_proj)
    be = rng.uniform(-math.pi / 3, math.pi / 3, n_proj)
    s0, s1 = segments(n_seg)
    jo = rng.uniform(-0.5, 0.5, n_proj) if offsets else np.zeros(n_proj)
    ko = rng.uniform(-0.5, 0.5, n_proj) if offsets else np.zeros(n_proj)
    return Setup(shape=tuple(n), nj=nj, nk=nk, ell_max=ell_max, inner_angle=al,
                 outer_angle=be, seg_start=s0, seg_end=s1, j_offset=jo,
                 k_offset=ko, two_theta=two_theta, a=a, b=b)


# ------------------------------------------------------------- phantom fields


@dataclasses.dataclass
class PhantomField:
    """Per-voxel zonal model: inside-mask, fibre axis n and amplitudes a_l."""
    mask: np.ndarray        # [nx, ny, nz] bool
    dirs: np.ndarray        # [nx, ny, nz, 3] unit vectors (arbitrary outside)
    amps: np.ndarray        # [nx, ny, nz, L/2+1], zero outside the mask


def _centres(shape):
    ax = [np.arange(n, dtype=np.float64) for n in shape]
    return np.stack(np.meshgrid(*ax, indexing="ij"), axis=-1)


def _normalize(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def cylinder_phantom(n: int = 16, ell_max: int = 2) -> PhantomField:
    """Cylinder about +y (the rotation axis), radius 0.35 n, full length; the
    fibre axis lies in the x-z plane at angle pi*y/n; a0 = 1, a2 = 0.5."""
    X = _centres((n, n, n))
    h = 0.5 * (n - 1)
    rr = np.hypot(X[..., 0] - h, X[..., 2] - h)
    mask = rr <= 0.35 * n
    ang = math.pi * X[..., 1] / n
    dirs = np.stack([np.cos(ang), np.zeros_like(ang), np.sin(ang)], axis=-1)
    amps = np.zeros((n, n, n, ell_max // 2 + 1))
    amps[..., 0] = 1.0
    if ell_max >= 2:
        amps[..., 1] = 0.5
    amps[~mask] = 0.0
    return PhantomField(mask, dirs, amps)


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def ellipsoid_phantom(n: int, ell_max: int, n_ell: int, seed: int) -> PhantomField:
    """Random ellipsoids (centres U(0.25n, 0.75n)^3, semi-axes U(0.08n,
    0.25n), random orientation), each with fibre field n(x) = normalize(n0 +
    G (x - x0)/n), n0 uniform on the sphere, G ~ U(-1,1)^{3x3}, and zonal
    amplitudes a0~U(.5,1), a2~U(.2,.6), a4~U(0,.2), a6,a8~U(0,.1).  Later
    ellipsoids overwrite earlier ones; zero outside."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    X = _centres(shape)
    nl = ell_max // 2 + 1
    mask = np.zeros(shape, dtype=bool)
    dirs = np.zeros(shape + (3,))
    dirs[..., 2] = 1.0
    amps = np.zeros(shape + (nl,))
    lo = [0.5, 0.2, 0.0, 0.0, 0.0]
    hi = [1.0, 0.6, 0.2, 0.1, 0.1]
    for _ in range(n_ell):
        x0 = rng.uniform(0.25 * n, 0.75 * n, 3)
        semi = rng.uniform(0.08 * n, 0.25 * n, 3)
        Rot = _random_rotation(rng)
        n0 = _normalize(rng.normal(size=3))
        G = rng.uniform(-1.0, 1.0, (3, 3))
        a_l = np.array([rng.uniform(lo[min(i, 4)], hi[min(i, 4)]) for i in range(nl)])
        rel = X - x0
        loc = rel @ Rot            # coordinates in the ellipsoid frame
        inside = np.sum((loc / semi) ** 2, axis=-1) <= 1.0
        fib = _normalize(n0 + (rel / n) @ G.T)
        mask |= inside
        dirs[inside] = fib[inside]
        amps[inside] = a_l
    return PhantomField(mask, dirs, amps)


def plywood_phantom(n: int, ell_max: int, seed: int, n_layers: int = 10) -> PhantomField:
    """A block (central 80% of each axis) of n_layers layers stacked along z;
    in-plane fibres along x or y, alternating per layer, each voxel jittered by
    U(-5, 5) deg about z.  a0=1, a2=.5, a4=.2, a6=.1."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    X = _centres(shape)
    lo, hi = 0.1 * n, 0.9 * n
    mask = np.all((X >= lo) & (X < hi), axis=-1)
    layer = np.floor((X[..., 2] - lo) / ((hi - lo) / n_layers)).astype(int)
    base = np.where(layer % 2 == 0, 0.0, 0.5 * math.pi)
    jit = np.deg2rad(rng.uniform(-5.0, 5.0, shape))
    ang = base + jit
    dirs = np.stack([np.cos(ang), np.sin(ang), np.zeros_like(ang)], axis=-1)
    nl = ell_max // 2 + 1
    vals = [1.0, 0.5, 0.2, 0.1, 0.05]
    amps = np.zeros(shape + (nl,))
    for i in range(nl):
        amps[..., i] = vals[min(i, 4)]
    amps[~mask] = 0.0
    return PhantomField(mask, dirs, amps)


def phantom(name: str, seed: int | None = None) -> PhantomField:
    if name == "cyl16":
        return cylinder_phantom(16, 2)
    if name == "ell64":
        return ellipsoid_phantom(64, 4, 6, 1 if seed is None else seed)
    if name == "ell128":
        return ellipsoid_phantom(128, 8, 12, 2 if seed is None else seed)
    if name == "ply100":
        return plywood_phantom(100, 6, 3 if seed is None else seed)
    if name == "ell128c16":
        return ellipsoid_phantom(128, 4, 12, 2 if seed is None else seed)
    raise KeyError(name)


# --------------------------------------------------------------- test arrays


def random_volume(setup: Setup, seed: int, dtype=np.float64) -> np.ndarray:
    return np.random.default_rng(seed).normal(size=setup.volume_shape).astype(dtype)


def random_data(setup: Setup, seed: int, dtype=np.float64) -> np.ndarray:
    return np.random.default_rng(seed).normal(size=setup.data_shape).astype(dtype)


def random_weights(setup: Setup, seed: int, zero_frac: float = 0.1, dtype=np.float64):
    """W ~ U(0,1) with a fraction zero_frac set to exactly 0."""
    rng = np.random.default_rng(seed)
    W = rng.uniform(0.0, 1.0, setup.data_shape)
    W[rng.uniform(size=setup.data_shape) < zero_frac] = 0.0
    return W.astype(dtype)


def gaussian_noise(clean: np.ndarray, rel_sigma: float, seed: int) -> np.ndarray:
    """clean + N(0, (rel_sigma * mean|clean|)^2)."""
    rng = np.random.default_rng(seed)
    return clean + rng.normal(scale=rel_sigma * float(np.mean(np.abs(clean))), size=clean.shape)


def poisson_counts(clean: np.ndarray, mean_counts: float, seed: int) -> np.ndarray:
    """Scale clean data to the given mean and draw Poisson counts."""
    rng = np.random.default_rng(seed)
    scale = mean_counts / float(np.mean(clean))
    return rng.poisson(np.maximum(clean, 0.0) * scale).astype(np.float64) / scale
