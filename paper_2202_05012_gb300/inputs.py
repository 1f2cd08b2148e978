"""Seeded synthetic inputs for SUPA runs: model parameters and primaries.

This module holds plain data only -- parameter presets and seeded samplers of
primary particles -- and none of the method's arithmetic.  Both the CUDA path
and the CPU oracle consume what it produces; it imports neither of them.

Parameter presets follow the paper's statement of the model (Sec. 3 and
Algorithm 1 "Parameters", Table 2) with the readings listed in the design
notes: slice gap dz = 1, S = 3 slices per readout layer, constant
p_split = 0.5 and p_stop = 0.02, theta ~ U(pi/32, pi/16) and
eps ~ U(-theta/4, theta/4) (Table 2, SUPAv3-v5), an energy cut e_min and an
escape cut uz_min.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

THETA_FIXED, THETA_UNIFORM = 0, 1
EPS_ZERO, EPS_UNIFORM = 0, 1
SPLIT_MOMENTUM, SPLIT_LITERAL = 0, 1
ROI_FIXED, ROI_AXIS = 0, 1

# One primary particle: energy, impact point, incidence polar and azimuthal
# angle, and the index of its geometry in the launch (24 bytes, no padding).
PRIMARY_DTYPE = np.dtype(
    [("E", "<f4"), ("x0", "<f4"), ("y0", "<f4"), ("theta", "<f4"), ("phi", "<f4"), ("geom", "<u4")]
)


@dataclasses.dataclass
class Geometry:
    """Model and readout parameters of one detector (Algorithm 1 "Parameters")."""

    n_slices: int
    dz: float
    slice_to_layer: np.ndarray  # int32 [n_slices], -1 = dead slice
    n_layers: int
    p_stop: np.ndarray  # float64 [n_slices]
    p_split: np.ndarray  # float64 [n_slices]
    theta_mode: int = THETA_UNIFORM
    theta_lo: float = math.pi / 32
    theta_hi: float = math.pi / 16
    eps_mode: int = EPS_UNIFORM
    eps_frac: float = 0.25
    split_mode: int = SPLIT_MOMENTUM
    e_min: float = 0.05
    uz_min: float = 1e-3
    # downsampling grid (App. A.5): nx x ny cells of wx x wy per layer
    nx: int = 32
    ny: int = 32
    wx: float = 0.5
    wy: float = 0.5
    roi_mode: int = ROI_FIXED
    # lateral regions (Sec. 4.2): None, or a Regions record
    regions: "Regions | None" = None

    def layer_slice_range(self, layer: int) -> tuple[int, int]:
        ks = np.nonzero(self.slice_to_layer == layer)[0]
        return int(ks.min()), int(ks.max())


@dataclasses.dataclass
class Regions:
    """Concentric lateral regions around the z axis, each with its own
    meta-parameters (Sec. 4.2): region i holds r in [radius[i-1], radius[i])
    (radius[-1] = infinity); p_stop / p_split are [n_regions][n_slices]."""

    radius: np.ndarray    # float64 [n_regions - 1], increasing
    p_stop: np.ndarray    # float64 [n_regions][n_slices]
    p_split: np.ndarray   # float64 [n_regions][n_slices]
    theta_lo: np.ndarray  # float64 [n_regions]
    theta_hi: np.ndarray  # float64 [n_regions]
    eps_frac: np.ndarray  # float64 [n_regions]

    @property
    def n(self) -> int:
        return len(self.theta_lo)


def with_regions(g: Geometry, radius, p_stop, p_split, theta_lo, theta_hi, eps_frac) -> Geometry:
    """Give geometry g lateral regions; scalar p_stop / p_split entries are
    broadcast over the slices."""
    R = len(theta_lo)
    ps = np.array([np.full(g.n_slices, v, dtype=np.float64) if np.ndim(v) == 0 else np.asarray(v, np.float64)
                   for v in p_stop])
    pp = np.array([np.full(g.n_slices, v, dtype=np.float64) if np.ndim(v) == 0 else np.asarray(v, np.float64)
                   for v in p_split])
    g.regions = Regions(np.asarray(radius, np.float64), ps.reshape(R, g.n_slices), pp.reshape(R, g.n_slices),
                        np.asarray(theta_lo, np.float64), np.asarray(theta_hi, np.float64),
                        np.asarray(eps_frac, np.float64))
    return g


def supa_d(n_layers: int, slices_per_layer: int = 3, n_dead_front: int = 0, *, p_stop: float = 0.02,
           p_split: float = 0.5, e_min: float = 0.05, grid: int = 32, roi_mode: int = ROI_FIXED,
           roi_width: float = 16.0) -> Geometry:
    """The default layered detector: n_layers readout layers of S slices each."""
    n = n_dead_front + n_layers * slices_per_layer
    s2l = np.full(n, -1, dtype=np.int32)
    for k in range(n_dead_front, n):
        s2l[k] = (k - n_dead_front) // slices_per_layer
    w = roi_width / grid
    return Geometry(
        n_slices=n, dz=1.0, slice_to_layer=s2l, n_layers=n_layers,
        p_stop=np.full(n, p_stop, dtype=np.float64), p_split=np.full(n, p_split, dtype=np.float64),
        e_min=e_min, nx=grid, ny=grid, wx=w, wy=w, roi_mode=roi_mode,
    )


def supa_v1() -> Geometry:
    """SUPAv1 (Table 2; App. A.2.1): theta = pi/24, eps = 0, always split on
    slices 0..6, always stop from slice 7 on; one layer L0 = slices [5, 10]."""
    n = 11
    s2l = np.full(n, -1, dtype=np.int32)
    s2l[5:11] = 0
    p_split = np.where(np.arange(n) < 7, 1.0, 0.0)
    p_stop = np.where(np.arange(n) < 7, 0.0, 1.0)
    return Geometry(
        n_slices=n, dz=1.0, slice_to_layer=s2l, n_layers=1, p_stop=p_stop, p_split=p_split,
        theta_mode=THETA_FIXED, theta_lo=math.pi / 24, theta_hi=math.pi / 24, eps_mode=EPS_ZERO,
        eps_frac=0.0, e_min=0.0, nx=32, ny=32, wx=0.5, wy=0.5,
    )


def supa_calogan() -> Geometry:
    """A CaloGAN-like detector (Sec. 3.2, "Datasets and calorimeter
    structure"; the grid experiments): three readout layers in proportion to
    CaloGAN's 90, 347 and 43 mm, here 6, 22 and 3 slices of the SUPA-D model
    (the paper does not give its slice split), over a 16 dz square region
    with the cells of calogan_grids()."""
    s2l = np.array([0] * 6 + [1] * 22 + [2] * 3, dtype=np.int32)
    n = len(s2l)
    return Geometry(
        n_slices=n, dz=1.0, slice_to_layer=s2l, n_layers=3, p_stop=np.full(n, 0.02), p_split=np.full(n, 0.5),
        nx=12, ny=12, wx=16.0 / 12, wy=16.0 / 12, roi_mode=ROI_FIXED,
    )


def calogan_grids(width: float = 16.0) -> list[tuple[int, int, float, float]]:
    """Per-layer cells (nx, ny, wx, wy) of the CaloGAN-like detector at "1x":
    3 x 96, 12 x 12 and 12 x 6 (rows x columns: ny x nx) over one square
    region of side `width`."""
    return [(nx, ny, width / nx, width / ny) for (ny, nx) in ((3, 96), (12, 12), (12, 6))]


def primaries(n: int, seed: int, *, e_lo: float, e_hi: float, log_uniform: bool = False,
              theta_max_deg: float = 0.0, entry_halfwidth: float = 0.0, n_geoms: int = 1) -> np.ndarray:
    """Seeded primaries: energy U[e_lo, e_hi] (or log-uniform), polar angle
    U[0, theta_max], azimuth U[0, 2pi), entry point U[-h, h]^2, geometry
    index round-robin over n_geoms then shuffled."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = np.zeros(n, dtype=PRIMARY_DTYPE)
    if log_uniform:
        p["E"] = np.exp(rng.uniform(math.log(e_lo), math.log(e_hi), n)).astype(np.float32)
    else:
        p["E"] = rng.uniform(e_lo, e_hi, n).astype(np.float32)
    if theta_max_deg > 0:
        p["theta"] = rng.uniform(0.0, math.radians(theta_max_deg), n).astype(np.float32)
        p["phi"] = rng.uniform(0.0, 2 * math.pi, n).astype(np.float32)
    if entry_halfwidth > 0:
        p["x0"] = rng.uniform(-entry_halfwidth, entry_halfwidth, n).astype(np.float32)
        p["y0"] = rng.uniform(-entry_halfwidth, entry_halfwidth, n).astype(np.float32)
    if n_geoms > 1:
        g = (np.arange(n) % n_geoms).astype(np.uint32)
        rng.shuffle(g)
        p["geom"] = g
    return p


def mlp_init(seed: int, shapes=((256, 6), (256, 256), (256, 256), (90, 256))):
    """Seeded initial parameters of the surrogate network: weights
    U(-1/sqrt(fan_in), 1/sqrt(fan_in)), biases zero; float64 [(W, b)]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for n_out, n_in in shapes:
        a = 1.0 / math.sqrt(n_in)
        out.append((rng.uniform(-a, a, (n_out, n_in)), np.zeros(n_out)))
    return out


def subshower_primaries(n: int, seed: int, *, e_lo: float = 0.05, e_hi: float = 1.0, theta_max_deg: float = 45.0,
                        n_layers: int = 30, slices_per_layer: int = 3) -> tuple[np.ndarray, np.ndarray]:
    """Seeded sub-shower starts for surrogate training data: E log-uniform in
    [e_lo, e_hi], polar angle U[0, theta_max], azimuth U[0, 2pi), start layer
    U{0..n_layers-1} and start slice uniform within that layer.  Returns the
    primaries (geometry field = start slice << 16) and the start slices."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = np.zeros(n, dtype=PRIMARY_DTYPE)
    p["E"] = np.exp(rng.uniform(math.log(e_lo), math.log(e_hi), n)).astype(np.float32)
    p["theta"] = rng.uniform(0.0, math.radians(theta_max_deg), n).astype(np.float32)
    p["phi"] = rng.uniform(0.0, 2 * math.pi, n).astype(np.float32)
    layer = rng.integers(0, n_layers, n)
    k0 = (layer * slices_per_layer + rng.integers(0, slices_per_layer, n)).astype(np.uint32)
    p["geom"] = k0 << np.uint32(16)
    return p, k0


# ---- the workloads of the benchmark configurations ------------------------

def workload_plain10(n: int = 1000):
    """1,000 showers, seed 0: E ~ U[1,10], normal incidence at the origin,
    10 layers, 10 x 32 x 32 grid."""
    return supa_d(10, grid=32, roi_mode=ROI_FIXED), primaries(n, 0, e_lo=1.0, e_hi=10.0)


def workload_plain30(n: int = 1_000_000, seed: int = 1):
    """1,000,000 showers, seed 1: E ~ U[1,100], polar angle U[0,30 deg],
    entry within +-1 cell, 30 layers, 30 x 64 x 64 grid centred on the
    nominal shower axis (another seed: more showers of the same kind)."""
    g = supa_d(30, grid=64, roi_mode=ROI_AXIS)
    return g, primaries(n, seed, e_lo=1.0, e_hi=100.0, theta_max_deg=30.0, entry_halfwidth=g.wx)


def workload_mixed4(n: int = 4_000_000):
    """4,000,000 showers, seed 2: E log-uniform [1,1000], four geometries of
    10/20/30/50 layers mixed in one launch."""
    geoms = [supa_d(L, grid=64, roi_mode=ROI_AXIS) for L in (10, 20, 30, 50)]
    return geoms, primaries(n, 2, e_lo=1.0, e_hi=1000.0, log_uniform=True, n_geoms=4)


def workload_plain50(n: int = 10_000_000, seed: int = 4):
    """10,000,000 showers, seed 4: E log-uniform [10,1000], polar angle
    U[0,45 deg], 50 layers, 50 x 128 x 128 grid (another seed: more showers
    of the same kind)."""
    g = supa_d(50, grid=128, roi_mode=ROI_AXIS)
    return g, primaries(n, seed, e_lo=10.0, e_hi=1000.0, log_uniform=True, theta_max_deg=45.0)
