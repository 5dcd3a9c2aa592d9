"""Seeded synthetic chaff clouds, incidence lists and observation lists.

Every workload of the solver is a cloud of straight thin wires ("chaffs", Sec. II-A): a centre,
a unit direction, a length, a radius and a segment count per wire.  The statistics below restate
the workload descriptions the method is exercised on (uniform or Gaussian-clustered centres,
directions uniform on the sphere, lengths uniform in an interval or drawn from a few fixed values,
radius 1e-3 wavelength, wavelength 1 so k = 2*pi).  The paper's own clouds (uniform in a sphere
at a given density, Sec. III and IV) are of the same kind.

Only NumPy's PCG64 generator is used, so a seed gives the same cloud on every machine.
Nothing here evaluates the method: no kernel, no quadrature, no solve.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

WAVELENGTH = 1.0
K0 = 2.0 * math.pi / WAVELENGTH
RADIUS = 1e-3 * WAVELENGTH
SEG_MAX = 0.08 * WAVELENGTH


@dataclasses.dataclass
class Cloud:
    """A wire cloud in structure-of-arrays form (all float64 except ``nseg``)."""

    centres: np.ndarray  # (nw, 3)
    dirs: np.ndarray  # (nw, 3), unit vectors
    lengths: np.ndarray  # (nw,)
    radii: np.ndarray  # (nw,)
    nseg: np.ndarray  # (nw,) int32, segments per wire (unknowns per wire = nseg - 1)
    name: str = ""

    @property
    def nw(self) -> int:
        return int(self.centres.shape[0])

    @property
    def n_unknowns(self) -> int:
        return int(np.sum(self.nseg.astype(np.int64) - 1))

    def subset(self, idx) -> "Cloud":
        idx = np.asarray(idx)
        return Cloud(self.centres[idx].copy(), self.dirs[idx].copy(), self.lengths[idx].copy(),
                     self.radii[idx].copy(), self.nseg[idx].copy(), self.name + "[subset]")

    def check(self) -> None:
        nw = self.nw
        assert self.centres.shape == (nw, 3) and self.dirs.shape == (nw, 3)
        assert self.lengths.shape == (nw,) and self.radii.shape == (nw,) and self.nseg.shape == (nw,)
        assert self.nseg.dtype == np.int32


def _unit_directions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Directions uniform on the unit sphere: normalised standard-normal triples."""
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def _nseg_for(lengths: np.ndarray, seg_max: float = SEG_MAX) -> np.ndarray:
    """Segment count keeping every segment at most ``seg_max`` long (ceil(L / seg_max))."""
    return np.ceil(lengths / seg_max).astype(np.int32)


def _make(centres, dirs, lengths, nseg, name, radius=RADIUS) -> Cloud:
    c = Cloud(np.ascontiguousarray(centres, dtype=np.float64),
              np.ascontiguousarray(dirs, dtype=np.float64),
              np.ascontiguousarray(lengths, dtype=np.float64),
              np.full(len(lengths), radius, dtype=np.float64),
              np.ascontiguousarray(nseg, dtype=np.int32), name)
    c.check()
    return c


def cloud_small(seed: int = 0) -> Cloud:
    """200 wires of length 0.5, 8 segments each (N = 1400), centres uniform in a 20-wavelength cube."""
    rng = np.random.default_rng(seed)
    nw = 200
    centres = rng.uniform(-10.0, 10.0, size=(nw, 3))
    dirs = _unit_directions(rng, nw)
    lengths = np.full(nw, 0.5)
    return _make(centres, dirs, lengths, np.full(nw, 8, dtype=np.int32), "small")


def cloud_mid(seed: int = 1, nw: int = 10_000) -> Cloud:
    """10,000 wires, lengths U[0.3, 0.6], centres 3-D Gaussian with sigma = 30 wavelengths."""
    rng = np.random.default_rng(seed)
    centres = rng.normal(0.0, 30.0, size=(nw, 3))
    dirs = _unit_directions(rng, nw)
    lengths = rng.uniform(0.3, 0.6, size=nw)
    return _make(centres, dirs, lengths, _nseg_for(lengths), "mid")


def batching_sizes(n_snap: int = 64, seed: int = 999, lo: int = 2_000, hi: int = 50_000) -> np.ndarray:
    """Snapshot wire counts, log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_snap))).astype(np.int64)


def cloud_batching_snapshot(i: int, nw: int | None = None, density: float = 0.005) -> Cloud:
    """Snapshot i of the batching workload: mid-config wire statistics, centres uniform in a cube
    whose side gives ``density`` wires per cubic wavelength."""
    if nw is None:
        nw = int(batching_sizes()[i])
    rng = np.random.default_rng(1000 + i)
    side = (nw / density) ** (1.0 / 3.0)
    centres = rng.uniform(-side / 2, side / 2, size=(nw, 3))
    dirs = _unit_directions(rng, nw)
    lengths = rng.uniform(0.3, 0.6, size=nw)
    return _make(centres, dirs, lengths, _nseg_for(lengths), f"batching[{i}]")


def cloud_precision(seed: int = 3, nw: int = 200_000) -> Cloud:
    """200,000 wires in a 350-wavelength cube, lengths 0.35/0.45/0.5 in equal shares."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-175.0, 175.0, size=(nw, 3))
    dirs = _unit_directions(rng, nw)
    lengths = np.array([0.35, 0.45, 0.5])[rng.permutation(np.arange(nw) % 3)]
    return _make(centres, dirs, lengths, _nseg_for(lengths), "precision")


def cloud_learned(seed: int = 4, nw: int = 1_000_000, n_clusters: int = 8, sigma: float = 40.0) -> Cloud:
    """1,000,000 wires in 8 Gaussian clusters (sigma 40) whose centres are uniform in [-180, 180]^3.
    A smaller ``nw`` with sigma = 40 (nw / 1e6)^(1/3) keeps the wire density of the full cloud."""
    rng = np.random.default_rng(seed)
    cc = rng.uniform(-180.0, 180.0, size=(n_clusters, 3))
    which = rng.integers(0, n_clusters, size=nw)
    centres = cc[which] + rng.normal(0.0, sigma, size=(nw, 3))
    dirs = _unit_directions(rng, nw)
    lengths = rng.uniform(0.3, 0.6, size=nw)
    return _make(centres, dirs, lengths, _nseg_for(lengths), "learned")


def cloud_uniform_cube(nw: int, side: float, seed: int, length=(0.3, 0.6), nseg: int | None = None,
                       radius: float = RADIUS) -> Cloud:
    """Small test clouds: centres uniform in a cube, random directions.  ``length`` is a float or an
    interval; ``nseg`` fixes the segment count, else the 0.08-wavelength rule applies."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-side / 2, side / 2, size=(nw, 3))
    dirs = _unit_directions(rng, nw)
    if np.isscalar(length):
        lengths = np.full(nw, float(length))
    else:
        lengths = rng.uniform(length[0], length[1], size=nw)
    ns = np.full(nw, nseg, dtype=np.int32) if nseg is not None else _nseg_for(lengths)
    return _make(centres, dirs, lengths, ns, f"cube{nw}", radius)


def cloud_single(length: float = 0.5, nseg: int = 16, direction=(0.0, 0.0, 1.0), centre=(0.0, 0.0, 0.0),
                 radius: float = RADIUS) -> Cloud:
    """One straight wire (a dipole)."""
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return _make(np.asarray([centre], dtype=np.float64), d[None, :], np.array([length]),
                 np.array([nseg], dtype=np.int32), "single", radius)


def incidences_single_minus_z() -> np.ndarray:
    """One plane wave travelling along -z, theta-polarised: arrival direction +z (theta=0, phi=0),
    polarisation angle 0.  Rows are (theta, phi, psi) in radians."""
    return np.array([[0.0, 0.0, 0.0]])


def incidences_monostatic(n: int) -> np.ndarray:
    """n arrival directions theta = 0..180 degrees evenly spaced in the phi = 0 plane, theta-polarised
    (181 -> 1 degree, 91 -> 2 degrees, 37 -> 5 degrees)."""
    th = np.linspace(0.0, math.pi, n)
    return np.stack([th, np.zeros(n), np.zeros(n)], axis=1)


def observations_phi_cut(n: int) -> np.ndarray:
    """n observation directions in the theta = 90 degree plane, phi = 0 .. 360 * (n-1)/n degrees.
    Rows are (theta, phi) in radians."""
    ph = np.arange(n) * (2.0 * math.pi / n)
    return np.stack([np.full(n, math.pi / 2), ph], axis=1)


# Named workloads: cloud factory, coupling radius, incidences, observations, solver settings.
CONFIGS = {
    "small": dict(cloud=cloud_small, k=K0, r_c=3.0, inc=incidences_single_minus_z,
                  obs=lambda: observations_phi_cut(360), tol=1e-6, restart=50),
    "mid": dict(cloud=cloud_mid, k=K0, r_c=3.0, inc=incidences_single_minus_z,
                obs=lambda: observations_phi_cut(720), tol=1e-6, restart=50),
    "batching": dict(cloud=cloud_batching_snapshot, k=K0, r_c=3.0, inc=lambda: incidences_monostatic(181),
                     obs=None, tol=1e-6, restart=50),
    "precision": dict(cloud=cloud_precision, k=K0, r_c=4.0, inc=lambda: incidences_monostatic(91),
                      obs=None, tol=1e-6, restart=50),
    "learned": dict(cloud=cloud_learned, k=K0, r_c=3.0, inc=lambda: incidences_monostatic(37),
                    obs=None, tol=1e-6, restart=50),
}


def cloud_by_name(name: str, **kw) -> Cloud:
    return CONFIGS[name]["cloud"](**kw)
