"""Seeded synthetic catalogues shaped like the paper's w(theta) workloads.

This module only draws inputs: positions on the sphere (RA, Dec in degrees,
interleaved float64 ``[ra0, dec0, ra1, dec1, ...]``) and the bin ranges of each
workload.  It holds none of the pair-counting or estimator arithmetic, so both
the CUDA path and the CPU oracle can take their inputs from it.

The paper measured on a decorated N-body galaxy catalogue in the field
0 < RA < 90 deg, 0 < Dec < 90 deg with flat randoms over the same field
(Sec. 2.2).  That dataset is not available, so clustered catalogues stand in
for it: cluster centres are uniform on the footprint, each centre gets a
Poisson number of members, and each member is offset from its centre by a 2-D
Gaussian in the local tangent plane.  Randoms are uniform (equal-area) on the
same footprint, as the paper requires of its random catalogue (Sec. 2).

Every stream is derived from ``numpy.random.SeedSequence(seed, spawn_key=...)``
with a key naming (workload, catalogue, role, index), so catalogues are
independent and reproducible on any machine.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Tuple

import numpy as np

DEG = math.pi / 180.0
ARCMIN = 1.0 / 60.0  # degrees

# spawn-key vocabulary: stable integers for the names used in stream keys
_KEYS = {
    "small": 1, "survey": 2, "batch": 3, "serve": 4, "largest": 5, "test": 6,
    "data": 10, "random": 11, "data2": 12, "random2": 13,
    "centres": 20, "members": 21, "offsets": 22, "uniform": 23, "sizes": 24,
    "patch": 25, "arrivals": 26, "kinds": 27, "subsample": 28,
}


def rng_for(seed: int, *path) -> np.random.Generator:
    """Independent generator for one (workload, catalogue, role, index) path."""
    key = tuple(_KEYS[p] if isinstance(p, str) else int(p) for p in path)
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed, spawn_key=key)))


# --------------------------------------------------------------------------
# footprints
# --------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Patch:
    """RA in [ra0, ra0 + width) (wrapping at 360), Dec in [dec0, dec1)."""
    ra0: float
    ra_width: float
    dec0: float
    dec1: float

    def sample(self, rng: np.random.Generator, n: int) -> Tuple[np.ndarray, np.ndarray]:
        ra = np.mod(self.ra0 + self.ra_width * rng.random(n), 360.0)
        s0, s1 = math.sin(self.dec0 * DEG), math.sin(self.dec1 * DEG)
        dec = np.arcsin(np.clip(s0 + (s1 - s0) * rng.random(n), -1.0, 1.0)) / DEG
        return ra, dec

    def contains(self, ra: np.ndarray, dec: np.ndarray) -> np.ndarray:
        dra = np.mod(ra - self.ra0, 360.0)
        return (dra < self.ra_width) & (dec >= self.dec0) & (dec < self.dec1)


@dataclasses.dataclass(frozen=True)
class Cap:
    """Spherical cap of the given radius about the north pole."""
    radius_deg: float

    def sample(self, rng, n):
        zmin = math.cos(self.radius_deg * DEG)
        z = zmin + (1.0 - zmin) * rng.random(n)
        ra = 360.0 * rng.random(n)
        dec = np.arcsin(np.clip(z, -1.0, 1.0)) / DEG
        return ra, dec

    def contains(self, ra, dec):
        return dec >= 90.0 - self.radius_deg


@dataclasses.dataclass(frozen=True)
class FullSky:
    def sample(self, rng, n):
        z = -1.0 + 2.0 * rng.random(n)
        ra = 360.0 * rng.random(n)
        dec = np.arcsin(np.clip(z, -1.0, 1.0)) / DEG
        return ra, dec

    def contains(self, ra, dec):
        return np.ones(np.shape(ra), dtype=bool)


def interleave(ra: np.ndarray, dec: np.ndarray) -> np.ndarray:
    out = np.empty((len(ra), 2), dtype=np.float64)
    out[:, 0] = ra
    out[:, 1] = dec
    return out.reshape(-1)


# --------------------------------------------------------------------------
# catalogues
# --------------------------------------------------------------------------
def uniform(footprint, n: int, seed: int, *path) -> np.ndarray:
    """n points uniform (equal-area) on the footprint."""
    ra, dec = footprint.sample(rng_for(seed, *path, "uniform"), n)
    return interleave(ra, dec)


def clustered(footprint, n: int, n_centres: int, sigma_arcmin: float,
              seed: int, *path, members_mean: float = 50.0) -> np.ndarray:
    """n clustered points: Poisson(members_mean) members per centre, Gaussian
    tangent-plane offsets of dispersion sigma per axis, members outside the
    footprint rejected, more centres drawn from the same streams until n points
    exist, then truncated to n in generation order."""
    rc = rng_for(seed, *path, "centres")
    rm = rng_for(seed, *path, "members")
    ro = rng_for(seed, *path, "offsets")
    sigma = sigma_arcmin * ARCMIN * DEG  # radians
    chunks_ra: List[np.ndarray] = []
    chunks_dec: List[np.ndarray] = []
    have = 0
    batch = max(1, n_centres)
    while have < n:
        cra, cdec = footprint.sample(rc, batch)
        k = rm.poisson(members_mean, batch)
        tot = int(k.sum())
        if tot == 0:
            continue
        idx = np.repeat(np.arange(batch), k)
        a, d = cra[idx] * DEG, cdec[idx] * DEG
        ca, sa, cd, sd = np.cos(a), np.sin(a), np.cos(d), np.sin(d)
        c = np.stack([cd * ca, cd * sa, sd], axis=1)
        east = np.stack([-sa, ca, np.zeros_like(a)], axis=1)
        north = np.stack([-sd * ca, -sd * sa, cd], axis=1)
        off = ro.normal(0.0, sigma, (tot, 2))
        p = c + off[:, :1] * east + off[:, 1:] * north
        p /= np.linalg.norm(p, axis=1, keepdims=True)
        ra = np.mod(np.arctan2(p[:, 1], p[:, 0]) / DEG, 360.0)
        dec = np.arctan2(p[:, 2], np.hypot(p[:, 0], p[:, 1])) / DEG
        keep = footprint.contains(ra, dec)
        chunks_ra.append(ra[keep])
        chunks_dec.append(dec[keep])
        have += int(keep.sum())
    ra = np.concatenate(chunks_ra)[:n]
    dec = np.concatenate(chunks_dec)[:n]
    return interleave(ra, dec)


def subsample(cat: np.ndarray, m: int, seed: int, *path) -> np.ndarray:
    """Seeded subsample of m points (without replacement, original order)."""
    n = len(cat) // 2
    if m >= n:
        return cat.copy()
    idx = np.sort(rng_for(seed, *path, "subsample").choice(n, m, replace=False))
    return cat.reshape(-1, 2)[idx].reshape(-1).copy()


# --------------------------------------------------------------------------
# workloads (the bin range is (lo_deg, hi_deg, n_bins), log-spaced)
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    data: np.ndarray
    rand: np.ndarray
    lo_deg: float
    hi_deg: float
    n_bins: int

    @property
    def n_d(self):
        return len(self.data) // 2

    @property
    def n_r(self):
        return len(self.rand) // 2

    @property
    def pairs(self) -> int:
        nd, nr = self.n_d, self.n_r
        return nd * (nd - 1) // 2 + nd * nr + nr * (nr - 1) // 2


def small(seed: int = 1, n: int = 10_000) -> Workload:
    """10k clustered + 10k uniform in a 10x10 deg patch; 16 log bins 1'-5 deg."""
    fp = Patch(0.0, 10.0, 0.0, 10.0)
    d = clustered(fp, n, max(1, round(200 * n / 10_000)), 3.0, seed, "small", "data")
    r = uniform(fp, n, seed, "small", "random")
    return Workload("small", d, r, 1.0 * ARCMIN, 5.0, 16)


def survey(seed: int = 1, n: int = 1_000_000, n_rand: int | None = None) -> Workload:
    """1M clustered (20k centres, sigma 2') + 1M uniform in a 60 deg polar cap;
    32 log bins 0.5'-20 deg."""
    fp = Cap(60.0)
    nr = n if n_rand is None else n_rand
    d = clustered(fp, n, max(1, round(20_000 * n / 1_000_000)), 2.0, seed, "survey", "data")
    r = uniform(fp, nr, seed, "survey", "random")
    return Workload("survey", d, r, 0.5 * ARCMIN, 20.0, 32)


def largest(seed: int = 1, n: int = 10_000_000) -> Workload:
    """10M clustered (200k centres, sigma 1') + 10M uniform full sky;
    64 log bins 0.2'-30 deg."""
    fp = FullSky()
    d = clustered(fp, n, max(1, round(200_000 * n / 10_000_000)), 1.0, seed, "largest", "data")
    r = uniform(fp, n, seed, "largest", "random")
    return Workload("largest", d, r, 0.2 * ARCMIN, 30.0, 64)


@dataclasses.dataclass
class Mock:
    data: np.ndarray
    rand: np.ndarray


def batch_sizes(seed: int = 1, n_mocks: int = 256, n_lo: int = 20_000,
                n_hi: int = 400_000) -> np.ndarray:
    """Data sizes of the batch workload's mocks, log-uniform in [n_lo, n_hi]."""
    rs = rng_for(seed, "batch", "sizes")
    return np.rint(np.exp(rs.uniform(math.log(n_lo), math.log(n_hi), n_mocks))).astype(np.int64)


def batch_mock(seed: int, m: int, n_mocks: int = 256, n_lo: int = 20_000,
               n_hi: int = 400_000) -> Mock:
    """Mock m of batch_mocks alone (same streams, same points)."""
    n = int(batch_sizes(seed, n_mocks, n_lo, n_hi)[m])
    rp = rng_for(seed, "batch", "patch")
    ra0 = rp.uniform(0.0, 360.0, n_mocks)
    dec0 = rp.uniform(-60.0, 45.0, n_mocks)
    fp = Patch(float(ra0[m]), 15.0, float(dec0[m]), float(dec0[m]) + 15.0)
    d = clustered(fp, n, math.ceil(n / 50), 3.0, seed, "batch", "data", m)
    r = uniform(fp, 2 * n, seed, "batch", "random", m)
    return Mock(d, r)


def batch_mocks(seed: int = 1, n_mocks: int = 256, n_lo: int = 20_000,
                n_hi: int = 400_000) -> Tuple[List[Mock], Tuple[float, float, int]]:
    """256 mocks, sizes log-uniform in [20k, 400k], each clustered (n/50
    centres, sigma 3') in its own 15x15 deg patch with 2x uniform randoms;
    16 log bins 1'-5 deg."""
    mocks = [batch_mock(seed, m, n_mocks, n_lo, n_hi) for m in range(n_mocks)]
    return mocks, (1.0 * ARCMIN, 5.0, 16)


@dataclasses.dataclass
class Request:
    t_arrive: float          # seconds after the stream starts
    kind: str                # "auto" or "cross"
    data: np.ndarray
    rand: np.ndarray
    data2: np.ndarray | None = None
    rand2: np.ndarray | None = None


def _serve_plan(seed, n_requests, n_lo, n_hi, rate_hz, auto_frac):
    ra = rng_for(seed, "serve", "arrivals")
    gaps = ra.exponential(1.0 / rate_hz, n_requests)
    t = np.cumsum(gaps) - gaps[0]
    rs = rng_for(seed, "serve", "sizes")
    sizes = np.rint(np.exp(rs.uniform(math.log(n_lo), math.log(n_hi), n_requests))).astype(np.int64)
    kinds = rng_for(seed, "serve", "kinds").random(n_requests) < auto_frac
    rp = rng_for(seed, "serve", "patch")
    ra0 = rp.uniform(0.0, 360.0, n_requests)
    dec0 = rp.uniform(-60.0, 45.0, n_requests)
    return t, sizes, kinds, ra0, dec0


def serve_sizes(seed: int = 1, n_requests: int = 2000, n_lo: int = 1_000,
                n_hi: int = 2_000_000, auto_frac: float = 0.7):
    """(sizes, is_auto) of the serve workload's requests."""
    _, sizes, kinds, _, _ = _serve_plan(seed, n_requests, n_lo, n_hi, 1.0, auto_frac)
    return sizes, kinds


def serve_request(seed: int, q: int, n_requests: int = 2000, n_lo: int = 1_000,
                  n_hi: int = 2_000_000, rate_hz: float = 1.0,
                  auto_frac: float = 0.7) -> Request:
    """Request q of serve_requests alone (same streams, same points)."""
    t, sizes, kinds, ra0, dec0 = _serve_plan(seed, n_requests, n_lo, n_hi, rate_hz, auto_frac)
    fp = Patch(float(ra0[q]), 15.0, float(dec0[q]), float(dec0[q]) + 15.0)
    n = int(sizes[q])
    nc = max(1, math.ceil(n / 50))
    d = clustered(fp, n, nc, 3.0, seed, "serve", "data", q)
    r = uniform(fp, n, seed, "serve", "random", q)
    if kinds[q]:
        return Request(float(t[q]), "auto", d, r)
    d2 = clustered(fp, n, nc, 3.0, seed, "serve", "data2", q)
    r2 = uniform(fp, n, seed, "serve", "random2", q)
    return Request(float(t[q]), "cross", d, r, d2, r2)


def serve_requests(seed: int = 1, n_requests: int = 2000, n_lo: int = 1_000,
                   n_hi: int = 2_000_000, rate_hz: float = 1.0,
                   auto_frac: float = 0.7) -> Tuple[List[Request], Tuple[float, float, int]]:
    """Poisson-arrival w(theta) requests, sizes log-uniform in [n_lo, n_hi] with
    1:1 randoms, 70% auto / 30% cross, each in a 15x15 deg patch clustered as
    the small workload; 24 log bins 1'-10 deg."""
    reqs = [serve_request(seed, q, n_requests, n_lo, n_hi, rate_hz, auto_frac)
            for q in range(n_requests)]
    return reqs, (1.0 * ARCMIN, 10.0, 24)


def grid_labels(ra_dec: np.ndarray, ra0: float, ra1: float, dec0: float, dec1: float,
                nx: int, ny: int) -> np.ndarray:
    """Region labels (int32) of points on an nx x ny grid of equal RA and Dec
    steps over [ra0, ra1) x [dec0, dec1); points outside are clamped to the
    nearest cell.  A jackknife region layout for patch footprints."""
    rd = np.asarray(ra_dec, np.float64).reshape(-1, 2)
    ra = np.mod(rd[:, 0] - ra0, 360.0)
    ix = np.clip(np.floor(ra / (ra1 - ra0) * nx), 0, nx - 1).astype(np.int64)
    iy = np.clip(np.floor((rd[:, 1] - dec0) / (dec1 - dec0) * ny), 0, ny - 1).astype(np.int64)
    return (iy * nx + ix).astype(np.int32)
