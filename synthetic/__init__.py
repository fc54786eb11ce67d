"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws random numbers and lays them out; it holds none of the
labelling arithmetic.  Both the CUDA path and the CPU oracle read the arrays it
returns, so a parity test compares the two on identical inputs.

Conventions (fixed point, Q = 512 units per voxel):
  * a grid of dims ``(n_x, n_y[, n_z])`` spans ``[0, 512 n_i)`` per axis;
  * site coordinates are int32 in ``[0, 512 n_i)``, stored ``[N_s, ndim]``
    with x first;
  * Laguerre weights are ``w = r_q**2`` (int64) with ``r_q = round(512 r)``;
  * Johnson-Mehl birth times ``t`` and growth speeds ``v`` are float64.

The random source is SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state advances by the golden
gamma 0x9E3779B97F4A7C15 and each output is the state passed through the
published 64-bit finaliser.  Every purpose (coordinates, radii, times, ...)
draws from its own substream, so changing one array never shifts another.
The paper's workloads are sites placed uniformly at random in the domain
(Section 3, "Poisson" sites); the Matern-cluster and lognormal-radius recipes
add the uneven and weighted cases the benchmark exercises.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

Q = 512
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """One SplitMix64 substream, identified by ``(seed, *path)``."""

    def __init__(self, seed: int, *path: int):
        s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        with np.errstate(over="ignore"):
            for p in path:
                s = _mix(s + _GAMMA * np.uint64((p + 1) & 0xFFFFFFFFFFFFFFFF))
        self._state = int(s[0])
        self._count = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self._count + 1, self._count + n + 1, dtype=np.uint64)
        self._count += n
        with np.errstate(over="ignore"):
            z = np.uint64(self._state) + idx * _GAMMA
            return _mix(z)

    def below(self, n: int, bound: int) -> np.ndarray:
        """n integers in [0, bound) (bound < 2**32), by the high-32-bit product."""
        assert 0 < bound < (1 << 32)
        hi = self.u64(n) >> np.uint64(32)
        return ((hi * np.uint64(bound)) >> np.uint64(32)).astype(np.int64)

    def u53(self, n: int) -> np.ndarray:
        """n float64 in [0, 1) with 53 random bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, n: int) -> np.ndarray:
        """n standard normals by Box-Muller (cosine branch)."""
        u1 = 1.0 - self.u53(n)  # (0, 1]
        u2 = self.u53(n)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# substream tags
_COORD, _RADIUS, _TIME, _PARENT, _CHILDREN, _OFFSET, _META = range(7)


def uniform_sites(dims, n_sites: int, seed: int, stream: int = 0) -> np.ndarray:
    """Sites i.i.d. uniform on the fixed-point lattice of the box."""
    dims = tuple(int(d) for d in dims)
    out = np.empty((n_sites, len(dims)), dtype=np.int32)
    for a, n in enumerate(dims):
        out[:, a] = Stream(seed, stream, _COORD, a).below(n_sites, Q * n)
    return out


def lognormal_weights(n_sites: int, seed: int, mu: float = math.log(4.0),
                      sigma: float = 0.3, stream: int = 0) -> np.ndarray:
    """Laguerre weights w = r_q^2 with r lognormal(mu, sigma) in voxels."""
    z = Stream(seed, stream, _RADIUS).normal(n_sites)
    r = np.exp(mu + sigma * z)
    rq = np.floor(Q * r + 0.5).astype(np.int64)
    return rq * rq


def jm_times(n_sites: int, seed: int, t_max: float = 50.0, stream: int = 0):
    """Birth times uniform in [0, t_max) and unit growth speed."""
    t = t_max * Stream(seed, stream, _TIME).u53(n_sites)
    v = np.ones(n_sites, dtype=np.float64)
    return t, v


def _poisson(stream: Stream, n: int, lam: float) -> np.ndarray:
    kmax = int(lam + 12.0 * math.sqrt(lam) + 20)
    pmf = np.empty(kmax + 1)
    pmf[0] = math.exp(-lam)
    for k in range(1, kmax + 1):
        pmf[k] = pmf[k - 1] * lam / k
    cdf = np.cumsum(pmf)
    cdf[-1] = 1.0
    return np.searchsorted(cdf, stream.u53(n), side="right").astype(np.int64)


def matern_sites(dims, n_parents: int, mean_children: float, radius_vox: float,
                 seed: int, periodic: bool = True, stream: int = 0) -> np.ndarray:
    """Matern cluster process: uniform parents, Poisson(mean) children each,
    child offsets uniform in a ball of ``radius_vox`` voxels (rejection on the
    fixed-point lattice), wrapped (periodic) or clipped (non-periodic) to the box."""
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    parents = uniform_sites(dims, n_parents, seed, stream=stream * 16 + 1).astype(np.int64)
    counts = _poisson(Stream(seed, stream, _CHILDREN), n_parents, mean_children)
    total = int(counts.sum())
    R = int(round(radius_vox * Q))
    off_stream = Stream(seed, stream, _OFFSET)
    offs = np.empty((0, nd), dtype=np.int64)
    need = total
    while need > 0:
        batch = int(need * (2.2 if nd == 3 else 1.4)) + 64
        cand = np.stack([off_stream.below(batch, 2 * R + 1) - R for _ in range(nd)], axis=1)
        ok = (cand * cand).sum(axis=1) <= R * R
        offs = np.concatenate([offs, cand[ok][:need]])
        need = total - offs.shape[0]
    owner = np.repeat(np.arange(n_parents), counts)
    pts = parents[owner] + offs
    L = np.array([Q * n for n in dims], dtype=np.int64)
    if periodic:
        pts = np.mod(pts, L)
    else:
        pts = np.clip(pts, 0, L - 1)
    return pts.astype(np.int32)


@dataclass
class Instance:
    """One labelling problem: a grid, its boundary conditions and its sites."""
    kind: str                      # "voronoi" | "laguerre" | "jm"
    dims: tuple                    # (n_x, n_y[, n_z])
    periodic: bool | int           # every axis (bool), or bit i of an int: axis i
    sites: np.ndarray              # int32 [N_s, ndim]
    w: np.ndarray | None = None    # int64 [N_s]      (laguerre)
    t: np.ndarray | None = None    # float64 [N_s]    (jm)
    v: np.ndarray | None = None    # float64 [N_s]    (jm)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_sites(self) -> int:
        return int(self.sites.shape[0])

    @property
    def n_voxels(self) -> int:
        return int(np.prod(self.dims))


def make_instance(kind: str, dims, n_sites: int, seed: int, periodic: bool,
                  stream: int = 0, sites: np.ndarray | None = None,
                  name: str = "") -> Instance:
    dims = tuple(int(d) for d in dims)
    if sites is None:
        sites = uniform_sites(dims, n_sites, seed, stream)
    n = sites.shape[0]
    inst = Instance(kind=kind, dims=dims, periodic=periodic, sites=sites, name=name)
    if kind == "laguerre":
        inst.w = lognormal_weights(n, seed, stream=stream)
    elif kind == "jm":
        inst.t, inst.v = jm_times(n, seed, stream=stream)
    elif kind != "voronoi":
        raise ValueError(kind)
    return inst


# ---- the benchmark's workloads, by what they are -------------------------

def voronoi_64_periodic_100() -> Instance:
    return make_instance("voronoi", (64, 64, 64), 100, seed=0, periodic=True,
                         name="voronoi-3d-64^3-periodic-100")


def laguerre_512_1e4() -> Instance:
    return make_instance("laguerre", (512, 512, 512), 10_000, seed=1, periodic=False,
                         name="laguerre-3d-512^3-nonperiodic-1e4")


def laguerre_16384sq_1e5() -> Instance:
    return make_instance("laguerre", (16384, 16384), 100_000, seed=2, periodic=False,
                         name="laguerre-2d-16384^2-nonperiodic-1e5")


def jm_1024_1e5() -> Instance:
    return make_instance("jm", (1024, 1024, 1024), 100_000, seed=3, periodic=True,
                         name="jm-3d-1024^3-periodic-1e5")


def precision_1024_1e6(kind: str, cluster: bool) -> Instance:
    dims = (1024, 1024, 1024)
    if cluster:
        sites = matern_sites(dims, 10_000, 100.0, 8.0, seed=5, periodic=True)
    else:
        sites = uniform_sites(dims, 1_000_000, seed=4)
    inst = make_instance(kind, dims, sites.shape[0], seed=5 if cluster else 4,
                         periodic=True, sites=sites,
                         name=f"{kind}-3d-1024^3-periodic-{'matern' if cluster else 'uniform'}-1e6")
    if cluster:
        # empty space between clusters: the largest distance from a voxel to the
        # nearest site is of the order of the parent spacing (~48 voxels)
        inst.meta["void_radius_vox"] = 72.0
    return inst


def batch_64(seed: int = 6, count: int = 64) -> list[Instance]:
    """Ensemble of uneven microstructures: per instance j (substream j) draw
    the dimension, edge, periodicity, site count and diagram type."""
    out = []
    for j in range(count):
        m = Stream(seed, j, _META)
        u = m.u53(6)
        nd = 2 if u[0] < 0.5 else 3
        if nd == 3:
            e = 64 + 32 * int(u[1] * 11)          # 64..384 step 32
            dims = (e, e, e)
        else:
            e = 512 * (1 + int(u[1] * 16))        # 512..8192 step 512
            dims = (e, e)
        periodic = bool(u[2] < 0.5)
        ns = int(round(math.exp(math.log(50.0) + u[3] * (math.log(5e4) - math.log(50.0)))))
        kind = ("voronoi", "laguerre", "jm")[min(2, int(u[4] * 3))]
        out.append(make_instance(kind, dims, ns, seed=seed, periodic=periodic, stream=j + 1,
                                 name=f"b{j}-{kind}-{nd}d-{e}-{'p' if periodic else 'np'}-{ns}"))
    return out
