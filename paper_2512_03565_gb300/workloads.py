"""Seeded synthetic particle systems shaped like the paper's workloads.

This module only *generates inputs*; it holds none of the force method's
arithmetic and is shared by the CUDA path's tests/bench and by the oracle's
tests.  Positions are returned as uint32 fixed point in SoA form (3, n):
coordinate = x_fp * L / 2^32 in a cubic periodic box of edge L.  Velocities
are float64 (3, n).

The paper's own inputs (AutoPas md-flexible YAML files for the Exploding Cube
and Exploding Liquid, Sec. 5.1 and 5.2) are not available; these generators
stand in for them with the sizes, densities, cutoffs and structure of the
workloads this library is measured on:

* ``uniform``      pure uniform random positions (one force evaluation only).
* ``stratified``   one particle per site of a cubic sub-lattice, jittered
                   uniformly inside the site so that the minimum separation is
                   max(0.4 a, 0.85 sigma); a homogeneous fluid-like start that
                   can be integrated without overlaps blowing up.
* ``fcc``          jittered face-centred cubic lattice (dense systems).
* ``slab``         two-phase liquid/vapour slab along z.
* ``droplet``      FCC liquid sphere in a large vacuum box.
* ``ensemble``     many independent boxes of uneven sizes and densities.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 20251203
TWO32 = 2.0 ** 32


@dataclass
class System:
    """One periodic cubic box of particles."""
    L: float
    pos: np.ndarray            # (3, n) uint32 fixed point
    vel: np.ndarray            # (3, n) float64
    rc: float = 2.5
    skin: float = 0.3
    eps: float = 1.0
    sigma: float = 1.0
    mass: float = 1.0
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[1])


def _frac_to_fp(frac: np.ndarray) -> np.ndarray:
    """Fractions of the box in [0, 1) -> uint32 fixed point (floor, wrap)."""
    f = np.mod(frac, 1.0)
    q = np.floor(f * TWO32)
    q[q >= TWO32] = 0.0
    return q.astype(np.uint64).astype(np.uint32)


def maxwell_boltzmann(rng: np.random.Generator, n: int, T: float, mass: float = 1.0) -> np.ndarray:
    """Velocities N(0, sqrt(T/m)) per component, centre-of-mass removed and
    rescaled to temperature T exactly (k_B = 1, 3n - 3 degrees of freedom)."""
    v = rng.normal(0.0, math.sqrt(T / mass), size=(3, n))
    if n > 1:
        v -= v.mean(axis=1, keepdims=True)
        ke2 = mass * float((v * v).sum())
        dof = 3 * n - 3
        if ke2 > 0:
            v *= math.sqrt(T * dof / ke2)
    return v


def box_edge(n: int, rho: float) -> float:
    return (n / rho) ** (1.0 / 3.0)


def uniform(n: int, rho: float, seed: int, T: float = 1.0, **kw) -> System:
    rng = np.random.default_rng(seed)
    L = box_edge(n, rho)
    pos = _frac_to_fp(rng.random((3, n)))
    return System(L=L, pos=pos, vel=maxwell_boltzmann(rng, n, T), name=f"uniform n={n} rho={rho}", **kw)


def _stratified_fracs(rng, n: int, L: float) -> np.ndarray:
    ns = int(math.ceil(n ** (1.0 / 3.0) - 1e-9))
    while ns ** 3 < n:
        ns += 1
    a = L / ns
    sites = rng.choice(ns ** 3, size=n, replace=False) if ns ** 3 > n else np.arange(n)
    sx, sy, sz = sites % ns, (sites // ns) % ns, sites // (ns * ns)
    min_sep = max(0.4 * a, min(0.85, a))
    h = max(0.0, (1.0 - min_sep / a) / 2.0)     # half-width of the jitter, in site units
    jit = rng.uniform(-h, h, size=(3, n))
    frac = (np.stack([sx, sy, sz]).astype(np.float64) + 0.5 + jit) / ns
    return frac


def stratified(n: int, rho: float, seed: int, T: float = 1.0, **kw) -> System:
    rng = np.random.default_rng(seed)
    L = box_edge(n, rho)
    pos = _frac_to_fp(_stratified_fracs(rng, n, L))
    return System(L=L, pos=pos, vel=maxwell_boltzmann(rng, n, T), name=f"stratified n={n} rho={rho}", **kw)


_FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])


def fcc_sites(m: int) -> np.ndarray:
    """Fractional coordinates (3, 4 m^3) of an m x m x m FCC lattice in a unit box."""
    g = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1).reshape(-1, 3)
    pts = (g[:, None, :] + _FCC_BASIS[None, :, :]).reshape(-1, 3) / m
    return pts.T.copy()


def fcc(n: int, rho: float, seed: int, T: float = 1.0, jitter: float = 0.02, **kw) -> System:
    """Jittered FCC at density rho; n sites drawn from the smallest m^3 lattice."""
    rng = np.random.default_rng(seed)
    L = box_edge(n, rho)
    m = 1
    while 4 * m ** 3 < n:
        m += 1
    pts = fcc_sites(m)
    if pts.shape[1] > n:
        pts = pts[:, np.sort(rng.choice(pts.shape[1], size=n, replace=False))]
    pts = pts + rng.uniform(-jitter, jitter, size=pts.shape) / m
    return System(L=L, pos=_frac_to_fp(pts), vel=maxwell_boltzmann(rng, n, T), name=f"fcc n={n} rho={rho}", **kw)


def perfect_fcc(m: int, rho: float) -> System:
    """Perfect FCC, m^3 unit cells; for m a power of two every site is an exact
    fixed-point value."""
    n = 4 * m ** 3
    L = box_edge(n, rho)
    return System(L=L, pos=_frac_to_fp(fcc_sites(m)), vel=np.zeros((3, n)), name=f"perfect fcc m={m}")


def homogeneous(n: int, rho: float, seed: int, T: float = 1.0, **kw) -> System:
    """Homogeneous fluid start: stratified below rho 0.9, jittered FCC above."""
    if rho >= 0.9:
        return fcc(n, rho, seed, T, **kw)
    return stratified(n, rho, seed, T, **kw)


def _stratified_region(rng, n: int, ext: np.ndarray) -> np.ndarray:
    """n jittered sites in an axis-aligned region of extents ext (3,), absolute
    units, returned as positions relative to the region's corner."""
    a = (float(np.prod(ext)) / n) ** (1.0 / 3.0)
    dims = np.maximum(1, np.floor(ext / a).astype(int))
    k = 0
    while int(np.prod(dims)) < n:
        dims[k % 3] += 1
        k += 1
    cells = int(np.prod(dims))
    sites = rng.choice(cells, size=n, replace=False) if cells > n else np.arange(n)
    idx = np.stack([sites % dims[0], (sites // dims[0]) % dims[1], sites // (dims[0] * dims[1])])
    step = ext / dims
    amin = float(step.min())
    min_sep = max(0.4 * amin, min(0.85, amin))
    h = max(0.0, (1.0 - min_sep / amin) / 2.0)
    jit = rng.uniform(-h, h, size=(3, n))
    return (idx + 0.5 + jit) * step[:, None]


def slab(n: int, rho_liq: float, rho_vap: float, frac: float, seed: int, T: float = 1.0, **kw) -> System:
    """Two-phase slab normal to z: a liquid layer of thickness frac*L at rho_liq
    and vapour elsewhere at rho_vap, in a cube sized for the mean density."""
    rng = np.random.default_rng(seed)
    rho_mean = frac * rho_liq + (1.0 - frac) * rho_vap
    L = box_edge(n, rho_mean)
    n_liq = int(round(n * frac * rho_liq / rho_mean))
    n_vap = n - n_liq
    liq = _stratified_region(rng, n_liq, np.array([L, L, frac * L])) / L
    liq[2] += 0.5 - frac / 2.0
    vap = _stratified_region(rng, n_vap, np.array([L, L, (1.0 - frac) * L])) / L
    vap[2] = np.mod(vap[2] + 0.5 + frac / 2.0, 1.0)
    pts = np.concatenate([liq, vap], axis=1)[:, rng.permutation(n)]
    return System(L=L, pos=_frac_to_fp(pts), vel=maxwell_boltzmann(rng, n, T),
                  name=f"slab n={n} frac={frac}", meta={"rho_liq": rho_liq, "rho_vap": rho_vap}, **kw)


def droplet(radius: float, rho: float = 0.8, seed: int = BASE_SEED + 3, T: float = 1.2,
            box_factor: float = 4.0, **kw) -> System:
    """FCC liquid sphere of the given radius at density rho, centred in a
    periodic vacuum box of edge box_factor * diameter."""
    rng = np.random.default_rng(seed)
    a = (4.0 / rho) ** (1.0 / 3.0)
    m = int(math.ceil(2 * radius / a)) + 2
    pts = fcc_sites(m) * m * a - m * a / 2.0            # absolute, centred at 0
    r = np.sqrt((pts ** 2).sum(axis=0))
    pts = pts[:, r <= radius]
    n = pts.shape[1]
    L = box_factor * 2.0 * radius
    pts = pts + rng.uniform(-0.01, 0.01, size=pts.shape) * a
    frac = pts / L + 0.5
    return System(L=L, pos=_frac_to_fp(frac), vel=maxwell_boltzmann(rng, n, T),
                  name=f"droplet R={radius} n={n}", **kw)


def ensemble(nboxes: int = 256, nmin: int = 500, nmax: int = 50000, rho_lo: float = 0.1,
             rho_hi: float = 1.0, seed: int = BASE_SEED + 4, T: float = 1.0, **kw) -> list:
    """Independent boxes: N log-uniform in [nmin, nmax], rho uniform in [rho_lo, rho_hi]."""
    rng = np.random.default_rng(seed)
    ns = np.floor(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=nboxes))).astype(int)
    rhos = rng.uniform(rho_lo, rho_hi, size=nboxes)
    seeds = rng.integers(0, 2 ** 31 - 1, size=nboxes)
    return [homogeneous(int(n), float(r), int(s), T, **kw) for n, r, s in zip(ns, rhos, seeds)]


def exploding_cube(n: int, rho: float = 0.9, box_factor: float = 3.0, seed: int = BASE_SEED + 5,
                   T: float = 1.2, **kw) -> System:
    """Dense jittered-FCC cube of n particles at density rho centred in a periodic
    vacuum box of edge box_factor x the cube's edge (the shape of the paper's
    "Exploding Cube" benchmark, Sec. 5.1)."""
    rng = np.random.default_rng(seed)
    side = (n / rho) ** (1.0 / 3.0)
    L = box_factor * side
    m = 1
    while 4 * m ** 3 < n:
        m += 1
    pts = fcc_sites(m)
    if pts.shape[1] > n:
        pts = pts[:, np.sort(rng.choice(pts.shape[1], size=n, replace=False))]
    pts = pts + rng.uniform(-0.02, 0.02, size=pts.shape) / m
    frac = 0.5 + (pts - 0.5) * (side / L)
    return System(L=L, pos=_frac_to_fp(frac), vel=maxwell_boltzmann(rng, n, T),
                  name=f"cube n={n} factor={box_factor}", **kw)


def vacuum_extension(rc: float = 2.5, seed: int = BASE_SEED + 6) -> list:
    """Inhomogeneous, vacuum-dominated systems that extend the density sweep:
    liquid spheres (R 20, 30, 45) in boxes of 4x their diameter and dense cubes in
    boxes of 3x and 5x their edge -- all smaller than the expanding-droplet
    workload, which stays out of the training data."""
    out = []
    for k, R in enumerate([20.0, 30.0, 45.0]):
        out.append(droplet(R, 0.8, seed + k, T=1.2, rc=rc, skin=0.3))
    for k, (n, f) in enumerate([(100000, 3.0), (300000, 5.0)]):
        out.append(exploding_cube(n, 0.9, f, seed + 10 + k, T=1.2, rc=rc, skin=0.3))
    return out


# --- the named workloads ---------------------------------------------------

def config1() -> System:
    """1,000 LJ particles, uniform random, density 0.8 (L = 10.7722), rc 2.5, one FP64 evaluation."""
    return uniform(1000, 0.8, BASE_SEED + 0, T=1.0, rc=2.5, skin=0.3)


def config2(n: int = 1048576) -> System:
    """Homogeneous LJ fluid, density 0.75 (L = 111.818 at n = 2^20), rc 2.5, skin 0.3, T = 1."""
    return homogeneous(n, 0.75, BASE_SEED + 1, T=1.0, rc=2.5, skin=0.3)


def config3(rc: float = 2.5, scale: float = 1.0) -> list:
    """Density sweep: 16 uniform boxes (rho log-spaced 0.05..1.2, N cycling over
    100k..2M) and 8 two-phase slabs (liquid 0.8 / vapour 0.02, slab fraction
    0.3..0.65).  scale < 1 shrinks every N (for quick runs)."""
    out = []
    rhos = np.exp(np.linspace(math.log(0.05), math.log(1.2), 16))
    nlist = [100_000, 200_000, 500_000, 1_000_000, 2_000_000]
    for k, rho in enumerate(rhos):
        n = max(2000, int(nlist[k % len(nlist)] * scale))
        out.append(homogeneous(n, float(rho), BASE_SEED + 2 + 1000 * k, T=1.0, rc=rc, skin=0.3))
    for k, f in enumerate(np.arange(0.30, 0.66, 0.05)):
        n = max(2000, int(nlist[k % len(nlist)] * scale))
        out.append(slab(n, 0.8, 0.02, float(f), BASE_SEED + 2 + 1000 * (16 + k), T=1.0, rc=rc, skin=0.3))
    return out


def config4(radius: float = 84.19) -> System:
    """Expanding droplet: FCC sphere at rho 0.8, T 1.2, box 4x the diameter."""
    return droplet(radius, 0.8, BASE_SEED + 3, T=1.2, rc=2.5, skin=0.3)


def config5(nboxes: int = 256, nmin: int = 500, nmax: int = 50000) -> list:
    """Batched ensemble: N log-uniform [500, 50000], rho uniform [0.1, 1.0]."""
    return ensemble(nboxes, nmin, nmax, 0.1, 1.0, BASE_SEED + 4, T=1.0, rc=2.5, skin=0.3)
