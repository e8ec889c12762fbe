"""Seeded synthetic workloads: grids, sensors, pixel directions, geometries.

This module is the one thing the CUDA path and the FP64 oracle share.  It
holds none of the method's arithmetic (no ray march, indicator, flux,
likelihood, prior or sampler): it only lays out the inputs of a problem the
way the paper's simulated experiment is shaped (Sec. 4: layered cave, a
lattice of sensors under it, radiograph pixel grids), with sizes taken from
the two standard workloads below.  Random draws use numpy's PCG64 seeded
through ``SeedSequence``; they are inputs, not part of the method.

Geometry recipe (the paper's expert cave model is not public): each surface
is a base height plus three Gaussian bumps (amplitude 10 m, sigma 30 m,
centres uniform over the box's xy extent), then clipped so that every
surface stays at least ``delta`` above the one below and inside the box.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

# Unit densities in g/cc (rock 2.65, muck 1.9, air 0.0012).
ROCK, MUCK, AIR = 2.65, 1.9, 0.0012


@dataclass
class Workload:
    name: str
    box: tuple = (200.0, 200.0, 150.0)
    R: int = 16                    # surface grid rows (y)
    Q: int = 16                    # surface grid cols (x)
    bases: tuple = (40.0, 70.0, 110.0)   # base height per surface, bottom to top
    rho: tuple = (ROCK, MUCK, AIR, ROCK)  # unit densities bottom to top (L+1)
    sensors: tuple = ()            # ((x, y, z), ...)
    n_zenith: int = 32
    n_azimuth: int = 32
    zenith_max_deg: float = 60.0
    G: int = 64                    # samples per ray
    gamma: float = 1.0             # sigmoid scale (m); 0 = Heaviside
    I0: float = 1.0e4
    Lambda: float = 150.0          # attenuation length (mwe)
    tau: float = 0.01              # prior precision scale (1/m^2)
    car_r: float = 0.99            # CAR spatial dependence
    delta: float = 0.1             # minimum thickness (m)
    n_chains: int = 4
    n_super: int = 10
    n_within: int = 10
    bump_amp: float = 10.0
    bump_sigma: float = 30.0
    n_bumps: int = 3
    seed_geom: int = 1
    seed_data: int = 2
    seed_init: int = 3
    seed_mcmc: int = 4
    rw_sigma: float = 0.02         # random-walk step (m)
    extra: dict = field(default_factory=dict)

    @property
    def L(self) -> int:
        return len(self.bases)

    @property
    def S(self) -> int:
        return len(self.sensors)

    @property
    def P(self) -> int:
        return self.n_zenith * self.n_azimuth

    def as_dict(self) -> dict:
        d = asdict(self)
        d["L"], d["S"], d["P"] = self.L, self.S, self.P
        return d


def tiny() -> Workload:
    """16x16 grid, 3 surfaces, 2 sensors x 32x32 pixels (zenith 0-60 deg), 64 samples, 4 chains."""
    Lx, Ly = 200.0, 200.0
    return Workload(
        name="tiny-16x16x3-2s-32x32px-g64",
        sensors=((Lx / 3.0, Ly / 2.0, 20.0), (2.0 * Lx / 3.0, Ly / 2.0, 20.0)),
        n_chains=4, n_super=10, n_within=10, rw_sigma=0.05)


def scenario() -> Workload:
    """64x64 grid, 4 surfaces, 16 sensors on a 4x4 lattice x 64x64 pixels (zenith 0-70 deg),
    256 samples per ray, 1024 chains, 100 x 10 steps."""
    Lx, Ly = 200.0, 200.0
    sens = tuple(((i + 0.5) * Lx / 4.0, (j + 0.5) * Ly / 4.0, 20.0)
                 for j in range(4) for i in range(4))
    return Workload(
        name="scenario-64x64x4-16s-64x64px-g256",
        R=64, Q=64, bases=(40.0, 70.0, 110.0, 140.0),
        rho=(ROCK, MUCK, AIR, ROCK, AIR), sensors=sens,
        n_zenith=64, n_azimuth=64, zenith_max_deg=70.0, G=256,
        n_chains=1024, n_super=100, n_within=10, rw_sigma=0.002)


def small(R=5, Q=7, bases=(40.0, 75.0), rho=(ROCK, MUCK, AIR), n_sensors=2, n_zenith=5,
          n_azimuth=7, G=16, gamma=1.0, n_chains=3, zenith_max_deg=60.0, **kw) -> Workload:
    """Odd-sized problems for parity tests (non-square grids, ragged pixel counts)."""
    Lx, Ly = 200.0, 200.0
    sens = tuple(((k + 1) * Lx / (n_sensors + 1), Ly * (0.3 + 0.4 * (k % 2)), 20.0)
                 for k in range(n_sensors))
    return Workload(name=f"small-{R}x{Q}x{len(bases)}", R=R, Q=Q, bases=tuple(bases),
                    rho=tuple(rho), sensors=sens, n_zenith=n_zenith, n_azimuth=n_azimuth,
                    zenith_max_deg=zenith_max_deg, G=G, gamma=gamma, n_chains=n_chains, **kw)


def pixel_dirs(n_zenith: int, n_azimuth: int, zenith_max_deg: float) -> np.ndarray:
    """Unit directions at the centres of a polar pixel grid, [n_zenith*n_azimuth][3].

    Pixel p = i*n_azimuth + j looks along zenith (i+1/2)*zmax/n_zenith and
    azimuth (j+1/2)*2pi/n_azimuth; the image centre points straight up.
    """
    zmax = math.radians(zenith_max_deg)
    th = (np.arange(n_zenith) + 0.5) * zmax / n_zenith
    ph = (np.arange(n_azimuth) + 0.5) * 2.0 * math.pi / n_azimuth
    T, F = np.meshgrid(th, ph, indexing="ij")
    d = np.stack([np.sin(T) * np.cos(F), np.sin(T) * np.sin(F), np.cos(T)], axis=-1)
    return np.ascontiguousarray(d.reshape(-1, 3))


def node_xy(w: Workload):
    """Node coordinates of the surface grid: x_c = c*Lx/(Q-1), y_r = r*Ly/(R-1)."""
    x = np.arange(w.Q) * (w.box[0] / (w.Q - 1))
    y = np.arange(w.R) * (w.box[1] / (w.R - 1))
    return np.meshgrid(x, y, indexing="xy")  # each [R][Q]


def _order_and_clip(H: np.ndarray, Lz: float, delta: float) -> np.ndarray:
    L = H.shape[0]
    out = H.copy()
    for l in range(L):
        out[l] = np.clip(out[l], (l + 1) * delta, Lz - (L - l) * delta)
    for l in range(1, L):
        out[l] = np.maximum(out[l], out[l - 1] + delta)
    return out


def geometry(w: Workload, seed) -> np.ndarray:
    """One ordered geometry [L][R][Q] (FP64): base heights plus Gaussian bumps."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))
    X, Y = node_xy(w)
    H = np.empty((w.L, w.R, w.Q))
    for l, base in enumerate(w.bases):
        h = np.full((w.R, w.Q), float(base))
        for _ in range(w.n_bumps):
            cx, cy = rng.uniform(0.0, w.box[0]), rng.uniform(0.0, w.box[1])
            h += w.bump_amp * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * w.bump_sigma ** 2))
        H[l] = h
    return _order_and_clip(H, w.box[2], w.delta)


def true_geometry(w: Workload) -> np.ndarray:
    return geometry(w, [w.seed_geom])


def prior_mean(w: Workload) -> np.ndarray:
    """Prior mean: each surface's base height, clipped like a geometry."""
    H = np.stack([np.full((w.R, w.Q), float(b)) for b in w.bases])
    return _order_and_clip(H, w.box[2], w.delta)


def init_chains(w: Workload, n_chains: int | None = None) -> np.ndarray:
    """Independent starting geometries, one per chain: [C][L][R][Q] FP64."""
    n = w.n_chains if n_chains is None else n_chains
    return np.stack([geometry(w, [w.seed_init, c]) for c in range(n)])


def problem(w: Workload) -> dict:
    """Everything a solver needs except the counts, as plain numpy arrays."""
    d = w.as_dict()
    d.update(
        box=np.asarray(w.box, np.float64),
        rho=np.asarray(w.rho, np.float64),
        sensors=np.asarray(w.sensors, np.float64).reshape(-1, 3),
        dirs=pixel_dirs(w.n_zenith, w.n_azimuth, w.zenith_max_deg),
        mu=prior_mean(w),
        H_true=true_geometry(w),
    )
    return d


def perturbed(H: np.ndarray, scale: float, seed) -> np.ndarray:
    """H plus i.i.d. N(0, scale^2) noise (a generic off-mode test input)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))
    return H + scale * rng.standard_normal(H.shape)


def serving_mix(n_requests: int, seed: int = 5, small_scale: bool = False) -> list:
    """Uneven inversion requests: grid 32^2-128^2, 3-5 surfaces, 4-32 sensors,
    32^2-96^2 pixels, 128-384 samples, 64-1024 chains, 1e3-1e4 steps, sizes
    log-uniform; Poisson arrivals at 20 per second.  small_scale shrinks every
    size for tests."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed)))

    def lu(lo, hi):
        return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))

    reqs, t = [], 0.0
    base_by_L = {3: (40.0, 70.0, 110.0), 4: (40.0, 70.0, 110.0, 140.0),
                 5: (30.0, 55.0, 80.0, 110.0, 140.0)}
    rho_by_L = {3: (ROCK, MUCK, AIR, ROCK), 4: (ROCK, MUCK, AIR, ROCK, AIR),
                5: (ROCK, MUCK, AIR, MUCK, ROCK, AIR)}
    for i in range(n_requests):
        t += rng.exponential(1.0 / 20.0)
        L = int(rng.integers(3, 6))
        if small_scale:
            g, ns, npx, G, C, steps = lu(6, 12), lu(1, 3), lu(4, 8), lu(16, 32), lu(2, 8), lu(4, 12)
        else:
            g, ns, npx, G, C, steps = lu(32, 128), lu(4, 32), lu(32, 96), lu(128, 384), lu(64, 1024), lu(1000, 10000)
        side = int(math.ceil(math.sqrt(ns)))
        sens = tuple(((a + 0.5) * 200.0 / side, (b + 0.5) * 200.0 / side, 20.0)
                     for b in range(side) for a in range(side))[:ns]
        w = Workload(name=f"req{i}", R=g, Q=g, bases=base_by_L[L], rho=rho_by_L[L], sensors=sens,
                     n_zenith=npx, n_azimuth=npx, zenith_max_deg=60.0, G=G, n_chains=C,
                     n_super=max(1, steps // 10), n_within=10 if steps >= 10 else steps,
                     seed_geom=100 + i, seed_data=200 + i, seed_init=300 + i, seed_mcmc=400 + i)
        w.extra["arrival_s"] = t
        reqs.append(w)
    return reqs
