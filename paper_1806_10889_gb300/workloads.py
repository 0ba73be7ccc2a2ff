"""Seeded synthetic workloads of the tissue SSA.

This module only *describes* inputs: tissue geometry, seeds, Poisson means of
the initial counts and model rates.  It holds none of the method's arithmetic
and imports neither the CUDA binding nor the oracle, so both sides can take
their inputs from here.

The paper's experiments use synthetic tissues only: identical cubic cells in a
2-D layer with at most four neighbours (Sec. III-A1), 8x8 cells for strong
scaling and 100 cells per node for weak scaling (Sec. III-C).  The workloads
below keep that structure (square cell grids, every cell an n x n voxel
lattice, per-tissue seeds) at the sizes of this build's benchmark suite.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

# Notch-Delta lattice model: Delta production 10/(1+(R/20)^2) per voxel, Notch
# production 5 per voxel, decay 0.1 (D, N) and 0.2 (R), hop rate 1.0 per
# molecule and direction, face binding 0.01*D*N producing one R in the cell
# that gave the Notch.  k_in / k_off (in-voxel D+N <-> R) are test-only.
ND_MODEL = dict(kD=10.0, K=20.0, kN=5.0, gD=0.1, gN=0.1, gR=0.2,
                hopD=1.0, hopN=1.0, hopR=1.0, k_in=0.0, k_off=0.0, k_bind=0.01)


@dataclass(frozen=True)
class TissueSpec:
    """One tissue: geometry, random key and model (plain numbers only)."""
    width: int
    height: int
    n: int
    seed: int
    tissue_id: int = 0
    init_lambda: tuple = (5.0, 5.0, 5.0)
    model: dict = field(default_factory=lambda: dict(ND_MODEL))

    @property
    def cells(self) -> int:
        return self.width * self.height

    @property
    def V(self) -> int:
        return self.n * self.n

    @property
    def state_ints(self) -> int:
        return self.cells * 3 * self.V

    def with_model(self, **kw) -> "TissueSpec":
        m = dict(self.model)
        m.update(kw)
        return replace(self, model=m)


@dataclass(frozen=True)
class Run:
    tissue: TissueSpec
    dt: float
    n_steps: int


def tiny() -> Run:
    """2x2 tissue of 8x8-voxel cells, seed 1, dt = 0.1, T = 10 (100 steps)."""
    return Run(TissueSpec(2, 2, 8, seed=1, tissue_id=0), dt=0.1, n_steps=100)


def medium(dt: float = 0.1) -> Run:
    """64x64 tissue (4096 cells) of 16x16-voxel cells, seed 2, T = 50."""
    if dt not in (0.01, 0.1, 1.0):
        raise ValueError("medium tissue is defined for dt in {0.01, 0.1, 1.0}")
    return Run(TissueSpec(64, 64, 16, seed=2, tissue_id=0), dt=dt,
               n_steps=int(round(50.0 / dt)))


def large() -> Run:
    """256x256 tissue (65536 cells) of 32x32-voxel cells, seed 4, dt 0.1, T = 100."""
    return Run(TissueSpec(256, 256, 32, seed=4, tissue_id=0), dt=0.1, n_steps=1000)


def batch(count: int = 256) -> list[Run]:
    """Uneven tissues: side ~ U{2..64} cells, n in {8,16,32}, kD ~ U[5,20].

    Seed 3 for the generator and for every tissue's Philox key; tissue_id is
    the tissue's index, so each tissue's stream is intrinsic to it.
    dt = 0.1, T = 20 (200 steps).
    """
    rng = np.random.default_rng(3)
    side = rng.integers(2, 65, size=count)
    n = rng.choice(np.array([8, 16, 32]), size=count)
    kD = rng.uniform(5.0, 20.0, size=count)
    runs = []
    for i in range(count):
        spec = TissueSpec(int(side[i]), int(side[i]), int(n[i]), seed=3, tissue_id=i)
        runs.append(Run(spec.with_model(kD=float(kD[i])), dt=0.1, n_steps=200))
    return runs


@dataclass(frozen=True)
class Request:
    index: int
    arrival_s: float
    replicas: int
    side: int
    n: int
    n_steps: int
    dt: float

    def replica_specs(self) -> list[TissueSpec]:
        # request seed = request index, tissue_id = replica index
        return [TissueSpec(self.side, self.side, self.n, seed=self.index, tissue_id=r)
                for r in range(self.replicas)]


def serving(count: int = 500, rate_per_s: float = 50.0, T: float = 20.0,
            dt: float = 0.1) -> list[Request]:
    """Poisson arrivals (mean gap 1/rate), 1..64 replicas per request, side
    ~ lognormal(median 16 cells, sigma 0.8) clamped to [2, 128], 16x16 voxels."""
    rng = np.random.default_rng(5)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    arrivals = np.cumsum(gaps)
    replicas = rng.integers(1, 65, size=count)
    side = np.clip(np.rint(rng.lognormal(math.log(16.0), 0.8, size=count)), 2, 128)
    n_steps = int(round(T / dt))
    return [Request(i, float(arrivals[i]), int(replicas[i]), int(side[i]), 16, n_steps, dt)
            for i in range(count)]
