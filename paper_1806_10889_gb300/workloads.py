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


# The paper's Notch model (Sec. III-A1, Table I): diffusion constant 1e-12 m^2/s,
# transcription t_D = 100/s, DNA binding k_a = 1e-18 m^3/s, unbinding
# k_d = 25/s, Delta -> NICD k_N = 1/s; every species but DNA decays at a rate d
# the paper does not give (1/s here).  Cells are cubes of side 1 um (the
# network file's "wsize", Fig. 2).  On an n x n lattice each voxel is a column
# of h x h x L (h = L/n), so the hop rate per direction is D/h^2 = n^2 per s
# and the binding rate per NICD molecule in the promoter's voxel is
# k_a / (h^2 L) = n^2 per s.  Time unit: seconds, dt = 0.1 s (the network
# file's end_time).
CELL_SIDE_M = 1e-6
TABLE1 = dict(D=1e-12, tD=100.0, ka=1e-18, kd=25.0, kN=1.0)
PROMOTER_DECAY = 1.0


def promoter_model(n: int, d: float = PROMOTER_DECAY) -> dict:
    """Table I in lattice units for cells of n x n voxels (see above)."""
    h = CELL_SIDE_M / n
    return dict(kind="promoter", tD=TABLE1["tD"], ka=TABLE1["ka"] / (h * h * CELL_SIDE_M),
                kd=TABLE1["kd"], kN=TABLE1["kN"], d=d, hop=TABLE1["D"] / (h * h))


def is_promoter(model: dict) -> bool:
    return model.get("kind") == "promoter"


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
    # chi per cell: "lattice" (every cell a voxel lattice), "well_mixed" (every
    # cell well mixed) or "edge:K" (lattice within K cells of the tissue's
    # edge, well mixed inside: detail where cells signal, Sec. IV)
    fidelity: str = "lattice"

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


def fidelity_mask(spec: TissueSpec):
    """uint8 per cell, 1 = well-mixed chi; None when every cell is a lattice."""
    if spec.fidelity == "lattice":
        return None
    if spec.fidelity == "well_mixed":
        return np.ones(spec.cells, dtype=np.uint8)
    if spec.fidelity.startswith("edge:"):
        k = int(spec.fidelity.split(":", 1)[1])
        cx = np.arange(spec.width)[None, :]
        cy = np.arange(spec.height)[:, None]
        edge = np.minimum(np.minimum(cx, spec.width - 1 - cx), np.minimum(cy, spec.height - 1 - cy))
        return (edge >= k).astype(np.uint8).ravel()
    raise ValueError(f"unknown fidelity {spec.fidelity!r}")


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


def promoter(side: int = 64, n: int = 16, dt: float = 0.1, n_steps: int = 500) -> Run:
    """The promoter model on a side x side tissue of n x n-voxel cells, seed 6.
    Initial Delta and NICD Poisson(0.2) and Poisson(0.05) per voxel (about
    the steady state of 16x16 cells: ~50 Delta and ~12 NICD per cell), every
    promoter free."""
    spec = TissueSpec(side, side, n, seed=6, tissue_id=0, init_lambda=(0.2, 0.05, 0.0),
                      model=promoter_model(n))
    return Run(spec, dt=dt, n_steps=n_steps)


def mixed_fidelity(side: int = 64, n: int = 16, edge: int = 8, dt: float = 0.1,
                   n_steps: int = 500) -> Run:
    """The promoter tissue with lattice cells within `edge` cells of the
    tissue's edge and well-mixed cells inside (2304 of 4096 at the defaults)."""
    r = promoter(side, n, dt, n_steps)
    return Run(replace(r.tissue, fidelity=f"edge:{edge}"), dt=dt, n_steps=n_steps)


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
