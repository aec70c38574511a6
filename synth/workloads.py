"""Workload parameter sets (lattice, gauge spread, hopping parameter, levels).

Only numbers live here.  Degrees follow the convention used throughout the
library: a polynomial p of degree D comes from a GMRES cycle of length
m = D + 1 (m harmonic Ritz values); a double polynomial (m_in, m_out) has
p_double of degree m_in*m_out - 1 and residual polynomial of degree
m_in*m_out.

Levels are listed from the most expensive (top, M^-1 minus the highest
degree polynomial) to the cheapest Monte Carlo level; the last polynomial is
traced exactly.
"""
from dataclasses import dataclass, field


@dataclass(frozen=True)
class Workload:
    name: str
    dims: tuple            # (Lx, Ly, Lz, Lt)
    eps: float             # gauge spread
    kappa: float
    gauge_seed: int
    noise_seed: int
    polys: tuple           # ("single", m) or ("double", m_in, m_out), highest degree first
    noises: tuple          # noise count per Monte Carlo level, top level first
    thetas: tuple          # operator insertions: "1" and/or "g4"
    deflate_k: int
    t_antiperiodic: int = 1
    precision: str = "f64"
    notes: str = ""

    @property
    def volume(self):
        v = 1
        for d in self.dims:
            v *= d
        return v


WORKLOADS = {
    "c1_4x4x4x4": Workload(
        name="c1_4x4x4x4", dims=(4, 4, 4, 4), eps=0.5, kappa=0.12, gauge_seed=1, noise_seed=0,
        polys=(("single", 16),), noises=(32,), thetas=("1",), deflate_k=0,
        notes="plain MMC: Tr(M^-1 - p) by 32 noises + exact Tr(p), vs dense LU"),
    "c2_8x8x8x8": Workload(
        name="c2_8x8x8x8", dims=(8, 8, 8, 8), eps=0.3, kappa=0.155, gauge_seed=1, noise_seed=1,
        polys=(("double", 20, 10), ("single", 51), ("single", 11)), noises=(64, 64, 64),
        thetas=("1", "g4"), deflate_k=10,
        notes="full multilevel MMC in FP64"),
    "c3_16x16x16x16": Workload(
        name="c3_16x16x16x16", dims=(16, 16, 16, 16), eps=0.3, kappa=0.155, gauge_seed=1,
        noise_seed=2, polys=(("double", 20, 10), ("single", 51), ("single", 11)),
        noises=(256, 256, 256), thetas=("1",), deflate_k=40, precision="bf16",
        notes="precision form: FP32 arithmetic, BF16 spinor storage, refined solves"),
    "c4_24x24x24x24": Workload(
        name="c4_24x24x24x24", dims=(24, 24, 24, 24), eps=0.25, kappa=0.1565, gauge_seed=1,
        noise_seed=3, polys=(("double", 40, 8), ("single", 129), ("single", 33), ("single", 9)),
        noises=(8, 32, 128, 512), thetas=("1",), deflate_k=100, precision="bf16",
        notes="batched form: all levels in one captured launch sequence"),
}
