"""The standard workloads, named by what they are.

Each entry fixes the structures (through seeds and sizes), the descriptor
hyperparameters and the GAP model inputs (sparse-set box, its selection and the
weights).  Values are plain numbers; nothing here computes a descriptor.

Hyperparameters not fixed by the workload description default to: a single
"atom sigma" for both channels (sigma_r0 = sigma_p0), no radial growth of the
widths (alpha_r = alpha_p = 0), amplitude exponent a = 1, a 0.5 Angstrom buffer
zone ending at r_cut, filter parameter n_f = 4 and the central atom counted once.
"""
from __future__ import annotations

from dataclasses import dataclass, field

from .boxes import Batch, batched_boxes, concat, random_box


@dataclass(frozen=True)
class Workload:
    name: str
    description: str
    # structures
    kind: str                 # "box" or "batch"
    n_atoms: int = 0
    side: float | None = None
    density: float | None = None
    dmin: float = 1.2
    seed: int = 0
    species_probs: tuple | None = None
    n_struct: int = 1
    n_lo: int = 16
    n_hi: int = 2000
    rho_lo: float = 0.08
    rho_hi: float = 0.18
    # descriptor hyperparameters
    r_cut: float = 5.0
    buffer: float = 0.5
    sigma: float = 0.5
    n_max: int = 8
    l_max: int = 8
    n_species: int = 1
    # GAP model
    n_sparse: int = 0
    sparse_box_atoms: int = 0
    sparse_box_density: float = 0.15
    sparse_box_dmin: float = 1.2
    sparse_seed: int = 0
    alpha_seed: int = 0
    zeta: float = 4.0
    extra: dict = field(default_factory=dict)

    def params(self) -> dict:
        """Descriptor hyperparameters as a plain dict (same keys as the C-ABI struct)."""
        return dict(r_cut=self.r_cut, r_soft=self.r_cut - self.buffer,
                    sigma_r0=self.sigma, sigma_p0=self.sigma, alpha_r=0.0, alpha_p=0.0,
                    amp_a=1.0, n_f=4.0, central_weight=1.0, n_max=self.n_max,
                    l_max=self.l_max, n_species=self.n_species)

    def structures(self) -> Batch:
        if self.kind == "box":
            s = random_box(self.n_atoms, side=self.side, density=self.density,
                           dmin=self.dmin, seed=self.seed, species_probs=self.species_probs)
            return concat([s])
        return batched_boxes(self.n_struct, n_lo=self.n_lo, n_hi=self.n_hi,
                             rho_lo=self.rho_lo, rho_hi=self.rho_hi, dmin=self.dmin,
                             seed=self.seed)

    def sparse_box(self) -> Batch:
        """The separate box whose atoms provide the sparse-set environments."""
        s = random_box(self.sparse_box_atoms, density=self.sparse_box_density,
                       dmin=self.sparse_box_dmin, seed=self.sparse_seed,
                       species_probs=self.species_probs)
        return concat([s])


WORKLOADS = {
    w.name: w for w in [
        Workload(
            name="box64_n6l6",
            description="64-atom periodic cube, side 8.0 A, dmin 1.2 A, r_cut 3.7 A, "
                        "sigma 0.5 A, n_max = l_max = 6 (descriptors, FP64)",
            kind="box", n_atoms=64, side=8.0, dmin=1.2, seed=1, r_cut=3.7, sigma=0.5,
            n_max=6, l_max=6, n_sparse=32, sparse_box_atoms=64, sparse_box_density=0.125,
            sparse_seed=101, alpha_seed=201, zeta=4.0),
        Workload(
            name="box1000_n8l8",
            description="1000-atom periodic cube at 0.15 atoms/A^3, dmin 1.2 A, r_cut 5.0 A, "
                        "sigma 0.5 A, n_max = l_max = 8 (descriptors and forces)",
            kind="box", n_atoms=1000, density=0.15, dmin=1.2, seed=2, r_cut=5.0, sigma=0.5,
            n_max=8, l_max=8, n_sparse=500, sparse_box_atoms=1000, sparse_box_density=0.15,
            sparse_seed=102, alpha_seed=202, zeta=4.0),
        Workload(
            name="twospecies4096_n8l8",
            description="4096-atom two-species periodic cube (70/30), 0.10 atoms/A^3, dmin "
                        "1.0 A, r_cut 5.0 A, n_max = 8 per species, l_max = 8, 2000 sparse "
                        "environments, zeta 4 (GAP energy and forces)",
            kind="box", n_atoms=4096, density=0.10, dmin=1.0, seed=3,
            species_probs=(0.7, 0.3), r_cut=5.0, sigma=0.5, n_max=8, l_max=8, n_species=2,
            n_sparse=2000, sparse_box_atoms=4096, sparse_box_density=0.10,
            sparse_box_dmin=1.0, sparse_seed=103, alpha_seed=203, zeta=4.0),
        Workload(
            name="batch256_n8l8",
            description="256 periodic cubes, 16-2000 atoms (log-uniform), 0.08-0.18 "
                        "atoms/A^3, r_cut 4.5 A, n_max = l_max = 8, 1000 sparse "
                        "environments, zeta 2 (batched GAP energy and forces)",
            kind="batch", n_struct=256, n_lo=16, n_hi=2000, rho_lo=0.08, rho_hi=0.18,
            dmin=1.2, seed=4, r_cut=4.5, sigma=0.5, n_max=8, l_max=8, n_sparse=1000,
            sparse_box_atoms=2000, sparse_box_density=0.13, sparse_seed=104,
            alpha_seed=204, zeta=2.0),
        Workload(
            name="box100k_n10l10",
            description="100,000-atom periodic cube at 0.15 atoms/A^3, dmin 1.2 A, r_cut 5.0 A, "
                        "n_max = l_max = 10, 4000 sparse environments, zeta 4 (one MD-step "
                        "evaluation: energies, forces, virial)",
            kind="box", n_atoms=100_000, density=0.15, dmin=1.2, seed=5, r_cut=5.0,
            sigma=0.5, n_max=10, l_max=10, n_sparse=4000, sparse_box_atoms=8000,
            sparse_box_density=0.15, sparse_seed=105, alpha_seed=205, zeta=4.0),
    ]
}


def get_workload(name: str) -> Workload:
    try:
        return WORKLOADS[name]
    except KeyError:
        raise KeyError(f"unknown workload {name!r}; known: {sorted(WORKLOADS)}") from None
