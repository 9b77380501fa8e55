"""Random periodic boxes by random sequential addition (RSA) with a minimum distance.

Every generator takes an explicit integer seed and uses ``numpy.random.default_rng``
(PCG64), whose stream is identical on x86-64 and AArch64, so the same structure is
produced on every machine.  Distances are compared squared (no square roots), so the
accept/reject decisions are exactly reproducible too.

Conventions shared with the library and the oracle:
  * ``cell`` rows are the lattice vectors (Angstrom);
  * positions are Cartesian (Angstrom) and lie inside the cell: their fractional
    coordinates ``pos @ inv(cell)`` are in [0, 1);
  * ``species`` are int32 in [0, n_species).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Structure:
    pos: np.ndarray      # [N, 3] float64
    cell: np.ndarray     # [3, 3] float64, rows = lattice vectors
    species: np.ndarray  # [N] int32

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])


@dataclass
class Batch:
    """Several periodic structures stored back to back (flattened atom arrays)."""
    pos: np.ndarray        # [N_total, 3] float64
    cell: np.ndarray       # [S, 3, 3] float64
    species: np.ndarray    # [N_total] int32
    atom_offs: np.ndarray  # [S + 1] int64

    @property
    def n_struct(self) -> int:
        return int(self.cell.shape[0])

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])

    def structure(self, s: int) -> Structure:
        a, b = int(self.atom_offs[s]), int(self.atom_offs[s + 1])
        return Structure(self.pos[a:b], self.cell[s], self.species[a:b])


def _rsa_cubic(n: int, side: float, dmin: float, rng: np.random.Generator,
               max_proposals: int) -> np.ndarray:
    """Sequential random addition of ``n`` points in a periodic cube.

    Candidates are drawn uniformly, in order, and a candidate is kept when its
    minimum-image distance to every point kept before it is at least ``dmin``.
    Candidates are drawn in blocks for speed; inside a block they are still
    resolved in order, so the result equals one-at-a-time insertion.
    """
    g = max(1, int(np.floor(side / dmin)))  # grid cells per edge, edge >= dmin
    cap = 16
    grid = -np.ones((g, g, g, cap), dtype=np.int64)
    fill = np.zeros((g, g, g), dtype=np.int64)
    out = np.empty((n, 3), dtype=np.float64)
    kept = 0
    proposed = 0
    d2min = dmin * dmin
    offs = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)],
                    dtype=np.int64)

    def min_image(d):
        return d - side * np.round(d / side)

    while kept < n:
        if proposed > max_proposals:
            raise RuntimeError(f"RSA: could not place {n} atoms in a {side:.3f} A box "
                               f"with dmin={dmin} after {proposed} proposals")
        k = int(min(1024, 2 * (n - kept) + 64))
        cand = rng.random((k, 3)) * side
        proposed += k
        cc = np.minimum((cand / side * g).astype(np.int64), g - 1)
        ok = np.ones(k, dtype=bool)
        if kept > 0:
            nb = (cc[:, None, :] + offs[None, :, :]) % g              # [k, 27, 3]
            idx = grid[nb[..., 0], nb[..., 1], nb[..., 2]]             # [k, 27, cap]
            idx = idx.reshape(k, -1)
            valid = idx >= 0
            pj = out[np.where(valid, idx, 0)]                          # [k, 27*cap, 3]
            d = min_image(pj - cand[:, None, :])
            d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
            ok = ~np.any(valid & (d2 < d2min), axis=1)
        surv = np.nonzero(ok)[0]
        accepted = np.ones(len(surv), dtype=bool)
        if len(surv) > 1:
            cs = cand[surv]
            d = min_image(cs[None, :, :] - cs[:, None, :])
            d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
            clash = np.tril(d2 < d2min, k=-1)     # clash[j, i]: i < j conflict
            for j in np.nonzero(clash.any(axis=1))[0]:
                if np.any(accepted[:j] & clash[j, :j]):
                    accepted[j] = False
        batch_kept = [int(t) for t in surv[accepted][: n - kept]]
        for t in batch_kept:
            a, b, c = cc[t]
            f = fill[a, b, c]
            if f >= cap:
                raise RuntimeError("RSA grid cell overflow")
            grid[a, b, c, f] = kept
            fill[a, b, c] = f + 1
            out[kept] = cand[t]
            kept += 1
    return out


def random_box(n_atoms: int, *, side: float | None = None, density: float | None = None,
               dmin: float = 1.2, seed: int = 0, species_probs=None,
               shear: float = 0.0) -> Structure:
    """A periodic box of ``n_atoms`` random atoms kept at least ``dmin`` apart.

    Give either ``side`` (cube edge, Angstrom) or ``density`` (atoms per cubic
    Angstrom).  ``species_probs`` (default: one species) assigns each atom a species
    by an independent draw after the positions.  ``shear`` > 0 maps the cube onto a
    triclinic cell (x += shear*y + shear*z); the minimum distance is then only
    approximate, which is fine for tests of cell handling.
    """
    if (side is None) == (density is None):
        raise ValueError("give exactly one of side / density")
    if side is None:
        side = float((n_atoms / density) ** (1.0 / 3.0))
    rng = np.random.default_rng(seed)
    pos = _rsa_cubic(n_atoms, side, dmin, rng, max_proposals=400 * n_atoms + 10000)
    cell = np.eye(3) * side
    if species_probs is None:
        species = np.zeros(n_atoms, dtype=np.int32)
    else:
        p = np.asarray(species_probs, dtype=np.float64)
        p = p / p.sum()
        u = rng.random(n_atoms)
        species = np.searchsorted(np.cumsum(p)[:-1], u, side="right").astype(np.int32)
    if shear:
        m = np.array([[1.0, 0.0, 0.0], [shear, 1.0, 0.0], [shear, 0.0, 1.0]])
        # fractional coordinates are kept: pos = frac @ cell with the new cell
        frac = pos / side
        cell = m @ cell
        pos = frac @ cell
    return Structure(pos=np.ascontiguousarray(pos), cell=np.ascontiguousarray(cell),
                     species=species)


def concat(structs) -> Batch:
    """Stack structures into one flattened batch."""
    n = [s.n_atoms for s in structs]
    offs = np.zeros(len(structs) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(n)
    return Batch(pos=np.ascontiguousarray(np.concatenate([s.pos for s in structs])),
                 cell=np.ascontiguousarray(np.stack([s.cell for s in structs])),
                 species=np.ascontiguousarray(np.concatenate([s.species for s in structs])),
                 atom_offs=offs)


def batched_boxes(n_struct: int, *, n_lo: int = 16, n_hi: int = 2000, rho_lo: float = 0.08,
                  rho_hi: float = 0.18, dmin: float = 1.2, seed: int = 0) -> Batch:
    """Many periodic cubes of uneven size: atom counts log-uniform in [n_lo, n_hi],
    number densities uniform in [rho_lo, rho_hi]."""
    rng = np.random.default_rng(seed)
    counts = np.rint(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=n_struct))).astype(int)
    rhos = rng.uniform(rho_lo, rho_hi, size=n_struct)
    sub = rng.integers(0, 2**31 - 1, size=n_struct)
    structs = [random_box(int(c), density=float(r), dmin=dmin, seed=int(s))
               for c, r, s in zip(counts, rhos, sub)]
    return concat(structs)


def sparse_indices(n_atoms: int, m: int, seed: int) -> np.ndarray:
    """``m`` distinct atom indices (sorted) for a GAP sparse set."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_atoms, size=m, replace=False)).astype(np.int64)


def gap_weights(m: int, seed: int, variance: float = 0.01) -> np.ndarray:
    """GAP coefficients alpha_s ~ N(0, variance)."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, np.sqrt(variance), size=m)


def random_rotation(seed: int, reflect: bool = False) -> np.ndarray:
    """A random orthogonal 3x3 matrix (det +1, or -1 with ``reflect``)."""
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    if reflect:
        q = q @ np.diag([1.0, 1.0, -1.0])
    return q
