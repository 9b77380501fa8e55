"""Brute-force periodic neighbour search (oracle side).

The atomic density of atom i collects every atom j, in every periodic image S, with
|r_j + S.h - r_i| < r_cut; atom i itself is counted once as the central atom (Sec. I:
the sum runs over atoms inside the cutoff sphere "possibly including i itself"), so
the pair (i, i, S = 0) is excluded here and added as the central term, while the
periodic self-images (i, i, S != 0) are ordinary neighbours.

The separation vector is evaluated in FP64 with one fixed operation order and no
fused multiply-add, so that the pair set is reproducible bit for bit:
    s   = (S1*h1 + S2*h2) + S3*h3        (per Cartesian component)
    r   = (x_j + s) - x_i                 when (i, j, S) is in canonical orientation,
    r   = -((x_i + (-s)) - x_j)           otherwise,
    d^2 = (r_x*r_x + r_y*r_y) + r_z*r_z,  kept when d^2 < r_cut^2 (strict).
The canonical orientation is i < j, or i == j with S lexicographically positive.
Evaluating both (i, j, S) and (j, i, -S) through the same orientation makes the pair
set exactly symmetric, with r_ji = -r_ij bit for bit.
Pairs are listed in canonical order: by centre i, then species of j, then j, then
(S1, S2, S3) lexicographically.
"""
from __future__ import annotations

import math

import numpy as np


def image_range(cell: np.ndarray, r_cut: float) -> np.ndarray:
    """Number of images needed along each lattice vector: ceil(r_cut / d_k) where d_k
    is the spacing of the lattice planes spanned by the other two vectors."""
    vol = abs(np.linalg.det(cell))
    n = []
    for k in range(3):
        a, b = cell[(k + 1) % 3], cell[(k + 2) % 3]
        d = vol / np.linalg.norm(np.cross(a, b))
        n.append(int(math.ceil(r_cut / d)))
    return np.array(n, dtype=np.int64)


def _lex_positive(shifts: np.ndarray) -> np.ndarray:
    """S > 0 in lexicographic order of (S1, S2, S3)."""
    s1, s2, s3 = shifts[:, 0], shifts[:, 1], shifts[:, 2]
    return (s1 > 0) | ((s1 == 0) & ((s2 > 0) | ((s2 == 0) & (s3 > 0))))


def structure_pairs(pos: np.ndarray, cell: np.ndarray, species: np.ndarray, r_cut: float,
                    centers=None, block: int = 64):
    """All pairs (i, j, S) of one structure with |r_ij| < r_cut, excluding (i, i, 0).

    ``centers`` (optional) restricts the centres i; j still runs over every atom.
    Returns (i, j, S[P, 3] int64, r[P, 3] float64) in canonical order.
    """
    pos = np.asarray(pos, dtype=np.float64)
    cell = np.asarray(cell, dtype=np.float64)
    n = pos.shape[0]
    rc2 = r_cut * r_cut
    nr = image_range(cell, r_cut)
    shifts = np.array([(a, b, c)
                       for a in range(-nr[0], nr[0] + 1)
                       for b in range(-nr[1], nr[1] + 1)
                       for c in range(-nr[2], nr[2] + 1)], dtype=np.int64)
    sf = shifts.astype(np.float64)
    svec = (sf[:, 0:1] * cell[0][None, :] + sf[:, 1:2] * cell[1][None, :]) \
        + sf[:, 2:3] * cell[2][None, :]                               # [nS, 3]
    zero_shift = np.all(shifts == 0, axis=1)
    if centers is None:
        centers = np.arange(n)
    centers = np.asarray(centers, dtype=np.int64)
    out_i, out_j, out_s, out_r = [], [], [], []
    block = max(1, min(block, 4_000_000 // (len(shifts) * max(n, 1))))
    for b0 in range(0, len(centers), block):
        ci = centers[b0:b0 + block]
        xi = pos[ci][:, None, None, :]                                # [b, 1, 1, 3]
        xj = pos[None, None, :, :]                                    # [1, 1, N, 3]
        sv = svec[None, :, None, :]                                   # [1, nS, 1, 3]
        r_can = (xj + sv) - xi
        r_alt = -((xi + (-sv)) - xj)
        jj = np.arange(n)[None, None, :]
        lexpos = _lex_positive(shifts)[None, :, None]
        canon = (jj > ci[:, None, None]) | ((jj == ci[:, None, None]) & lexpos)
        r = np.where(canon[..., None], r_can, r_alt)                  # [b, nS, N, 3]
        d2 = (r[..., 0] * r[..., 0] + r[..., 1] * r[..., 1]) + r[..., 2] * r[..., 2]
        keep = d2 < rc2
        keep &= ~(zero_shift[None, :, None] & (np.arange(n)[None, None, :] == ci[:, None, None]))
        bi, bs, bj = np.nonzero(keep)
        out_i.append(ci[bi])
        out_j.append(bj)
        out_s.append(shifts[bs])
        out_r.append(r[bi, bs, bj])
    i = np.concatenate(out_i) if out_i else np.zeros(0, np.int64)
    j = np.concatenate(out_j) if out_j else np.zeros(0, np.int64)
    s = np.concatenate(out_s) if out_s else np.zeros((0, 3), np.int64)
    r = np.concatenate(out_r) if out_r else np.zeros((0, 3), np.float64)
    order = np.lexsort((s[:, 2], s[:, 1], s[:, 0], j, species[j], i))
    return i[order], j[order], s[order], r[order]


def batch_pairs(batch, r_cut: float, centers=None):
    """Pairs of every structure of a flattened batch, with global atom indices.

    ``centers`` (optional, global indices) restricts the centres.
    Returns dict(i, j, shift, r, struct) in canonical order.
    """
    outs = {k: [] for k in ("i", "j", "shift", "r", "struct")}
    for s in range(batch.n_struct):
        a, b = int(batch.atom_offs[s]), int(batch.atom_offs[s + 1])
        if centers is None:
            loc = None
        else:
            c = np.asarray(centers)
            loc = c[(c >= a) & (c < b)] - a
            if len(loc) == 0:
                continue
        i, j, sh, r = structure_pairs(batch.pos[a:b], batch.cell[s], batch.species[a:b],
                                      r_cut, centers=loc)
        outs["i"].append(i + a)
        outs["j"].append(j + a)
        outs["shift"].append(sh)
        outs["r"].append(r)
        outs["struct"].append(np.full(len(i), s, dtype=np.int64))
    res = {}
    for k, v in outs.items():
        if v:
            res[k] = np.concatenate(v)
        else:
            res[k] = np.zeros((0, 3) if k in ("shift", "r") else 0,
                              dtype=np.float64 if k == "r" else np.int64)
    return res
