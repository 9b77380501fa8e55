"""GAP local energies (Sec. IV.A) and their exact position/strain derivatives (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

  k(i, s)   = (q_i . q_s)^zeta                       (Sec. I, SOAP kernel)
  eps_i     = sum_{s in sparse set} alpha_s k(i, s)   (Sec. IV.A)
  E_struct  = sum of eps_i over the atoms of a structure
  F_k       = -dE/dx_k
  virial_ab = -dE/d(strain_ab), the strain acting as r_a -> r_a + strain_ab r_b on every
              position and lattice vector; for pair separations this equals
              -sum_pairs (dE/dr_ij)_a (r_ij)_b.

Fitting side (Sec. IV.A: the alpha_s are fitted to the energies of N_t environments and
their 3 N_t force components, with the environments of the sparse set as basis):
  kernel_matrix       k(i, s) for descriptor rows against the sparse set (K_NM; with the
                      sparse rows themselves, K_MM)
  structure_rows      sum of k(i, s) over each structure's atoms (energy rows)
  kernel_gradients    dk[k, a, s] = d/dx_{k,a} of that sum for the structure of atom k
                      (force rows: a model with weights alpha has F_k = -dk[k] @ alpha)

The paper gives no derivative formulas (it states its implementation lacks kernel
derivatives), so forces and virial here are the exact derivatives of the energy,
taken by PyTorch autograd through the same FP64 operations that compute it.
"""
from __future__ import annotations

import numpy as np
import torch

from . import basis, neighbours, soap
from .params import Params

DT = torch.float64


def kernel_power(s: torch.Tensor, zeta: float) -> torch.Tensor:
    """(q_i . q_s)^zeta: repeated multiplication for integer zeta; otherwise the dot
    product is clamped at 0 before the power (it lies in [0, 1] up to rounding)."""
    if float(zeta).is_integer() and zeta >= 1:
        out = s
        for _ in range(int(zeta) - 1):
            out = out * s
        return out
    return torch.clamp(s, min=0.0) ** zeta


def local_energies(q: torch.Tensor, q_sparse: torch.Tensor, alpha: torch.Tensor,
                   zeta: float) -> torch.Tensor:
    """eps_i = sum_s alpha_s (q_i . q_s)^zeta for packed descriptors q [N, D], q_sparse [M, D]."""
    return kernel_power(q @ q_sparse.T, zeta) @ alpha


def kernel_matrix(q, q_sparse, zeta: float) -> torch.Tensor:
    """k(i, s) = (q_i . q_s)^zeta for rows q [N, D] against q_sparse [M, D]: [N, M]."""
    return kernel_power(torch.as_tensor(q, dtype=DT) @ torch.as_tensor(q_sparse, dtype=DT).T, zeta)


def structure_rows(k_atom, atom_offs) -> torch.Tensor:
    """Per-structure sums of kernel rows: out[t, s] = sum over atoms i of t of k_atom[i, s]."""
    k_atom = torch.as_tensor(k_atom, dtype=DT)
    offs = np.asarray(atom_offs)
    return torch.stack([k_atom[offs[t]:offs[t + 1]].sum(dim=0) for t in range(len(offs) - 1)])


def kernel_gradients(batch, P: Params, q_sparse, zeta: float, atoms=None, sparse=None, W=None,
                     chunk: int = 64) -> np.ndarray:
    """dk[k, a, s] = d/dx_{k,a} sum_{i in the structure of k} (q_i . q_s)^zeta for the listed
    atoms k (default: all, in index order) and sparse environments s (default: all).

    Only centres i that can depend on x_k contribute: k itself and every atom with k among
    its neighbours (any image); their descriptors are taken with autograd through the same
    FP64 operations as the energy, one backward pass per sparse environment.
    Returns [len(atoms), 3, len(sparse)] (NumPy FP64).
    """
    if W is None:
        W = basis.orthonormaliser(P.n_max, P.r_cut, P.sigma_r0)
    qs_all = torch.as_tensor(np.asarray(q_sparse), dtype=DT)
    sparse = np.arange(len(qs_all)) if sparse is None else np.asarray(sparse, dtype=np.int64)
    qs = qs_all[torch.as_tensor(sparse)]
    if atoms is None:
        atoms = np.arange(batch.n_atoms)
        centers = atoms
    else:
        atoms = np.asarray(atoms, dtype=np.int64)
        near = neighbours.batch_pairs(batch, P.r_cut, centers=np.unique(atoms))
        centers = np.unique(np.concatenate([atoms, near["j"]]))
    pairs = neighbours.batch_pairs(batch, P.r_cut, centers=centers)
    pos = torch.as_tensor(batch.pos, dtype=DT).clone().requires_grad_(True)
    cell = torch.as_tensor(batch.cell, dtype=DT)
    grad = torch.zeros((len(sparse), batch.n_atoms, 3), dtype=DT)
    for c0 in range(0, len(centers), chunk):
        cc = centers[c0:c0 + chunk]
        sel = (pairs["i"] >= cc[0]) & (pairs["i"] <= cc[-1])
        sub = {k: v[sel] for k, v in pairs.items()}
        q = _local_descriptor(P, W, pos, cell, batch.species, cc, sub)
        k = kernel_matrix(q, qs, zeta)                       # [chunk, Ms]
        for t in range(len(sparse)):
            g, = torch.autograd.grad(k[:, t].sum(), pos, retain_graph=t + 1 < len(sparse))
            grad[t] += g
    return grad[:, torch.as_tensor(atoms), :].permute(1, 2, 0).numpy()


def sparse_set(batch, P: Params, indices, W=None) -> np.ndarray:
    """Packed descriptors of the chosen atoms of a (separate) structure: [M, D]."""
    d = soap.descriptors(batch, P, centers=np.asarray(indices), W=W)
    pos = np.searchsorted(d["centers"], np.asarray(indices))
    return d["q"].numpy()[pos]


def _local_descriptor(P, W, pos_t, cell_t, species, centers, pairs):
    c_re, c_im = soap.expansion_coefficients(P, W, pos_t, cell_t, species, centers, pairs)
    p = soap.power_spectrum(c_re, c_im)
    pnorm = torch.sqrt((p * p).sum(dim=(1, 2, 3)))
    return soap.pack(p / pnorm[:, None, None, None])


def evaluate(batch, P: Params, q_sparse, alpha, zeta: float, *, forces: bool = True,
             virial: bool = True, struct_weight=None, W=None, chunk: int = 128):
    """Energies and, optionally, forces and virial of a whole flattened batch.

    ``struct_weight`` [S] (default ones) weights each structure's energy in the scalar
    that is differentiated (the adjoint input dE/dE_struct).
    Returns dict(e_atom [N], e_struct [S], forces [N, 3], virial [S, 3, 3]) as NumPy FP64.
    """
    if W is None:
        W = basis.orthonormaliser(P.n_max, P.r_cut, P.sigma_r0)
    n, ns = batch.n_atoms, batch.n_struct
    pairs = neighbours.batch_pairs(batch, P.r_cut)
    struct_of = np.repeat(np.arange(ns), np.diff(batch.atom_offs))
    if struct_weight is None:
        struct_weight = np.ones(ns)
    sw = torch.as_tensor(np.asarray(struct_weight, dtype=np.float64))
    qs = torch.as_tensor(np.asarray(q_sparse), dtype=DT)
    al = torch.as_tensor(np.asarray(alpha), dtype=DT)
    pos0 = torch.as_tensor(batch.pos, dtype=DT)
    cell0 = torch.as_tensor(batch.cell, dtype=DT)
    pos = pos0.clone().requires_grad_(forces)
    strain = torch.zeros((ns, 3, 3), dtype=DT, requires_grad=virial)
    e_atom = np.zeros(n)
    centers_all = np.arange(n)
    for c0 in range(0, n, chunk):
        cc = centers_all[c0:c0 + chunk]
        sel = (pairs["i"] >= cc[0]) & (pairs["i"] <= cc[-1])
        sub = {k: v[sel] for k, v in pairs.items()}
        sa = torch.as_tensor(struct_of)
        pos_s = pos + torch.einsum("kab,kb->ka", strain[sa], pos)
        cell_s = cell0 + torch.einsum("sab,srb->sra", strain, cell0)
        q = _local_descriptor(P, W, pos_s, cell_s, batch.species, cc, sub)
        eps = local_energies(q, qs, al, zeta)
        e_atom[cc] = eps.detach().numpy()
        if forces or virial:
            (eps * sw[torch.as_tensor(struct_of[cc])]).sum().backward()
    e_struct = np.array([e_atom[batch.atom_offs[s]:batch.atom_offs[s + 1]].sum()
                         for s in range(ns)])
    out = {"e_atom": e_atom, "e_struct": e_struct}
    if forces:
        out["forces"] = -pos.grad.numpy()
    if virial:
        out["virial"] = -strain.grad.numpy()
    return out


def forces_at(batch, P: Params, q_sparse, alpha, zeta: float, atoms, W=None, chunk: int = 64):
    """Forces on a few atoms of a large batch: F_k = -d/dx_k of the sum of eps_i over the
    centres i that can depend on x_k (k itself and every centre within r_cut of it)."""
    if W is None:
        W = basis.orthonormaliser(P.n_max, P.r_cut, P.sigma_r0)
    atoms = np.unique(np.asarray(atoms, dtype=np.int64))
    near = neighbours.batch_pairs(batch, P.r_cut, centers=atoms)
    centers = np.unique(np.concatenate([atoms, near["j"]]))
    pairs = neighbours.batch_pairs(batch, P.r_cut, centers=centers)
    qs = torch.as_tensor(np.asarray(q_sparse), dtype=DT)
    al = torch.as_tensor(np.asarray(alpha), dtype=DT)
    pos = torch.as_tensor(batch.pos, dtype=DT).clone().requires_grad_(True)
    cell = torch.as_tensor(batch.cell, dtype=DT)
    for c0 in range(0, len(centers), chunk):
        cc = centers[c0:c0 + chunk]
        sel = (pairs["i"] >= cc[0]) & (pairs["i"] <= cc[-1])
        sub = {k: v[sel] for k, v in pairs.items()}
        q = _local_descriptor(P, W, pos, cell, batch.species, cc, sub)
        local_energies(q, qs, al, zeta).sum().backward()
    return -pos.grad.numpy()[atoms], atoms
