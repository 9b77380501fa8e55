"""Shared helpers of the GPU parity tests: oracle models and error measures.

Error measures (relative, scale-invariant):
  descriptors  max over atoms of |p_gpu - p_ref| / |p_ref| (p = q |p|, packed layout)
  energies     |dE_struct| / |E_struct| per structure (max) and |d eps|_2 / |eps|_2
  forces       |dF|_2 / |F|_2 over all components
"""
from __future__ import annotations

import functools

import numpy as np

import synth
from oracle import Params, basis, gap


def rel_rows(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))


def rel_all(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@functools.lru_cache(maxsize=None)
def oracle_W(n_max, r_cut, sigma_r0):
    return basis.orthonormaliser(n_max, r_cut, sigma_r0)


@functools.lru_cache(maxsize=None)
def sparse_model(name: str, m: int | None = None):
    """Oracle sparse-set descriptors and weights of a named workload (m overrides size)."""
    w = synth.get_workload(name)
    P = Params.from_dict(w.params())
    m = w.n_sparse if m is None else m
    sb = w.sparse_box()
    idx = synth.sparse_indices(sb.n_atoms, m, w.sparse_seed)
    qs = gap.sparse_set(sb, P, idx, W=oracle_W(P.n_max, P.r_cut, P.sigma_r0))
    al = synth.gap_weights(m, w.alpha_seed)
    return P, qs, al, w.zeta
