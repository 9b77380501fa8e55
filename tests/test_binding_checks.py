"""Argument checks of the Python binding that run before any library call (no GPU).

The library reads positions and species as device arrays of n_atoms entries, so the
binding refuses host tensors, wrong dtypes and shapes, and mismatched batch metadata.
"""
import numpy as np
import pytest
import torch

from paper_1905_02142_gb300.api import Structures


def cpu_structures(n=4, n_struct=1):
    offs = np.linspace(0, n, n_struct + 1).astype(np.int64)
    return Structures(np.zeros((n, 3)), np.tile(np.eye(3) * 5.0, (n_struct, 1, 1)),
                      np.zeros(n, np.int32), offs, device="cpu")


def test_host_tensors_are_refused():
    with pytest.raises(ValueError, match="pos must be a contiguous CUDA"):
        cpu_structures().c_batch()


@pytest.mark.parametrize("kw, msg", [
    (dict(pos=np.zeros((4, 2))), "pos must be"),
    (dict(species=np.zeros(3, np.int32)), "species must be"),
    (dict(atom_offs=[0, 2, 4]), "atom_offs must be"),
])
def test_shapes_are_checked(kw, msg):
    args = dict(pos=np.zeros((4, 3)), cell=np.eye(3) * 5.0, species=np.zeros(4, np.int32),
                atom_offs=[0, 4])
    args.update(kw)
    with pytest.raises(ValueError, match=msg):
        Structures(args["pos"], args["cell"], args["species"], args["atom_offs"], device="cpu")


def test_overrides_are_checked_too():
    s = cpu_structures()
    with pytest.raises(ValueError, match="pos must be"):
        s.c_batch(pos=torch.zeros(4, 3, dtype=torch.float32))
