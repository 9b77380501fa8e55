"""Plain, slow FP64 CPU oracle for the separable-density SOAP descriptor and GAP model.

TEST INFRASTRUCTURE ONLY.  Nothing in the library's compute path imports this
package: only the tests, the smoke check and the CPU-baseline leg of the benchmark
use it, to produce the reference values the CUDA path is compared against.

It is written from Caro, "Optimizing many-body atomic descriptors for enhanced
computational performance of machine learning based interatomic potentials"
(arXiv:1905.02142), in FP64 PyTorch CPU tensor operations, vectorised over neighbour
pairs, with no blocking or fusion beyond what the paper's formulas state.  Forces
and the virial are the exact derivatives of the energy obtained with PyTorch
autograd (the paper gives no derivative formulas).

Modules:
  neighbours -- brute-force periodic neighbour search (all images, strict cutoff)
  basis      -- radial basis, overlap matrix S and W = S^-1/2 (Sec. III.A)
  soap       -- density expansion coefficients, power spectrum, normalised descriptor
  gap        -- GAP local energies, total energies, forces and virial
"""
from .params import Params  # noqa: F401
from . import neighbours, basis, soap, gap  # noqa: F401
