"""Hyperparameters of the separable-density SOAP descriptor (oracle side).

Names follow the paper: sigma_{0,r}, sigma_{0,perp}, alpha_r, alpha_perp and the
amplitude exponent a of Eq. 15; r_soft, r_hard (= r_cut) and n_f of the density
smoothing of Sec. III.B; n_max radial functions (n_max - 1 polynomials plus one
Gaussian, Sec. III.A) and l_max.

``eq08_weight`` selects the angular weight.  By default the coefficient of Y_lm is
4 pi e^{-z} i_l(z) Y*_lm, which is what projecting the addition-theorem expansion of
term (3) of Eq. 05 onto orthonormal Y_lm gives; Eq. 08 as printed carries an extra
factor (2l+1), available with ``eq08_weight=True``.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Params:
    r_cut: float
    r_soft: float
    sigma_r0: float
    sigma_p0: float
    alpha_r: float = 0.0
    alpha_p: float = 0.0
    amp_a: float = 1.0
    n_f: float = 4.0
    central_weight: float = 1.0
    n_max: int = 8
    l_max: int = 8
    n_species: int = 1
    eq08_weight: bool = False

    @property
    def r_hard(self) -> float:
        return self.r_cut

    @property
    def n_channels(self) -> int:
        return self.n_species * self.n_max

    @property
    def dim(self) -> int:
        """Length of the packed descriptor: channel pairs (c1 <= c2) times (l_max + 1)."""
        nc = self.n_channels
        return nc * (nc + 1) // 2 * (self.l_max + 1)

    @staticmethod
    def from_dict(d: dict) -> "Params":
        keys = Params.__dataclass_fields__.keys()
        return Params(**{k: v for k, v in d.items() if k in keys})
