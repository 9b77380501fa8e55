"""Separable-density SOAP expansion coefficients, power spectrum and descriptor (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).  FP64 PyTorch CPU operations,
vectorised over neighbour pairs; every function names the passage of Caro,
arXiv:1905.02142, that it writes out.

Conventions:
  * channel index ch = species(j) * n_max + n; the central atom adds to its own
    species' channels;
  * complex coefficients c_nlm are kept for m >= 0 only (Eq. 09 needs no more), as
    separate real and imaginary parts in [.., l, m] arrays that are zero for m > l;
  * the packed descriptor lists, for each channel pair ch1 <= ch2 (row-major over the
    upper triangle) and each l = 0..l_max, the value p[ch1, ch2, l], multiplied by
    sqrt(2) when ch1 != ch2, so that dot products of packed vectors equal the full
    sums over (n, n', l) of Sec. I.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import basis, neighbours
from .params import Params

DT = torch.float64
SQRT2 = math.sqrt(2.0)
FOUR_PI = 4.0 * math.pi


def widths_and_amplitude(rj: torch.Tensor, P: Params):
    """Eq. 15: sigma_r,j = sigma_0r + alpha_r r_j, sigma_perp,j = sigma_0perp + alpha_perp r_j,
    A_j = (sigma_r,j sigma_perp,j^2)^-1 (1 + 2 x^3 - 3 x^2)^a with x = r_j / r_cut."""
    sr = P.sigma_r0 + P.alpha_r * rj
    sp = P.sigma_p0 + P.alpha_p * rj
    x = rj / P.r_cut
    poly = 1.0 + 2.0 * x ** 3 - 3.0 * x ** 2
    if P.amp_a == 0.0:
        damp = torch.ones_like(rj)
    else:
        damp = poly.clamp(min=0.0) ** P.amp_a
    return sr, sp, damp / (sr * sp * sp)


def smoothing_function(r, P: Params):
    """The density smoothing function f(r) of Sec. III.B (used by the quadrature pins)."""
    r = torch.as_tensor(r, dtype=DT)
    buf = torch.exp(-0.5 * P.n_f ** 2 * (r - P.r_soft) ** 2 / (P.r_hard - P.r_soft) ** 2) \
        if P.r_hard > P.r_soft else torch.zeros_like(r)
    return torch.where(r < P.r_soft, torch.ones_like(r),
                       torch.where(r > P.r_hard, torch.zeros_like(r), buf))


def _erf_difference(lo: torch.Tensor, hi: torch.Tensor) -> torch.Tensor:
    """erf(hi) - erf(lo) for lo <= hi; complementary error functions are used when both
    arguments have the same sign (identical in exact arithmetic, fewer lost digits)."""
    mid = torch.erf(hi) - torch.erf(lo)
    pos = torch.erfc(lo) - torch.erfc(hi)
    neg = torch.erfc(-hi) - torch.erfc(-lo)
    return torch.where(lo >= 0.0, pos, torch.where(hi <= 0.0, neg, mid))


def radial_integrals(c: torch.Tensor, w: torch.Tensor, a: float, b: float, r_cut: float,
                     kmax: int) -> torch.Tensor:
    """J_k = int_a^b (1 - r/r_cut)^k exp(-(r - c)^2 / (2 w^2)) dr for k = 0..kmax.

    Sec. III.A: N_alpha b_alpha = J_{alpha+2}.  The sequence starts from the erf seed
    (b_{-2}, i.e. J_0), obtains J_1 from J_0 with the b_{-3} term dropped (its factor
    alpha+1 vanishes), and continues with the recursion Eq. 04:
      J_{k+2} = (k+1) (w/r_cut)^2 J_k + (1 - c/r_cut) J_{k+1}
                + (w^2/r_cut) [(1 - r/r_cut)^(k+1) exp(-(r-c)^2/(2w^2))]_a^b.
    """
    ga = torch.exp(-(a - c) ** 2 / (2.0 * w * w))
    gb = torch.exp(-(b - c) ** 2 / (2.0 * w * w))
    j0 = w * math.sqrt(math.pi / 2.0) * _erf_difference((a - c) / (SQRT2 * w),
                                                         (b - c) / (SQRT2 * w))
    eps = (w / r_cut) ** 2
    beta = 1.0 - c / r_cut
    bcoef = w * w / r_cut
    ta, tb = 1.0 - a / r_cut, 1.0 - b / r_cut
    out = [j0, beta * j0 + bcoef * (gb - ga)]
    tak, tbk = ta, tb
    for k in range(0, kmax - 1):
        out.append((k + 1) * eps * out[k] + beta * out[k + 1] + bcoef * (tbk * gb - tak * ga))
        tak, tbk = tak * ta, tbk * tb
    return torch.stack(out[:kmax + 1], dim=-1)


def gaussian_row(rj: torch.Tensor, sr: torch.Tensor, sigma_r0: float) -> torch.Tensor:
    """Overlap of the auxiliary Gaussian phi_nmax (Eq. 06) with the radial Gaussian of
    neighbour j on [0, inf): the closed form given after Eq. 04 in Sec. III.A."""
    s0 = sigma_r0
    sstar = torch.sqrt(s0 * s0 + sr * sr)
    return (math.pi ** 0.25 / math.sqrt(s0) * torch.exp(-rj * rj / (2.0 * sstar * sstar))
            * (s0 * sr / sstar) * (1.0 + torch.erf(s0 * rj / (SQRT2 * sr * sstar))))


def radial_coefficients(rj: torch.Tensor, P: Params) -> torch.Tensor:
    """b_alpha^j of Eq. 01 in the primitive basis, alpha = 1..n_max: [P, n_max].

    Includes the amplitude A_j (Eq. 15) and the smoothing f (Sec. III.B): the range is
    split into [0, r_soft], where the radial Gaussian is expanded as is, and
    [r_soft, r_hard], where f times the Gaussian is again a Gaussian (width s, centre mu,
    amplitude C) and the same recursion applies.  The Gaussian row uses the closed form.
    """
    sr, sp, amp = widths_and_amplitude(rj, P)
    kmax = P.n_max + 1
    rs = min(P.r_soft, P.r_hard)
    jk = radial_integrals(rj, sr, 0.0, rs, P.r_cut, kmax)
    if rs < P.r_hard:
        tau = (P.r_hard - rs) / P.n_f
        s2 = 1.0 / (1.0 / (sr * sr) + 1.0 / (tau * tau))
        mu = s2 * (rj / (sr * sr) + rs / (tau * tau))
        amp_c = torch.exp(-(rj - rs) ** 2 / (2.0 * (sr * sr + tau * tau)))
        jk = jk + amp_c[:, None] * radial_integrals(mu, torch.sqrt(s2), rs, P.r_hard,
                                                    P.r_cut, kmax)
    alphas = np.arange(1, P.n_max)
    norms = torch.as_tensor(basis.poly_norm(alphas, P.r_cut), dtype=DT)
    b_poly = jk[:, alphas + 2] / norms[None, :]
    b_gauss = gaussian_row(rj, sr, P.sigma_r0)
    return torch.cat([b_poly, b_gauss[:, None]], dim=1) * amp[:, None]


def _double_factorial(n: int) -> float:
    out = 1.0
    while n > 1:
        out *= n
        n -= 2
    return out


ILEXP_SERIES_MAX_Z = 40.0


def ilexp(z: torch.Tensor, l_max: int) -> torch.Tensor:
    """ilexp(x; l) = e^{-x^2} i_l(x^2) (Sec. III.C) as a function of z = x^2: [P, l_max+1].

    Written from the definition of the modified spherical Bessel function i_l:
      z <= 40: its power series, e^{-z} sum_k z^(l+2k) / (2^k k! (2l+2k+1)!!), whose terms
               are all positive;
      z > 40 : its finite closed form,
               e^{-z} i_l(z) = (1/2z) [ sum_k (-1)^k a_lk (2z)^-k
                                         + (-1)^(l+1) e^{-2z} sum_k a_lk (2z)^-k ],
               a_lk = (l+k)! / (k! (l-k)!), k = 0..l.
    """
    small = z <= ILEXP_SERIES_MAX_Z
    zs = torch.where(small, z, torch.ones_like(z))
    zl = torch.where(small, torch.full_like(z, 2.0 * ILEXP_SERIES_MAX_Z), z)
    e_s = torch.exp(-zs)
    e_l = torch.exp(-2.0 * zl)
    t = 1.0 / (2.0 * zl)
    cols = []
    for l in range(l_max + 1):
        term = zs ** l / _double_factorial(2 * l + 1)
        acc = term
        for k in range(200):
            term = term * zs * zs / (2.0 * (k + 1) * (2 * l + 2 * k + 3))
            acc = acc + term
        series = e_s * acc
        s1 = torch.zeros_like(zl)
        s2 = torch.zeros_like(zl)
        tk = torch.ones_like(zl)
        for k in range(l + 1):
            a_lk = math.factorial(l + k) / (math.factorial(k) * math.factorial(l - k))
            s1 = s1 + (-1) ** k * a_lk * tk
            s2 = s2 + a_lk * tk
            tk = tk * t
        closed = t * (s1 + (-1) ** (l + 1) * e_l * s2)
        cols.append(torch.where(small, series, closed))
    return torch.stack(cols, dim=-1)


def associated_legendre(x: torch.Tensor, l_max: int) -> torch.Tensor:
    """P_lm(x) for 0 <= m <= l <= l_max with the Condon-Shortley phase: [P, l+1, m+1].

    The seeds are the sectoral values P_mm = (-1)^m (2m-1)!! (1-x^2)^(m/2) (which give
    the six starting polynomials tabulated in Sec. III.C), P_{m+1,m} = (2m+1) x P_mm, and
    the recursion on l of Sec. III.C,
      P_lm = ((2l-1) x P_{l-1,m} - (l+m-1) P_{l-2,m}) / (l-m).
    """
    sq = torch.sqrt(torch.clamp(1.0 - x * x, min=0.0))
    rows = [[None] * (l_max + 1) for _ in range(l_max + 1)]
    pmm = torch.ones_like(x)
    for m in range(l_max + 1):
        if m > 0:
            pmm = -(2 * m - 1) * sq * pmm
        rows[m][m] = pmm
        if m + 1 <= l_max:
            rows[m + 1][m] = (2 * m + 1) * x * pmm
        for l in range(m + 2, l_max + 1):
            rows[l][m] = ((2 * l - 1) * x * rows[l - 1][m] - (l + m - 1) * rows[l - 2][m]) / (l - m)
    zero = torch.zeros_like(x)
    return torch.stack([torch.stack([rows[l][m] if m <= l else zero
                                     for m in range(l_max + 1)], dim=-1)
                        for l in range(l_max + 1)], dim=-2)


def reduced_legendre(x: torch.Tensor, l_max: int) -> torch.Tensor:
    """P_lm(x) / (1-x^2)^(m/2) for 0 <= m <= l <= l_max (Condon-Shortley phase): the same
    recursion in l as ``associated_legendre``, started from (-1)^m (2m-1)!!, so that the
    sin(theta)^m factor can be carried by (x + iy)^m instead (no pole singularity)."""
    rows = [[None] * (l_max + 1) for _ in range(l_max + 1)]
    for m in range(l_max + 1):
        pmm = torch.full_like(x, (-1.0) ** m * _double_factorial(2 * m - 1))
        rows[m][m] = pmm
        if m + 1 <= l_max:
            rows[m + 1][m] = (2 * m + 1) * x * pmm
        for l in range(m + 2, l_max + 1):
            rows[l][m] = ((2 * l - 1) * x * rows[l - 1][m] - (l + m - 1) * rows[l - 2][m]) / (l - m)
    zero = torch.zeros_like(x)
    return torch.stack([torch.stack([rows[l][m] if m <= l else zero
                                     for m in range(l_max + 1)], dim=-1)
                        for l in range(l_max + 1)], dim=-2)


def conj_spherical_harmonics(rhat: torch.Tensor, l_max: int):
    """Real and imaginary parts of Y*_lm(theta_j, phi_j), m >= 0 (Sec. III.C):
    sqrt((2l+1)(l-m)! / (4 pi (l+m)!)) e^{-i m phi} P_lm(cos theta).

    sin(theta)^m e^{i m phi} = (x + i y)^m on the unit sphere, so the harmonics are
    evaluated as the reduced P_lm times C_m - i S_m, where C_m = rho^m cos(m phi) and
    S_m = rho^m sin(m phi) follow the Chebyshev recursion of Sec. III.C multiplied by
    rho^m: C_m = 2x C_{m-1} - rho^2 C_{m-2} (same for S_m).  This is the same function
    without the division by rho, so it and its gradient stay finite on the z axis.
    Returns two [P, l+1, m+1] tensors.
    """
    x, y, z = rhat[:, 0], rhat[:, 1], rhat[:, 2]
    rho2 = x * x + y * y
    cos_m = [torch.ones_like(x), x]
    sin_m = [torch.zeros_like(x), y]
    for m in range(2, l_max + 1):
        cos_m.append(2.0 * x * cos_m[m - 1] - rho2 * cos_m[m - 2])
        sin_m.append(2.0 * x * sin_m[m - 1] - rho2 * sin_m[m - 2])
    cos_m = torch.stack(cos_m[:l_max + 1], dim=-1)   # [P, m]
    sin_m = torch.stack(sin_m[:l_max + 1], dim=-1)
    plm = reduced_legendre(z, l_max)                 # [P, l, m]
    k = np.zeros((l_max + 1, l_max + 1))
    for l in range(l_max + 1):
        for m in range(l + 1):
            k[l, m] = math.sqrt((2 * l + 1) * math.factorial(l - m)
                                / (4.0 * math.pi * math.factorial(l + m)))
    k = torch.as_tensor(k, dtype=DT)
    re = k[None] * plm * cos_m[:, None, :]
    im = -k[None] * plm * sin_m[:, None, :]
    return re, im


def pair_vectors(pos: torch.Tensor, cell: torch.Tensor, pairs: dict) -> torch.Tensor:
    """r_ij = r_j + S.h - r_i for the listed pairs (differentiable in pos and cell)."""
    i = torch.as_tensor(pairs["i"])
    j = torch.as_tensor(pairs["j"])
    s = torch.as_tensor(pairs["shift"], dtype=DT)
    h = cell[torch.as_tensor(pairs["struct"])]                    # [P, 3, 3]
    svec = torch.einsum("pk,pkc->pc", s, h)
    return pos[j] + svec - pos[i]


def expansion_coefficients(P: Params, W: np.ndarray, pos: torch.Tensor, cell: torch.Tensor,
                           species: np.ndarray, centers: np.ndarray, pairs: dict):
    """c_nlm of every centre in ``centers`` (sorted), Eqs. 01 and 08 summed over j (Sec. II),
    plus the central atom: returns (re, im), each [n_centers, n_channels, l+1, m+1].

    Per neighbour j (species s_j, distance r_j, direction r_hat_j, z_j = r_j^2/sigma_perp,j^2):
      c^j_{s_j n l m} = 4 pi b_n^j ilexp(x_j; l) Y*_lm(r_hat_j)   [x (2l+1) with eq08_weight],
      b_n^j = sum_alpha W_n,alpha b_alpha^j.
    The central atom (r = 0) has ilexp(0; l) = delta_l0 and Y_00 = 1/sqrt(4 pi), so it
    adds central_weight * sqrt(4 pi) b_n(0) to c_{s_i n 0 0}.
    """
    n_c = len(centers)
    lmax = P.l_max
    wt = torch.as_tensor(W, dtype=DT)
    loc = np.searchsorted(centers, pairs["i"])
    assert np.all(centers[loc] == pairs["i"])
    r = pair_vectors(pos, cell, pairs)
    rj = torch.sqrt((r * r).sum(dim=1))
    rhat = r / rj[:, None]
    b_alpha = radial_coefficients(rj, P)                          # [P, n_max]
    b_n = b_alpha @ wt.T
    _, sp, _ = widths_and_amplitude(rj, P)
    il = ilexp(rj * rj / (sp * sp), lmax)                         # [P, l]
    if P.eq08_weight:
        il = il * torch.as_tensor([2 * l + 1 for l in range(lmax + 1)], dtype=DT)[None, :]
    yre, yim = conj_spherical_harmonics(rhat, lmax)               # [P, l, m]
    ang_re = FOUR_PI * il[:, :, None] * yre
    ang_im = FOUR_PI * il[:, :, None] * yim
    contrib_re = b_n[:, :, None, None] * ang_re[:, None, :, :]    # [P, n, l, m]
    contrib_im = b_n[:, :, None, None] * ang_im[:, None, :, :]
    ns, nm = P.n_species, P.n_max
    slot = torch.as_tensor(loc * ns + species[pairs["j"]], dtype=torch.int64)
    shape = (n_c * ns, nm, lmax + 1, lmax + 1)
    c_re = torch.zeros(shape, dtype=DT).index_add(0, slot, contrib_re)
    c_im = torch.zeros(shape, dtype=DT).index_add(0, slot, contrib_im)
    # central atom
    b0 = radial_coefficients(torch.zeros(1, dtype=DT), P) @ wt.T  # [1, n_max]
    cen = torch.zeros(shape, dtype=DT)
    cslot = torch.as_tensor(np.arange(n_c) * ns + species[centers], dtype=torch.int64)
    cen[cslot, :, 0, 0] = P.central_weight * math.sqrt(FOUR_PI) * b0[0][None, :]
    c_re = c_re + cen
    return (c_re.reshape(n_c, ns * nm, lmax + 1, lmax + 1),
            c_im.reshape(n_c, ns * nm, lmax + 1, lmax + 1))


def power_spectrum(c_re: torch.Tensor, c_im: torch.Tensor) -> torch.Tensor:
    """p_{n n' l} by Eq. 09: c_nl0 c*_n'l0 + 2 sum_{m>=1} Re(c_nlm c*_n'lm): [.., ch, ch', l]."""
    lmax = c_re.shape[-1] - 1
    wm = torch.full((lmax + 1,), 2.0, dtype=DT)
    wm[0] = 1.0
    return (torch.einsum("iaxm,ibxm,m->iabx", c_re, c_re, wm)
            + torch.einsum("iaxm,ibxm,m->iabx", c_im, c_im, wm))


def pack(p_full: torch.Tensor) -> torch.Tensor:
    """Packed layout of the module docstring: [.., n_ch(n_ch+1)/2 * (l+1)]."""
    nc = p_full.shape[-2]
    parts = []
    for a in range(nc):
        for b in range(a, nc):
            v = p_full[..., a, b, :]
            parts.append(v if a == b else SQRT2 * v)
    return torch.cat(parts, dim=-1)


def unpack(vec: torch.Tensor, n_ch: int, l_max: int) -> torch.Tensor:
    """Inverse of ``pack`` (symmetric full array)."""
    out = torch.zeros(vec.shape[:-1] + (n_ch, n_ch, l_max + 1), dtype=vec.dtype)
    k = 0
    for a in range(n_ch):
        for b in range(a, n_ch):
            v = vec[..., k:k + l_max + 1]
            if a != b:
                v = v / SQRT2
            out[..., a, b, :] = v
            out[..., b, a, :] = v
            k += l_max + 1
    return out


def descriptors(batch, P: Params, centers=None, W=None, pairs=None, chunk: int = 256):
    """Descriptors of the listed centres (default: all atoms) of a flattened batch.

    Returns dict: centers, pairs, c_re, c_im, p (full), pnorm, q (packed) -- all FP64.
    q = p / sqrt(p . p) (Sec. I), the norm taken over the full (n, n', l) array.
    """
    if W is None:
        W = basis.orthonormaliser(P.n_max, P.r_cut, P.sigma_r0)
    if centers is None:
        centers = np.arange(batch.n_atoms)
    centers = np.unique(np.asarray(centers, dtype=np.int64))
    if pairs is None:
        pairs = neighbours.batch_pairs(batch, P.r_cut, centers=centers)
    pos = torch.as_tensor(batch.pos, dtype=DT)
    cell = torch.as_tensor(batch.cell, dtype=DT)
    out = {"c_re": [], "c_im": [], "p": []}
    with torch.no_grad():
        for c0 in range(0, len(centers), chunk):
            cc = centers[c0:c0 + chunk]
            sel = (pairs["i"] >= cc[0]) & (pairs["i"] <= cc[-1])
            sub = {k: v[sel] for k, v in pairs.items()}
            c_re, c_im = expansion_coefficients(P, W, pos, cell, batch.species, cc, sub)
            out["c_re"].append(c_re)
            out["c_im"].append(c_im)
            out["p"].append(power_spectrum(c_re, c_im))
    res = {k: torch.cat(v) for k, v in out.items()}
    p = res["p"]
    pnorm = torch.sqrt((p * p).sum(dim=(1, 2, 3)))
    res["pnorm"] = pnorm
    res["q"] = pack(p / pnorm[:, None, None, None])
    res["centers"] = centers
    res["pairs"] = pairs
    res["W"] = W
    return res
