"""The rounding margin of the neighbour search's FP32 prefilter (no GPU).

The library classifies a candidate (i, j, S) by an FP32 squared separation computed from
FP32 positions and FP32 lattice vectors, in a fixed order of round-to-nearest operations
(dx = (x_j + s_x) - x_i with s = (S1 h1 + S2 h2) + S3 h3, d2 = (dx dx + dy dy) + dz dz).
Only candidates within a margin of r_cut^2 (or of zero) take the exact FP64 test, so the
pair set is bit-exact only if |d2_f32 - d2| + |fl(r_cut^2) - r_cut^2| never exceeds that
margin.  The margin is set per structure on the host, from the lattice-vector lengths and
the image range; the helper below restates that host computation, and the tests measure
the FP32 error against FP64 arithmetic on every candidate of sheared small and large
cells, requiring the margin to hold with the factor of two it claims.
"""
import math

import numpy as np
import pytest

F = np.float32


def host_margin(cell, rc, n_atoms):
    """Per-structure margin and image ranges as the library's geometry set-up forms them
    (cell rows are the lattice vectors)."""
    det = float(np.linalg.det(cell))
    H = sum(float(np.linalg.norm(cell[k])) for k in range(3))
    m = []
    for k in range(3):
        u, v = cell[(k + 1) % 3], cell[(k + 2) % 3]
        dk = abs(det) / float(np.linalg.norm(np.cross(u, v)))
        nb = max(1, math.floor(dk / rc))
        nb_cap = max(1, int(np.cbrt(max(n_atoms, 1))) + 1)
        nb = min(nb, 2 * nb_cap)
        m.append(math.floor(rc * nb / dk) + 1)
    X = H * (max(m) + 3)
    u = 2.0 ** -24
    margin = F(2.0 * (2.0 * math.sqrt(3.0) * 10.0 * rc * X * u + 4.0 * rc * rc * u) + 1e-30)
    return margin, m


def fp32_d2(xi, xj, shifts, h32):
    """FP32 squared separations of atom i to atoms xj [n, 3] under images shifts [k, 3],
    in the library's operation order: [k, n]."""
    f = shifts.astype(F)
    s = (f[:, 0:1] * h32[0][None, :] + f[:, 1:2] * h32[1][None, :]) + f[:, 2:3] * h32[2][None, :]
    d = (xj[None, :, :] + s[:, None, :]) - xi[None, None, :]
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


CASES = [  # (edge A, shear, atoms, r_cut, fractional corner the atoms fill)
    (3.1, 0.35, 7, 5.0, 1.0),        # many images, self-images
    (9.0, 0.2, 60, 5.0, 1.0),
    (46.371, 0.0, 200, 5.0, 1.0),    # the paper's timing box edge
    (87.36, 0.1, 300, 5.0, 0.3),     # the 100k-atom box edge, atoms packed in a corner
    (300.0, 0.3, 300, 6.0, 0.1),     # far from the origin: the last tenth of each edge
]


@pytest.mark.parametrize("edge, shear, n, rc, corner", CASES)
def test_fp32_prefilter_error_within_half_the_margin(edge, shear, n, rc, corner):
    rng = np.random.default_rng(int(edge * 10))
    cell = np.eye(3) * edge
    cell[1, 0] = shear * edge
    cell[2, 0] = shear * edge
    cell[2, 1] = 0.5 * shear * edge
    frac = 1.0 - corner * rng.random((n, 3))
    frac[frac >= 1.0] = 0.0
    frac[:4] = np.array([[0.0, 0.0, 0.0], [1 - 1e-12, 1 - 1e-12, 1 - 1e-12],
                         [0.5, 1 - 1e-12, 0.0], [1 - 1e-12, 0.0, 0.5]])[: min(4, n)]
    pos = frac @ cell
    margin, m = host_margin(cell, rc, n)
    h32 = cell.astype(F)
    x32 = pos.astype(F)
    rng_s = [np.arange(-(mk + 1), mk + 2) for mk in m]
    shifts = np.stack(np.meshgrid(*rng_s, indexing="ij"), axis=-1).reshape(-1, 3)
    shift64 = shifts.astype(np.float64) @ cell
    rc2 = rc * rc
    rc2_err = abs(float(F(rc2)) - rc2)
    worst = 0.0
    for i in range(n):
        d2f = fp32_d2(x32[i], x32, shifts, h32).astype(np.float64)
        d = (pos[None, :, :] + shift64[:, None, :]) - pos[i][None, None, :]
        d2 = np.einsum("knc,knc->kn", d, d)
        keep = d2 < 4.0 * rc2                      # candidates that matter to the decision
        err = np.abs(d2f - d2)[keep] + rc2_err
        worst = max(worst, float(err.max(initial=0.0)))
    assert worst > 0.0                             # pairs near the cutoff were tested
    assert worst <= 0.5 * float(margin), (worst, float(margin))


def test_margin_scales_with_the_cell_and_images():
    small, _ = host_margin(np.eye(3) * 10.0, 5.0, 100)
    large, _ = host_margin(np.eye(3) * 100.0, 5.0, 100)
    assert large > 5 * small                       # larger coordinates, larger rounding
    thin, m = host_margin(np.diag([2.0, 20.0, 20.0]), 5.0, 10)
    assert m[0] >= 3                               # several images along the thin edge
