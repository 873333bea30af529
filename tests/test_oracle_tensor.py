"""Pins for the oracle's demag tensor and demag field (CPU only).

Each check ties the oracle to something other than itself: a closed form
from a different derivation (Aharoni's prism formula), the definition
evaluated another way (quadrature vs Newell's closed form, binary128 vs
double), a physical identity (trace, parity, point-dipole limit, the
uniform-magnetisation energy of a prism) or brute force (direct sum).
"""
import math

import numpy as np
import pytest
import torch

from oracle import micromag as mm
from oracle import tensor as tn


def aharoni_Dz(a, b, c):
    """Demag factor along z of a 2a x 2b x 2c prism (Aharoni, J. Appl. Phys. 83,
    3432 (1998)): an independent closed form, not Newell's f/g."""
    r = math.sqrt(a * a + b * b + c * c)
    ab, bc, ac = math.hypot(a, b), math.hypot(b, c), math.hypot(a, c)
    s = ((b * b - c * c) / (2 * b * c) * math.log((r - a) / (r + a))
         + (a * a - c * c) / (2 * a * c) * math.log((r - b) / (r + b))
         + b / (2 * c) * math.log((ab + a) / (ab - a))
         + a / (2 * c) * math.log((ab + b) / (ab - b))
         + c / (2 * a) * math.log((bc - b) / (bc + b))
         + c / (2 * b) * math.log((ac - a) / (ac + a))
         + 2 * math.atan(a * b / (c * r))
         + (a ** 3 + b ** 3 - 2 * c ** 3) / (3 * a * b * c)
         + (a * a + b * b - 2 * c * c) / (3 * a * b * c) * r
         + c / (a * b) * (ac + bc)
         - (ab ** 3 + bc ** 3 + ac ** 3) / (3 * a * b * c))
    return s / math.pi


def test_cube_self_factor_is_one_third():
    N = tn.newell_closed_form(0, 0, 0, 1.0, 1.0, 1.0)
    assert np.allclose(N[:3], 1.0 / 3.0, atol=1e-14)
    assert np.allclose(N[3:], 0.0, atol=1e-14)
    # scale invariance of the dimensionless tensor
    N2 = tn.newell_closed_form(0, 0, 0, 2e-9, 2e-9, 2e-9)
    assert np.allclose(N, N2, atol=1e-14)


@pytest.mark.parametrize("dims", [(1, 2, 3), (5, 1, 0.2), (0.3, 0.7, 4), (3.9, 3.9, 3.0)])
def test_self_term_trace_one_and_matches_aharoni(dims):
    x, y, z = dims
    N = tn.newell_closed_form(0, 0, 0, x, y, z)
    assert abs(N[:3].sum() - 1.0) < 1e-13
    assert abs(N[2] - aharoni_Dz(x / 2, y / 2, z / 2)) < 1e-12
    assert abs(N[0] - aharoni_Dz(y / 2, z / 2, x / 2)) < 1e-12
    assert abs(N[1] - aharoni_Dz(z / 2, x / 2, y / 2)) < 1e-12


def test_trace_vanishes_off_self():
    rng = np.random.default_rng(1)
    for _ in range(50):
        d = rng.uniform(0.5, 3.0, 3)
        off = rng.integers(-6, 7, 3) * d
        if not off.any():
            continue
        N = tn.newell_closed_form(*off, *d)
        assert abs(N[:3].sum()) < 1e-12 * max(1.0, np.abs(N).max())


def test_parity_of_components():
    d = (1.0, 1.3, 0.8)
    base = (2.0, 3.0, 1.0)
    N0 = tn.newell_closed_form(base[0] * d[0], base[1] * d[1], base[2] * d[2], *d)
    for sx in (1, -1):
        for sy in (1, -1):
            for sz in (1, -1):
                N = tn.newell_closed_form(sx * base[0] * d[0], sy * base[1] * d[1], sz * base[2] * d[2], *d)
                for c, name in enumerate(tn.COMPONENTS):
                    px, py, pz = tn.PARITY[name]
                    f = (sx if px < 0 else 1) * (sy if py < 0 else 1) * (sz if pz < 0 else 1)
                    assert abs(N[c] - f * N0[c]) < 1e-14


def test_double_closed_form_and_quadrature_match_binary128():
    if not tn.has_binary128():
        pytest.skip("no binary128 arithmetic on this platform")
    rng = np.random.default_rng(2)
    worst = 0.0
    for _ in range(150):
        d = rng.uniform(0.6, 3.0, 3)
        off = rng.integers(0, 50, 3) * d
        q = tn.newell_binary128(*off, *d)
        a = tn.tensor_at(*off, *d)
        worst = max(worst, np.abs(a - q).max() / np.abs(q).max())
    assert worst < 1e-12
    # the quadrature alone converges to the closed form at moderate range
    off = np.array([6.0, 4.0, 2.0])
    q = tn.newell_binary128(*off, 1.0, 1.0, 1.0)
    assert np.abs(tn.quadrature(*off, 1, 1, 1, 8) - q).max() < 1e-13 * np.abs(q).max()


def test_point_dipole_limit():
    """N(R) -> (V/4pi)(delta_ij/R^3 - 3 R_i R_j/R^5) with relative error O((d/R)^2)."""
    d = np.array([1.0, 1.2, 0.7])
    V = d.prod()
    u = np.array([0.6, 0.5, 0.62])
    u /= np.linalg.norm(u)
    errs = []
    for R in (20.0, 40.0, 80.0, 160.0):
        r = R * u
        N = tn.tensor_at(*r, *d)
        dip = V / (4 * np.pi) * (np.eye(3) / R ** 3 - 3 * np.outer(r, r) / R ** 5)
        D6 = np.array([dip[0, 0], dip[1, 1], dip[2, 2], dip[0, 1], dip[0, 2], dip[1, 2]])
        errs.append(np.abs(N - D6).max() / np.abs(D6).max())
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.5 < q < 4.5 for q in ratios), (errs, ratios)


def test_thin_plate_limit():
    N = tn.newell_closed_form(0, 0, 0, 1000.0, 1000.0, 1.0)
    assert 0.99 < N[2] < 1.0
    assert N[0] < 0.005 and N[1] < 0.005


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 5, 2), (8, 8, 1), (16, 16, 4)])
def test_fft_convolution_equals_direct_sum(shape):
    nx, ny, nz = shape
    p = mm.Problem(nx, ny, nz, 2e-9, 3e-9, 1.5e-9, Ms=8e5)
    rng = np.random.default_rng(3)
    m = mm.normalize(torch.from_numpy(rng.normal(size=(nz, ny, nx, 3))))
    a = mm.demag_field(p, m)
    b = mm.demag_field_direct(p, m)
    assert float((a - b).abs().max() / b.abs().max()) < 1e-12
    tg = [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (nz // 2, ny // 2, nx // 3)]
    c = mm.demag_field_at(p, m, tg)
    for t, cell in enumerate(tg):
        assert np.abs(c[t] - b[cell].numpy()).max() < 1e-12 * float(b.abs().max())


@pytest.mark.parametrize("shape,cell", [((40, 20, 1), (3.9e-9, 3.9e-9, 3e-9)),
                                        ((6, 5, 4), (2e-9, 2e-9, 2e-9))])
def test_uniform_magnetisation_energy_equals_prism_factor(shape, cell):
    """Sum over all cell pairs of N(r_i - r_j) = n N_prism, so the demag energy of
    uniform m is (mu0 Ms^2 V_tot / 2) m.N_prism.m with N_prism from Aharoni."""
    nx, ny, nz = shape
    dx, dy, dz = cell
    Ms = 8e5
    p = mm.Problem(nx, ny, nz, dx, dy, dz, Ms=Ms)
    u = np.array([1.0, 0.25, 0.1])
    u /= np.linalg.norm(u)
    m = torch.from_numpy(np.broadcast_to(u, (nz, ny, nx, 3)).copy())
    E = mm.energies(p, m)["demag"]
    a, b, c = nx * dx / 2, ny * dy / 2, nz * dz / 2
    Nd = np.diag([aharoni_Dz(b, c, a), aharoni_Dz(c, a, b), aharoni_Dz(a, b, c)])
    Ec = 0.5 * mm.MU0 * Ms ** 2 * nx * ny * nz * p.V * u @ Nd @ u
    assert abs(E / Ec - 1.0) < 1e-9
