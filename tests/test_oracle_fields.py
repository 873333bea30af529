"""Pins for the oracle's local fields, LLG right-hand side, stepping and energies (CPU only)."""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import micromag as mm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_m(shape, seed):
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    return mm.normalize(torch.from_numpy(rng.normal(size=(nz, ny, nx, 3))))


def test_paper_exchange_length():
    """l_ex = sqrt(A/K_m), K_m = mu0 Ms^2 / 2 is 5 nm for the paper's SP2/SP3 material."""
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    A, Ms = g["sp2_A"], g["sp2_Ms"]
    lex = math.sqrt(A / (0.5 * mm.MU0 * Ms ** 2))
    assert abs(lex - g["sp2_lex_nm"] * 1e-9) < 1e-3 * 1e-9
    # Ku = 0.1 K_m for SP3
    assert abs(0.1 * 0.5 * mm.MU0 * Ms ** 2 / g["sp3_Ku"] - 1.0) < 1e-5  # the paper prints 7 digits


def test_exchange_helix_closed_form():
    nx, dx = 24, 2e-9
    k = 2 * math.pi / (8 * dx)
    p = mm.Problem(nx, 3, 2, dx, 2e-9, 2e-9, Ms=8e5, A=1.3e-11)
    x = (np.arange(nx) + 0.5) * dx
    row = np.stack([np.cos(k * x), np.sin(k * x), 0 * x], -1)
    m = torch.from_numpy(np.broadcast_to(row, (2, 3, nx, 3)).copy())
    H = mm.exchange_field(p, m)
    c = 2 * p.A / (mm.MU0 * 8e5) * (2 * math.cos(k * dx) - 2) / dx ** 2
    inner = H[:, :, 1:-1]
    assert torch.allclose(inner, c * m[:, :, 1:-1], rtol=1e-12, atol=1e-9 * abs(c))


def test_exchange_uniform_is_zero_and_energy_is_face_sum():
    p = mm.Problem(5, 4, 3, 2e-9, 2.5e-9, 1.5e-9, Ms=8e5, A=1.3e-11)
    u = torch.tensor([0.3, -0.4, 0.5], dtype=torch.float64)
    mu = mm.normalize(u.expand(3, 4, 5, 3).clone())
    assert float(mm.exchange_field(p, mu).abs().max()) == 0.0
    m = rand_m(p.shape, 4)
    E = mm.energies(p, m)["exch"]
    faces = 0.0
    for axis, h in ((2, p.dx), (1, p.dy), (0, p.dz)):
        d = torch.diff(m, dim=axis)
        faces += float((d ** 2).sum()) / h ** 2
    assert abs(E / (p.A * p.V * faces) - 1.0) < 1e-12


def test_dmi_cycloid_closed_form_and_uniform_edges():
    nx, dx, D = 32, 2e-9, 2e-3
    k = 2 * math.pi / (10 * dx)
    p = mm.Problem(nx, 4, 1, dx, 2e-9, 2e-9, Ms=8e5, A=1.3e-11, D=D, dmi=True)
    x = (np.arange(nx) + 0.5) * dx
    row = np.stack([np.sin(k * x), 0 * x, np.cos(k * x)], -1)
    m = torch.from_numpy(np.broadcast_to(row, (1, 4, nx, 3)).copy())
    H = mm.dmi_field(p, m)
    c = -2 * D / (mm.MU0 * 8e5) * math.sin(k * dx) / dx
    # interior in x and in y (the chiral y ghosts act on m_y, so edge rows differ)
    assert torch.allclose(H[:, 1:-1, 1:-1], c * m[:, 1:-1, 1:-1], rtol=1e-12, atol=1e-9 * abs(c))
    mu = torch.zeros((1, 4, nx, 3), dtype=torch.float64)
    mu[..., 2] = 1.0
    Hu = mm.dmi_field(p, mu)
    assert float(Hu[:, 1:-1, 1:-1].abs().max()) < 1e-6
    assert float(Hu[:, :, 0].abs().max()) > 1e3


def _linear_part(p, v):
    """exchange + DMI + demag applied to an arbitrary (not unit) field v."""
    mp = mm.ghosted(p, v)
    return mm.exchange_field(p, v, mp) + mm.dmi_field(p, v, mp) + mm.demag_field(p, v)


@pytest.mark.parametrize("dmi", [False, True])
def test_linear_operator_is_ms_weighted_symmetric(dmi):
    shape = (2, 5, 6)
    rng = np.random.default_rng(5)
    Ms = rng.uniform(6e5, 1e6, size=shape)
    p = mm.Problem(6, 5, 2, 2e-9, 2.5e-9, 3e-9, Ms=Ms, A=1.3e-11, D=1.7e-3, dmi=dmi)
    a = torch.from_numpy(rng.normal(size=shape + (3,)))
    b = torch.from_numpy(rng.normal(size=shape + (3,)))
    Ms_t = torch.from_numpy(Ms)[..., None]
    lhs = float((Ms_t * a * _linear_part(p, b)).sum())
    rhs = float((Ms_t * b * _linear_part(p, a)).sum())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_heff_is_energy_gradient():
    """H_eff,i = -(1/(mu0 Ms_i V)) dE/dm_i for every term together, chiral boundary and Ms map included."""
    shape = (2, 4, 5)
    rng = np.random.default_rng(6)
    Ms = rng.uniform(6e5, 1e6, size=shape)
    axis = rng.normal(size=shape + (3,))
    axis /= np.linalg.norm(axis, axis=-1, keepdims=True)
    p = mm.Problem(5, 4, 2, 2e-9, 2.5e-9, 3e-9, Ms=Ms, A=1.3e-11, D=1.7e-3, dmi=True,
                   Ku=rng.uniform(1e4, 5e4, size=shape), ku_axis=axis, h_bias=(1e4, -2e4, 3e4))
    m = rand_m(shape, 7)
    H = mm.heff(p, m)

    def E(mm_):
        return sum(mm.energies(p, mm_).values())

    h = 1e-5
    for (k, j, i, c) in [(0, 0, 0, 0), (1, 3, 4, 2), (0, 2, 2, 1), (1, 0, 4, 0), (0, 3, 1, 2)]:
        e = torch.zeros_like(m)
        e[k, j, i, c] = h
        g = (E(m + e) - E(m - e)) / (2 * h)
        ref = -g / (mm.MU0 * Ms[k, j, i] * p.V)
        assert abs(ref - float(H[k, j, i, c])) < 1e-7 * float(H.abs().max())


def test_anisotropy_and_zeeman_energies():
    p = mm.Problem(3, 2, 1, 2e-9, 2e-9, 2e-9, Ms=8e5, Ku=5e3, ku_axis=(0, 0, 1.0), h_bias=(0, 0, 1e4))
    up = torch.zeros((1, 2, 3, 3), dtype=torch.float64)
    up[..., 2] = 1.0
    side = torch.zeros_like(up)
    side[..., 0] = 1.0
    assert abs(mm.energies(p, up)["anis"]) < 1e-30
    assert abs(mm.energies(p, side)["anis"] - 5e3 * p.V * 6) < 1e-30
    assert abs(mm.energies(p, up)["zeeman"] + mm.MU0 * 8e5 * 1e4 * p.V * 6) < 1e-28


def test_llg_orthogonality_and_fixed_point():
    p = mm.Problem(4, 4, 2, 2e-9, 2e-9, 2e-9, Ms=8e5, alpha=0.3, h_bias=(1e4, 2e4, -3e4))
    m = rand_m(p.shape, 8)
    H = mm.heff(p, m)
    dm = mm.llg_rhs(p, m, H)
    assert float((m * dm).sum(-1).abs().max()) < 1e-12 * float(dm.abs().max())
    assert float(mm.llg_rhs(p, m, 3.7e4 * m).abs().max()) < 1e-6


def _macrospin(alpha, dt, nsteps, H=1e5, precession=True, method="rk4"):
    p = mm.Problem(1, 1, 1, 2e-9, 2e-9, 2e-9, Ms=8e5, A=0.0, alpha=alpha, h_bias=(0, 0, H), demag=False,
                   precession=precession)
    th0, ph0 = 2.0, 0.3
    m = torch.tensor([[[[math.sin(th0) * math.cos(ph0), math.sin(th0) * math.sin(ph0), math.cos(th0)]]]],
                     dtype=torch.float64)
    mt = mm.run(p, m, dt, nsteps, method=method)
    t = dt * nsteps
    c = p.gamma * H / (1 + alpha ** 2)
    th = 2 * math.atan(math.tan(th0 / 2) * math.exp(-alpha * c * t))
    ph = ph0 + (c * t if precession else 0.0)
    ref = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    return np.abs(mt.numpy().ravel() - ref).max()


def test_macrospin_closed_form_and_rk4_order():
    """Precession at gamma0 H/(1+alpha^2) and tan(theta/2) decaying as exp(-alpha gamma0 H t/(1+alpha^2));
    RK4 error falls as dt^4."""
    T = 2e-11
    e1 = _macrospin(0.1, T / 100, 100)
    e2 = _macrospin(0.1, T / 200, 200)
    assert e1 < 1e-6
    assert 12.0 < e1 / e2 < 20.0
    # cube with demag on: the self field is -M/3, parallel to m, so it exerts no torque
    p = mm.Problem(1, 1, 1, 2e-9, 2e-9, 2e-9, Ms=8e5, alpha=0.1, h_bias=(0, 0, 1e5))
    m = mm.normalize(torch.tensor([[[[0.6, 0.1, -0.5]]]], dtype=torch.float64))
    Hd = mm.demag_field(p, m)
    assert torch.allclose(Hd, -8e5 / 3 * m, rtol=1e-12)


def test_macrospin_forward_euler_is_first_order_with_unit_norm():
    """Forward Euler with renormalisation (Sec. II-D, III-E) converges to the
    same closed form at first order: halving dt halves the error at a fixed
    time; every step leaves |m| = 1."""
    T = 2e-11
    e1 = _macrospin(0.1, T / 400, 400, method="euler")
    e2 = _macrospin(0.1, T / 800, 800, method="euler")
    assert e1 < 5e-2
    assert 1.8 < e1 / e2 < 2.2
    p = mm.Problem(6, 5, 2, 2e-9, 2e-9, 2e-9, Ms=8e5, A=1.3e-11, Ku=5e3, alpha=0.5, h_bias=(0, 0, 1e4))
    m = rand_m(p.shape, 31)
    for _ in range(5):
        m = mm.euler_step(p, m, 1e-13)
        assert float((m.norm(dim=-1) - 1).abs().max()) < 1e-15


def test_macrospin_without_precession_relaxes_in_its_plane():
    """Damping term only (the relaxation switch): the azimuth stays fixed and
    the polar angle follows the same tan(theta/2) law as with precession;
    RK4 error falls as dt^4 (alpha = 1, 0.3 ns: tan(theta/2) shrinks 28-fold)."""
    T = 3e-10
    e1 = _macrospin(1.0, T / 50, 50, precession=False)
    e2 = _macrospin(1.0, T / 100, 100, precession=False)
    assert e1 < 1e-6
    assert 12.0 < e1 / e2 < 20.0


def test_energy_decays_and_norm_conserved_plain():
    p = mm.Problem(8, 8, 2, 2e-9, 2e-9, 2e-9, Ms=8e5, A=1.3e-11, Ku=5e3, alpha=0.5, h_bias=(0, 0, 1e4))
    m = rand_m(p.shape, 9)
    last = sum(mm.energies(p, m).values())
    for _ in range(40):
        m = mm.rk4_step(p, m, 1e-14)
        e = sum(mm.energies(p, m).values())
        assert e <= last + 1e-12 * abs(last)
        last = e
    assert float((torch.linalg.vector_norm(m, dim=-1) - 1).abs().max()) < 1e-15
