"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in the oracle (a dropped term, a wrong sign or
factor, a swapped operand, a missing mode corner, a skipped step of an
algorithm) through monkeypatch and checks that the pin meant to guard that
part fails.  The planted versions live only here, in the test process.
"""
import math

import numpy as np
import pytest
import torch

import test_oracle_adjoint as pins_adj
import test_oracle_cnn as pins_cnn
import test_oracle_fields as pins_fields
import test_oracle_fno as pins_fno
import test_oracle_mri as pins_mri
import test_oracle_sp3 as pins_sp3
import test_oracle_tensor as pins_tensor
from oracle import cnn, fno, mri
from oracle import micromag as mm
from oracle import tensor as tn
from test_oracle_adjoint import setup  # noqa: F401  (the adjoint pins' module fixture)


def planted_fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


# ---------------------------------------------------------------------------
# local fields
# ---------------------------------------------------------------------------

def test_exchange_without_the_z_term_is_caught(monkeypatch):
    def exch(p, m, mp=None):
        mp = mm.ghosted(p, m) if mp is None else mp
        c = mp[1:-1, 1:-1, 1:-1]
        lap = ((mp[1:-1, 1:-1, 2:] + mp[1:-1, 1:-1, :-2] - 2 * c) / p.dx ** 2
               + (mp[1:-1, 2:, 1:-1] + mp[1:-1, :-2, 1:-1] - 2 * c) / p.dy ** 2)
        return (2.0 * p.A / (mm.MU0 * mm.ms_field(p)))[..., None] * lap
    monkeypatch.setattr(mm, "exchange_field", exch)
    planted_fails(pins_fields.test_exchange_uniform_is_zero_and_energy_is_face_sum)


def test_exchange_with_A_for_2A_is_caught(monkeypatch):
    orig = mm.exchange_field
    monkeypatch.setattr(mm, "exchange_field", lambda p, m, mp=None: 0.5 * orig(p, m, mp))
    planted_fails(pins_fields.test_exchange_helix_closed_form)


def test_dmi_with_the_wrong_sign_is_caught(monkeypatch):
    orig = mm.dmi_field
    monkeypatch.setattr(mm, "dmi_field", lambda p, m, mp=None: -orig(p, m, mp))
    planted_fails(pins_fields.test_dmi_cycloid_closed_form_and_uniform_edges)


def test_dmi_with_swapped_divergence_terms_is_caught(monkeypatch):
    def dmi(p, m, mp=None):
        if not p.dmi or p.D == 0.0:
            return torch.zeros_like(m)
        mp = mm.ghosted(p, m) if mp is None else mp
        ddx = (mp[1:-1, 1:-1, 2:] - mp[1:-1, 1:-1, :-2]) / (2 * p.dx)
        ddy = (mp[1:-1, 2:, 1:-1] - mp[1:-1, :-2, 1:-1]) / (2 * p.dy)
        H = torch.stack([ddx[..., 2], ddy[..., 2], -(ddx[..., 1] + ddy[..., 0])], dim=-1)
        return (2.0 * p.D / (mm.MU0 * mm.ms_field(p)))[..., None] * H
    monkeypatch.setattr(mm, "dmi_field", dmi)
    planted_fails(pins_fields.test_dmi_cycloid_closed_form_and_uniform_edges)


def test_chiral_ghost_with_the_wrong_sign_is_caught(monkeypatch):
    """Ghost m_g = m_b + h (D/2A) (e_z x n) x m_b instead of minus."""
    orig = mm.ghosted

    def ghosted(p, m):
        q = mm.Problem(p.nx, p.ny, p.nz, p.dx, p.dy, p.dz, Ms=p.Ms, A=p.A, Ku=p.Ku, ku_axis=p.ku_axis, D=-p.D,
                       alpha=p.alpha, gamma=p.gamma, h_bias=p.h_bias, dmi=p.dmi, demag=p.demag)
        return orig(q, m)
    monkeypatch.setattr(mm, "ghosted", ghosted)
    planted_fails(pins_fields.test_linear_operator_is_ms_weighted_symmetric, True)


def test_chiral_ghost_at_the_wrong_distance_is_caught(monkeypatch):
    """The y-face ghosts built with dx instead of dy (cells are not cubes)."""
    orig = mm.ghosted

    def ghosted(p, m):
        q = mm.Problem(p.nx, p.ny, p.nz, p.dx, p.dx, p.dz, Ms=p.Ms, A=p.A, Ku=p.Ku, ku_axis=p.ku_axis, D=p.D,
                       alpha=p.alpha, gamma=p.gamma, h_bias=p.h_bias, dmi=p.dmi, demag=p.demag)
        return orig(q, m)
    monkeypatch.setattr(mm, "ghosted", ghosted)
    planted_fails(pins_fields.test_heff_is_energy_gradient)


def test_demag_energy_without_its_half_is_caught(monkeypatch):
    orig = mm.energies

    def energies(p, m):
        e = orig(p, m)
        e["demag"] *= 2.0
        return e
    monkeypatch.setattr(mm, "energies", energies)
    planted_fails(pins_fields.test_heff_is_energy_gradient)


def test_anisotropy_with_Ku_for_2Ku_is_caught(monkeypatch):
    orig = mm.anisotropy_field
    monkeypatch.setattr(mm, "anisotropy_field", lambda p, m: 0.5 * orig(p, m))
    planted_fails(pins_fields.test_heff_is_energy_gradient)


def test_zeeman_energy_without_mu0_is_caught(monkeypatch):
    orig = mm.energies

    def energies(p, m):
        e = orig(p, m)
        e["zeeman"] /= mm.MU0
        return e
    monkeypatch.setattr(mm, "energies", energies)
    planted_fails(pins_fields.test_anisotropy_and_zeeman_energies)


# ---------------------------------------------------------------------------
# demag
# ---------------------------------------------------------------------------

def test_demag_fft_path_with_a_swapped_off_diagonal_is_caught(monkeypatch):
    pairs = dict(mm._PAIRS)
    pairs[(0, 1)] = pairs[(1, 0)] = 4  # N_xz where N_xy belongs
    pairs[(0, 2)] = pairs[(2, 0)] = 3
    orig = mm._convolve

    def convolve(p, M):
        saved = mm._PAIRS
        mm._PAIRS = pairs
        try:
            return orig(p, M)
        finally:
            mm._PAIRS = saved
    monkeypatch.setattr(mm, "_convolve", convolve)
    planted_fails(pins_tensor.test_fft_convolution_equals_direct_sum, (3, 5, 2))


def test_demag_without_the_minus_sign_is_caught(monkeypatch):
    orig = mm._convolve
    monkeypatch.setattr(mm, "_convolve", lambda p, M: -orig(p, M))
    planted_fails(pins_tensor.test_fft_convolution_equals_direct_sum, (3, 5, 2))


def test_tensor_with_swapped_off_diagonals_is_caught(monkeypatch):
    orig = tn.newell_closed_form

    def newell(*a):
        N = np.array(orig(*a), dtype=np.float64)
        return N[[0, 1, 2, 4, 3, 5]]
    monkeypatch.setattr(tn, "newell_closed_form", newell)
    planted_fails(pins_tensor.test_parity_of_components)


def test_tensor_with_a_wrong_self_factor_is_caught(monkeypatch):
    orig = tn.newell_closed_form

    def newell(*a):
        N = np.array(orig(*a), dtype=np.float64)
        N[2] *= 1.0 + 1e-6
        return N
    monkeypatch.setattr(tn, "newell_closed_form", newell)
    planted_fails(pins_tensor.test_self_term_trace_one_and_matches_aharoni, (1, 2, 3))


def test_full_tensor_with_a_wrong_parity_is_caught(monkeypatch):
    """N_xy taken as even in X when the octant is unfolded to signed offsets:
    the operator loses its symmetry and the unfolded and octant-based sums
    disagree."""
    orig = tn.tensor_full

    def full(nx, ny, nz, dx, dy, dz):
        f = orig(nx, ny, nz, dx, dy, dz)
        x = np.arange(-(nx - 1), nx)
        f[3] = f[3] * (np.sign(x) + (x == 0))[None, None, :]
        return f
    monkeypatch.setattr(tn, "tensor_full", full)
    planted_fails(pins_fields.test_linear_operator_is_ms_weighted_symmetric, False)
    planted_fails(pins_tensor.test_fft_convolution_equals_direct_sum, (3, 5, 2))


def test_full_tensor_without_any_parity_is_caught(monkeypatch):
    """Every component unfolded as even: still symmetric, but the prism sum of
    a uniform field no longer gives Aharoni's factors."""
    orig = tn.tensor_full

    def full(nx, ny, nz, dx, dy, dz):
        f = orig(nx, ny, nz, dx, dy, dz)
        o = f[:, nz - 1:nz, ny - 1:ny, nx - 1:nx]
        return np.abs(f) * np.where(o < 0, -1.0, 1.0)
    monkeypatch.setattr(tn, "tensor_full", full)
    planted_fails(pins_tensor.test_uniform_magnetisation_energy_equals_prism_factor, (6, 5, 4),
                  (2e-9, 2e-9, 2e-9))


# ---------------------------------------------------------------------------
# LLG and time stepping
# ---------------------------------------------------------------------------

def _llg(prec_sign=1.0, damp_sign=1.0, denom=lambda a: 1.0 + a * a):
    def llg_rhs(p, m, H):
        c = -p.gamma / denom(p.alpha)
        mxH = torch.linalg.cross(m, H, dim=-1)
        mxmxH = torch.linalg.cross(m, mxH, dim=-1)
        prec = mxH if p.precession else torch.zeros_like(mxH)
        return c * (prec_sign * prec + damp_sign * p.alpha * mxmxH)
    return llg_rhs


def test_llg_with_reversed_damping_is_caught(monkeypatch):
    monkeypatch.setattr(mm, "llg_rhs", _llg(damp_sign=-1.0))
    planted_fails(pins_fields.test_energy_decays_and_norm_conserved_plain)


def test_llg_with_reversed_precession_is_caught(monkeypatch):
    monkeypatch.setattr(mm, "llg_rhs", _llg(prec_sign=-1.0))
    planted_fails(pins_fields.test_macrospin_closed_form_and_rk4_order)


def test_llg_with_1_plus_alpha_for_1_plus_alpha_squared_is_caught(monkeypatch):
    monkeypatch.setattr(mm, "llg_rhs", _llg(denom=lambda a: 1.0 + a))
    planted_fails(pins_fields.test_macrospin_closed_form_and_rk4_order)


def test_llg_ignoring_the_precession_switch_is_caught(monkeypatch):
    def llg_rhs(p, m, H):
        c = -p.gamma / (1.0 + p.alpha ** 2)
        mxH = torch.linalg.cross(m, H, dim=-1)
        return c * (mxH + p.alpha * torch.linalg.cross(m, mxH, dim=-1))
    monkeypatch.setattr(mm, "llg_rhs", llg_rhs)
    planted_fails(pins_fields.test_macrospin_without_precession_relaxes_in_its_plane)


def test_rk4_with_wrong_weights_is_caught(monkeypatch):
    def rk4(p, m0, dt, f=None):
        f = f or (lambda x: mm.rhs(p, x))
        k1 = f(m0)
        k2 = f(mm.normalize(m0 + 0.5 * dt * k1))
        k3 = f(mm.normalize(m0 + 0.5 * dt * k2))
        k4 = f(mm.normalize(m0 + dt * k3))
        return mm.normalize(m0 + (dt / 6.0) * (k1 + k2 + 2.0 * k3 + 2.0 * k4))
    monkeypatch.setattr(mm, "rk4_step", rk4)
    planted_fails(pins_fields.test_macrospin_closed_form_and_rk4_order)


def test_rk4_without_renormalisation_is_caught(monkeypatch):
    def rk4(p, m0, dt, f=None):
        f = f or (lambda x: mm.rhs(p, x))
        k1 = f(m0)
        k2 = f(m0 + 0.5 * dt * k1)
        k3 = f(m0 + 0.5 * dt * k2)
        k4 = f(m0 + dt * k3)
        return m0 + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    monkeypatch.setattr(mm, "rk4_step", rk4)
    planted_fails(pins_fields.test_energy_decays_and_norm_conserved_plain)


def test_euler_without_renormalisation_is_caught(monkeypatch):
    monkeypatch.setattr(mm, "euler_step", lambda p, m0, dt, f=None: m0 + dt * (f or (lambda x: mm.rhs(p, x)))(m0))
    planted_fails(pins_fields.test_macrospin_forward_euler_is_first_order_with_unit_norm)


def test_euler_with_half_the_step_is_caught(monkeypatch):
    orig = mm.euler_step
    monkeypatch.setattr(mm, "euler_step", lambda p, m0, dt, f=None: orig(p, m0, 0.5 * dt, f))
    planted_fails(pins_fields.test_macrospin_forward_euler_is_first_order_with_unit_norm)


def test_normalisation_by_the_squared_norm_is_caught(monkeypatch):
    monkeypatch.setattr(mm, "normalize", lambda m: m / (m * m).sum(-1, keepdim=True))
    planted_fails(pins_fields.test_energy_decays_and_norm_conserved_plain)


def test_central_exchange_energy_with_a_one_sided_step_is_caught(monkeypatch):
    orig = mm.exchange_energy_central
    monkeypatch.setattr(mm, "exchange_energy_central", lambda p, m: 4.0 * orig(p, m))
    planted_fails(pins_sp3.test_central_exchange_energy_of_a_helix)


# ---------------------------------------------------------------------------
# MRI
# ---------------------------------------------------------------------------

def test_mri_forcing_without_the_difference_of_rows_is_caught(monkeypatch):
    """r_i = sum_j a_ij f_slow(Y_j) / dc instead of (a_ij - a_{i-1,j})."""
    def mri_step(p, m, h, ratio=0.1, renorm=True, fast=None, slow=None):
        fast = fast or (lambda x: mri.fast_rhs(p, x))
        slow = slow or (lambda x: mri.slow_rhs(p, x))
        a = mri.KW3_A + (mri.KW3_B,)
        c = mri.KW3_C + (1.0,)
        Y, F = [m], []
        for i in range(1, 4):
            F.append(slow(Y[i - 1]))
            dc = c[i] - c[i - 1]
            r = sum(a[i][j] * F[j] for j in range(i)) / dc
            n = mri.fast_steps(dc, ratio)
            v = Y[i - 1]
            for _ in range(n):
                v = mri.kw3_step(lambda x: fast(x) + r, v, dc * h / n, renorm)
            Y.append(v)
        return Y[3]
    monkeypatch.setattr(mri, "mri_step", mri_step)
    planted_fails(pins_mri.test_without_fast_part_it_is_the_single_rate_method)


def test_fast_step_count_rounded_down_is_caught(monkeypatch):
    monkeypatch.setattr(mri, "fast_steps", lambda interval, ratio: max(1, math.floor(interval / ratio)))
    planted_fails(pins_mri.test_fast_step_counts)


def test_knoth_wolke_with_a_wrong_weight_is_caught(monkeypatch):
    monkeypatch.setattr(mri, "KW3_B", (1.0 / 6.0, 3.0 / 10.0, 7.0 / 15.0))
    planted_fails(pins_mri.test_knoth_wolke_tableau_is_third_order)


# ---------------------------------------------------------------------------
# learned surrogates
# ---------------------------------------------------------------------------

def test_gelu_with_the_tanh_approximation_is_caught(monkeypatch):
    monkeypatch.setattr(cnn, "gelu", lambda x: 0.5 * x * (1.0 + torch.tanh(
        math.sqrt(2.0 / math.pi) * (x + 0.044715 * x ** 3))))
    planted_fails(pins_cnn.test_gelu_closed_values)


def test_adam_without_bias_correction_is_caught(monkeypatch):
    def adam(flat, grad, m, v, t, lr, wd, beta1=0.9, beta2=0.999, eps=1e-8):
        flat, grad, m, v = (torch.as_tensor(a, dtype=torch.float64) for a in (flat, grad, m, v))
        g = grad + wd * flat
        m = beta1 * m + (1.0 - beta1) * g
        v = beta2 * v + (1.0 - beta2) * g * g
        return flat - lr * m / (v.sqrt() + eps), m, v
    monkeypatch.setattr(cnn, "adam_step", adam)
    planted_fails(pins_cnn.test_adam_first_step_by_hand)


def test_fno_without_the_high_corner_is_caught(monkeypatch):
    def spectral_conv(v, R, K):
        B, C, H, W = v.shape
        X = torch.fft.rfft2(v)
        Rc = torch.complex(R[..., 0], R[..., 1])
        Y = torch.einsum("bimn,mnio->bomn", X[:, :, :K, :K], Rc[:K])
        out = torch.zeros(B, R.shape[3], H, W // 2 + 1, dtype=torch.complex128)
        out[:, :, :K, :K] = Y
        return torch.fft.irfft2(out, s=(H, W))
    monkeypatch.setattr(fno, "spectral_conv", spectral_conv)
    planted_fails(pins_fno.test_plane_wave_passes_or_is_removed, -3, 2, 1.0)


def test_fno_inverse_as_the_real_part_of_a_full_inverse_is_caught(monkeypatch):
    """Half spectrum put into a full complex inverse FFT, real part taken:
    the mirror half of every kx > 0 mode is lost."""
    def spectral_conv(v, R, K):
        B, C, H, W = v.shape
        X = torch.fft.rfft2(v)
        rows = fno.kept_rows(H, K)
        Rc = torch.complex(R[..., 0], R[..., 1])
        Y = torch.einsum("bimn,mnio->bomn", X[:, :, rows, :K], Rc)
        out = torch.zeros(B, R.shape[3], H, W, dtype=torch.complex128)
        out[:, :, rows, :K] = Y
        return torch.fft.ifft2(out).real
    monkeypatch.setattr(fno, "spectral_conv", spectral_conv)
    planted_fails(pins_fno.test_spectral_conv_matches_explicit_sums, 6, 5, 2)


def test_fno_filter_transpose_without_conjugation_is_caught(monkeypatch):
    monkeypatch.setattr(fno, "adjoint_filters", lambda R: R.transpose(2, 3).clone())
    planted_fails(pins_fno.test_adjoint_filters_transpose_the_spectral_convolution)


# ---------------------------------------------------------------------------
# discrete adjoint
# ---------------------------------------------------------------------------



def test_demag_vjp_without_the_ms_factor_is_caught(monkeypatch, setup):  # noqa: F811
    def backward(ctx, g):
        m, Ms = ctx.saved_tensors
        u = torch.from_numpy(mm._convolve(ctx.p, g.detach().numpy()))
        return u, (m * u).sum(-1), None
    monkeypatch.setattr(mm._DemagOp, "backward", staticmethod(backward))
    planted_fails(pins_adj.test_dot_product_tangent_linear_vs_adjoint, setup)


def test_demag_vjp_without_its_ms_gradient_is_caught(monkeypatch, setup):  # noqa: F811
    def backward(ctx, g):
        m, Ms = ctx.saved_tensors
        u = torch.from_numpy(mm._convolve(ctx.p, g.detach().numpy()))
        return Ms[..., None] * u, torch.zeros_like(Ms), None
    monkeypatch.setattr(mm._DemagOp, "backward", staticmethod(backward))
    planted_fails(pins_adj.test_dot_product_tangent_linear_vs_adjoint, setup)


def _planted_gradient(state_offset=0, skip_normalisation=False, ms_last_step_only=False):
    """The oracle's reverse sweep with one planted mistake."""
    from oracle import adjoint as adj

    def gradient(p, m0_raw, dt, nsteps, objective):
        m0_raw = mm.as_t(m0_raw).detach()
        Ms = mm.ms_field(p).detach().clone()
        states = adj.forward_states(adj._with_ms(p, Ms), m0_raw, dt, nsteps)
        mT = states[-1].detach().requires_grad_(True)
        J = objective(mT)
        lam, = torch.autograd.grad(J, mT)
        g_ms = torch.zeros_like(Ms)
        for s in range(nsteps - 1, -1, -1):
            ms_var = Ms.clone().requires_grad_(True)
            q = adj._with_ms(p, ms_var)
            ms_in = states[s + state_offset].detach().requires_grad_(True)
            out = mm.rk4_step(q, ms_in, dt)
            lam, gms = torch.autograd.grad(out, (ms_in, ms_var), grad_outputs=lam)
            g_ms = gms if ms_last_step_only else g_ms + gms
        if skip_normalisation:
            return float(J.detach()), lam.detach(), g_ms.detach()
        raw = m0_raw.clone().requires_grad_(True)
        g_raw, = torch.autograd.grad(mm.normalize(raw), raw, grad_outputs=lam)
        return float(J.detach()), g_raw.detach(), g_ms.detach()
    return gradient


def test_reverse_sweep_on_the_wrong_stored_state_is_caught(monkeypatch, setup):  # noqa: F811
    from oracle import adjoint as adj
    monkeypatch.setattr(adj, "gradient", _planted_gradient(state_offset=1))
    planted_fails(pins_adj.test_dot_product_tangent_linear_vs_adjoint, setup)


def test_gradient_without_the_initial_normalisation_is_caught(monkeypatch, setup):  # noqa: F811
    from oracle import adjoint as adj
    monkeypatch.setattr(adj, "gradient", _planted_gradient(skip_normalisation=True))
    planted_fails(pins_adj.test_dot_product_tangent_linear_vs_adjoint, setup)


def test_ms_gradient_of_the_last_step_only_is_caught(monkeypatch, setup):  # noqa: F811
    from oracle import adjoint as adj
    monkeypatch.setattr(adj, "gradient", _planted_gradient(ms_last_step_only=True))
    planted_fails(pins_adj.test_dot_product_tangent_linear_vs_adjoint, setup)


def test_planted_gradient_without_a_mistake_passes(monkeypatch, setup):  # noqa: F811
    """Control: the planting helper itself reproduces the oracle's sweep."""
    from oracle import adjoint as adj
    monkeypatch.setattr(adj, "gradient", _planted_gradient())
    pins_adj.test_dot_product_tangent_linear_vs_adjoint(setup)
