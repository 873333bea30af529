"""Oracle: discrete adjoint of the RK4 time stepping (gradient of a final-state
objective with respect to the initial magnetisation and the Ms map).

TEST INFRASTRUCTURE ONLY (plain FP64 CPU; the product never imports it).

The gradient is the exact derivative of the oracle's own discrete forward map
(``micromag.rk4_step`` with renormalisation after every stage), taken one
step at a time: the forward run keeps every step's state, and the backward run
recomputes each step from its stored state under torch autograd and pulls the
cotangent back through it.  The objective sees m_T = F^T(normalize(m0)), so the
m0 gradient includes the initial renormalisation.  The demag operator's
backward uses the self-adjointness of the tensor convolution, which the
oracle's symmetry pin checks.  Finite differences pin this module (tests).
"""
import numpy as np
import torch

from . import micromag as mm


def patch_mean_mz(m, patch):
    """Mean of m_z over the cells [y0, y1) x [x0, x1) of every z plane."""
    (y0, y1), (x0, x1) = patch
    return m[:, y0:y1, x0:x1, 2].mean()


def _with_ms(p, Ms):
    q = mm.Problem(**{k: getattr(p, k) for k in ("nx", "ny", "nz", "dx", "dy", "dz", "A", "Ku", "ku_axis", "D",
                                                "alpha", "gamma", "h_bias", "dmi", "precession", "demag")},
                   Ms=Ms)
    q._cache = p._cache  # the tensor spectrum depends on the geometry only
    return q


def forward_states(p, m0_raw, dt, nsteps):
    """States m_0 = normalize(m0_raw), m_1, ..., m_nsteps (no gradient tracking)."""
    with torch.no_grad():
        m = mm.normalize(mm.as_t(m0_raw))
        states = [m]
        for _ in range(nsteps):
            m = mm.rk4_step(p, m, dt)
            states.append(m)
    return states


def gradient(p, m0_raw, dt, nsteps, objective):
    """(J, dJ/dm0_raw, dJ/dMs) for J = objective(m_nsteps).

    p.Ms may be a scalar or an (nz, ny, nx) map; the Ms gradient has the
    map's shape (per-cell) either way.
    """
    m0_raw = mm.as_t(m0_raw).detach()
    Ms = mm.ms_field(p).detach().clone()
    states = forward_states(_with_ms(p, Ms), m0_raw, dt, nsteps)
    mT = states[-1].detach().requires_grad_(True)
    J = objective(mT)
    lam, = torch.autograd.grad(J, mT)
    g_ms = torch.zeros_like(Ms)
    for s in range(nsteps - 1, -1, -1):
        ms_var = Ms.clone().requires_grad_(True)
        q = _with_ms(p, ms_var)
        ms_in = states[s].detach().requires_grad_(True)
        out = mm.rk4_step(q, ms_in, dt)
        lam, gms = torch.autograd.grad(out, (ms_in, ms_var), grad_outputs=lam)
        g_ms += gms
    raw = m0_raw.clone().requires_grad_(True)
    m0 = mm.normalize(raw)
    g_raw, = torch.autograd.grad(m0, raw, grad_outputs=lam)
    return float(J.detach()), g_raw.detach(), g_ms.detach()


def objective_value(p, m0_raw, dt, nsteps, objective, Ms=None):
    q = p if Ms is None else _with_ms(p, mm.as_t(Ms))
    with torch.no_grad():
        return float(objective(forward_states(q, m0_raw, dt, nsteps)[-1]))


def central_fd(p, m0_raw, dt, nsteps, objective, direction_m=None, direction_ms=None, h=1e-4):
    """Central difference of J along (direction_m in m0_raw, direction_ms in Ms)."""
    m0 = mm.as_t(m0_raw)
    Ms = mm.ms_field(p).clone()
    dm = torch.zeros_like(m0) if direction_m is None else mm.as_t(direction_m)
    ds = torch.zeros_like(Ms) if direction_ms is None else mm.as_t(direction_ms)
    jp = objective_value(p, m0 + h * dm, dt, nsteps, objective, Ms + h * ds)
    jm = objective_value(p, m0 - h * dm, dt, nsteps, objective, Ms - h * ds)
    return (jp - jm) / (2 * h)


def tangent_linear(p, m0_raw, dt, nsteps, dm0, dms=None):
    """Tangent-linear model: the directional derivative of m_nsteps along
    (dm0 in m0_raw, dms in Ms), by forward-mode differentiation of the same
    discrete forward map (independent of the reverse sweep in ``gradient``)."""
    import torch.autograd.forward_ad as fwd
    m0_raw = mm.as_t(m0_raw).detach()
    Ms = mm.ms_field(p).detach().clone()
    dms = torch.zeros_like(Ms) if dms is None else mm.as_t(dms)
    with fwd.dual_level():
        q = _with_ms(p, fwd.make_dual(Ms, dms))
        m = mm.normalize(fwd.make_dual(m0_raw, mm.as_t(dm0)))
        for _ in range(nsteps):
            m = mm.rk4_step(q, m, dt)
        return fwd.unpack_dual(m).tangent.detach()
