"""Oracle: the micromagnetic right-hand side, time stepping and energies.

TEST INFRASTRUCTURE ONLY.  A plain, slow FP64 CPU restatement of the paper's
method that the CUDA path is checked against; the product never imports it.
Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may call it.

Arrays: a magnetisation field ``m`` has shape (nz, ny, nx, 3) (cell (i, j, k)
at ``m[k, j, i]``), float64 torch tensors on the CPU.  Material maps (Ms, Ku)
are scalars or (nz, ny, nx) arrays; the easy axis is a 3-vector or an
(nz, ny, nx, 3) array.

Paper passages followed (MagneX, Sec. II):
  * LLG right-hand side, Eq. (1), with gamma_L = gamma/(1+alpha^2); written
    for m = M/Ms with gamma0 = mu0*|gamma| > 0:
        dm/dt = -gamma0/(1+alpha^2) [ m x H + alpha m x (m x H) ].
  * H_eff = H_bias + H_demag + H_ani + H_exch + H_DMI, Eq. (2).
  * Demag: H_d(r) = -sum_r' N(r - r') Ms m(r') (sign so that a cube's
    self-factor is 1/3), computed as a zero-padded FFT convolution on a grid of
    twice the problem size (Sec. II-B), or as the direct sum.
  * Anisotropy: H = 2 Ku/(mu0 Ms) (m . e_K) e_K; energy density
    Ku [1 - (e_K . m)^2].
  * Exchange: (2/(mu0 Ms^2)) div(A grad M) with second-order central
    differences (Sec. II-B): H_i = 2A/(mu0 Ms_i) sum_d (m_{i+d} + m_{i-d} - 2 m_i)/h_d^2.
  * Interfacial DMI: H = (2D/(mu0 Ms)) [grad m_z - (div m) e_z], in-plane
    derivatives only, central differences.
  * Boundary: Neumann without DMI; with DMI the inhomogeneous condition
    dm/dx_k = -(D/2A)(e_z x e_k) x m, imposed through a ghost cell
    m_g = m_b - h (D/2A) (e_z x n) x m_b at outward normal n (this reduces to
    m_g = m_b on z faces and whenever D = 0).
  * Renormalisation |m| = 1 after every stage and step (Sec. II-B).
  * Classical RK4 (Sec. III, four right-hand-side evaluations per step) and
    forward Euler (Sec. II-D, III-E).
"""
from dataclasses import dataclass, field
import math
import os

import numpy as np
import scipy.fft as sfft
import torch

from . import tensor as _tensor

MU0 = 4e-7 * math.pi
DT = torch.float64


@dataclass
class Problem:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    Ms: object = 8.0e5          # scalar or (nz, ny, nx)
    A: float = 1.3e-11
    Ku: object = 0.0            # scalar or (nz, ny, nx)
    ku_axis: object = (0.0, 0.0, 1.0)  # 3-vector or (nz, ny, nx, 3)
    D: float = 0.0
    alpha: float = 0.5
    gamma: float = 2.211e5      # gamma0 = mu0 |gamma|, m/(A s)
    h_bias: tuple = (0.0, 0.0, 0.0)
    dmi: bool = False           # interfacial DMI with chiral boundary ghosts
    precession: bool = True
    demag: bool = True
    _cache: dict = field(default_factory=dict, repr=False, compare=False)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def V(self):
        return self.dx * self.dy * self.dz


def as_t(x):
    if isinstance(x, torch.Tensor):
        return x.to(DT)
    return torch.as_tensor(np.asarray(x, dtype=np.float64))


def ms_field(p):
    Ms = as_t(p.Ms)
    return Ms.expand(p.shape) if Ms.ndim == 0 else Ms


def normalize(m):
    return m / torch.linalg.vector_norm(m, dim=-1, keepdim=True)


# --------------------------------------------------------------------------
# Demagnetisation
# --------------------------------------------------------------------------

def _workers():
    return os.cpu_count() or 1


def padded_tensor_spectrum(p):
    """rfftn of the tensor placed on the 2n-padded grid, shape (6, Pz, Py, Px//2+1), complex numpy."""
    key = "Nhat"
    if key in p._cache:
        return p._cache[key]
    nx, ny, nz = p.nx, p.ny, p.nz
    Px, Py, Pz = 2 * nx, 2 * ny, 2 * nz
    full = _tensor.tensor_full(nx, ny, nz, p.dx, p.dy, p.dz)
    Npad = np.zeros((6, Pz, Py, Px))
    oz = np.arange(-(nz - 1), nz) % Pz
    oy = np.arange(-(ny - 1), ny) % Py
    ox = np.arange(-(nx - 1), nx) % Px
    Npad[np.ix_(range(6), oz, oy, ox)] = full
    del full
    Nhat = sfft.rfftn(Npad, axes=(1, 2, 3), workers=_workers())
    p._cache[key] = Nhat
    return Nhat


_PAIRS = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3,
          (0, 2): 4, (2, 0): 4, (1, 2): 5, (2, 1): 5}


def _convolve(p, M):
    """-N * M for a (nz, ny, nx, 3) numpy field M (exact linear convolution by
    zero padding to twice the grid)."""
    nx, ny, nz = p.nx, p.ny, p.nz
    Px, Py, Pz = 2 * nx, 2 * ny, 2 * nz
    Mpad = np.zeros((3, Pz, Py, Px))
    Mpad[:, :nz, :ny, :nx] = np.moveaxis(M, -1, 0)
    Mhat = sfft.rfftn(Mpad, axes=(1, 2, 3), workers=_workers())
    del Mpad
    Nhat = padded_tensor_spectrum(p)
    H = np.empty((nz, ny, nx, 3))
    for i in range(3):
        Hhat = -sum(Nhat[_PAIRS[(i, j)]] * Mhat[j] for j in range(3))
        H[..., i] = sfft.irfftn(Hhat, s=(Pz, Py, Px), axes=(0, 1, 2), workers=_workers())[:nz, :ny, :nx]
    return H


class _DemagOp(torch.autograd.Function):
    """H_d = -N * (Ms m).  Forward is the plain FFT convolution.  Backward (used
    only by the discrete adjoint) relies on the convolution being self-adjoint,
    N_ij(-R) = N_ji(R), which the oracle's symmetry pin checks."""

    @staticmethod
    def forward(ctx, m, Ms, p):
        ctx.p = p
        ctx.save_for_backward(m, Ms)
        ctx.save_for_forward(m, Ms)
        M = (Ms[..., None] * m).detach().numpy()
        return torch.from_numpy(_convolve(p, M))

    @staticmethod
    def jvp(ctx, m_t, Ms_t, p_t):
        """Tangent (forward mode, used by the tangent-linear check of the
        adjoint): the operator is linear in Ms m, so the tangent is the same
        convolution of Ms dm + dMs m; no symmetry of N is assumed."""
        m, Ms = ctx.saved_tensors
        src = torch.zeros_like(m)
        if m_t is not None:
            src = src + Ms[..., None] * m_t
        if Ms_t is not None:
            src = src + Ms_t[..., None] * m
        return torch.from_numpy(_convolve(ctx.p, src.detach().numpy()))

    @staticmethod
    def backward(ctx, g):
        m, Ms = ctx.saved_tensors
        u = torch.from_numpy(_convolve(ctx.p, g.detach().numpy()))
        return Ms[..., None] * u, (m * u).sum(-1), None


def demag_field(p, m):
    """H_d by zero-padded FFT convolution (exact linear convolution)."""
    return _DemagOp.apply(m, ms_field(p).contiguous(), p)


def demag_field_direct(p, m):
    """H_d by the direct O(N^2) real-space sum (tiny grids only)."""
    nx, ny, nz = p.nx, p.ny, p.nz
    full = torch.from_numpy(_tensor.tensor_full(nx, ny, nz, p.dx, p.dy, p.dz))
    M = (ms_field(p)[..., None] * m).reshape(-1, 3)
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kk, jj, ii = kk.ravel(), jj.ravel(), ii.ravel()
    dk = kk[:, None] - kk[None, :] + nz - 1
    dj = jj[:, None] - jj[None, :] + ny - 1
    di = ii[:, None] - ii[None, :] + nx - 1
    H = torch.zeros((kk.size, 3), dtype=DT)
    for i in range(3):
        for j in range(3):
            Nij = full[_PAIRS[(i, j)]][dk, dj, di]  # (target, source)
            H[:, i] -= Nij @ M[:, j]
    return H.reshape(nz, ny, nx, 3)


def demag_field_at(p, m, targets, octant=None):
    """H_d at selected target cells (k, j, i) by the direct sum over all sources.

    Uses the tensor octant and each component's parity, so it scales to large
    grids for a handful of targets.
    """
    nx, ny, nz = p.nx, p.ny, p.nz
    if octant is None:
        octant = _tensor.tensor_octant(nx, ny, nz, p.dx, p.dy, p.dz)
    M = (ms_field(p)[..., None] * m).numpy()
    out = np.zeros((len(targets), 3))
    ks, js, is_ = np.arange(nz), np.arange(ny), np.arange(nx)
    for t, (k, j, i) in enumerate(targets):
        ox, oy, oz = i - is_, j - js, k - ks
        ax, ay, az = np.abs(ox), np.abs(oy), np.abs(oz)
        sx, sy, sz = np.where(ox < 0, -1.0, 1.0), np.where(oy < 0, -1.0, 1.0), np.where(oz < 0, -1.0, 1.0)
        for a in range(3):
            acc = 0.0
            for b in range(3):
                c = _PAIRS[(a, b)]
                px, py, pz = _tensor.PARITY[_tensor.COMPONENTS[c]]
                Nsub = octant[c][np.ix_(az, ay, ax)]
                f = ((sz if pz < 0 else np.ones(nz))[:, None, None]
                     * (sy if py < 0 else np.ones(ny))[None, :, None]
                     * (sx if px < 0 else np.ones(nx))[None, None, :])
                acc += np.sum(Nsub * f * M[..., b])
            out[t, a] = -acc
    return out


# --------------------------------------------------------------------------
# Local fields
# --------------------------------------------------------------------------

def ghosted(p, m):
    """m with one layer of face ghost cells, shape (nz+2, ny+2, nx+2, 3).

    Ghost at outward normal n: m_g = m_b - h (D/2A) (e_z x n) x m_b
    (Neumann, m_g = m_b, when DMI is off).  Edge and corner ghosts are never
    read by the 6-point and central-difference stencils.
    """
    nz, ny, nx = p.shape
    mp = torch.zeros((nz + 2, ny + 2, nx + 2, 3), dtype=DT)
    mp[1:-1, 1:-1, 1:-1] = m
    kappa = p.D / (2.0 * p.A) if (p.dmi and p.A != 0.0) else 0.0
    ez = torch.tensor([0.0, 0.0, 1.0], dtype=DT)

    def ghost(mb, normal, h):
        n = torch.tensor(normal, dtype=DT)
        t = torch.linalg.cross(ez, n)
        return mb - h * kappa * torch.linalg.cross(t.expand_as(mb), mb, dim=-1)

    mp[1:-1, 1:-1, 0] = ghost(m[:, :, 0], (-1.0, 0.0, 0.0), p.dx)
    mp[1:-1, 1:-1, -1] = ghost(m[:, :, -1], (1.0, 0.0, 0.0), p.dx)
    mp[1:-1, 0, 1:-1] = ghost(m[:, 0, :], (0.0, -1.0, 0.0), p.dy)
    mp[1:-1, -1, 1:-1] = ghost(m[:, -1, :], (0.0, 1.0, 0.0), p.dy)
    mp[0, 1:-1, 1:-1] = ghost(m[0], (0.0, 0.0, -1.0), p.dz)
    mp[-1, 1:-1, 1:-1] = ghost(m[-1], (0.0, 0.0, 1.0), p.dz)
    return mp


def exchange_field(p, m, mp=None):
    if mp is None:
        mp = ghosted(p, m)
    c = mp[1:-1, 1:-1, 1:-1]
    lap = ((mp[1:-1, 1:-1, 2:] + mp[1:-1, 1:-1, :-2] - 2 * c) / p.dx ** 2
           + (mp[1:-1, 2:, 1:-1] + mp[1:-1, :-2, 1:-1] - 2 * c) / p.dy ** 2
           + (mp[2:, 1:-1, 1:-1] + mp[:-2, 1:-1, 1:-1] - 2 * c) / p.dz ** 2)
    return (2.0 * p.A / (MU0 * ms_field(p)))[..., None] * lap


def dmi_field(p, m, mp=None):
    if not p.dmi or p.D == 0.0:
        return torch.zeros_like(m)
    if mp is None:
        mp = ghosted(p, m)
    ddx = (mp[1:-1, 1:-1, 2:] - mp[1:-1, 1:-1, :-2]) / (2 * p.dx)
    ddy = (mp[1:-1, 2:, 1:-1] - mp[1:-1, :-2, 1:-1]) / (2 * p.dy)
    H = torch.stack([ddx[..., 2], ddy[..., 2], -(ddx[..., 0] + ddy[..., 1])], dim=-1)
    return (2.0 * p.D / (MU0 * ms_field(p)))[..., None] * H


def anisotropy_field(p, m):
    Ku = as_t(p.Ku)
    e = as_t(p.ku_axis)
    if e.ndim == 1:
        e = e.expand(m.shape)
    proj = (m * e).sum(-1, keepdim=True)
    coef = 2.0 * Ku / (MU0 * ms_field(p))
    if coef.ndim > 0:
        coef = coef[..., None]
    return coef * proj * e


def zeeman_field(p, m):
    return as_t(p.h_bias).expand(m.shape).clone()


def field_terms(p, m):
    mp = ghosted(p, m)
    return {
        "demag": demag_field(p, m) if p.demag else torch.zeros_like(m),
        "exch": exchange_field(p, m, mp),
        "anis": anisotropy_field(p, m),
        "dmi": dmi_field(p, m, mp),
        "zeeman": zeeman_field(p, m),
    }


def heff(p, m):
    t = field_terms(p, m)
    return t["demag"] + t["exch"] + t["anis"] + t["dmi"] + t["zeeman"]


def heff_local(p, m):
    """H_eff without the demag term."""
    mp = ghosted(p, m)
    return exchange_field(p, m, mp) + anisotropy_field(p, m) + dmi_field(p, m, mp) + zeeman_field(p, m)


# --------------------------------------------------------------------------
# LLG and time stepping
# --------------------------------------------------------------------------

def llg_rhs(p, m, H):
    c = -p.gamma / (1.0 + p.alpha ** 2)
    mxH = torch.linalg.cross(m, H, dim=-1)
    mxmxH = torch.linalg.cross(m, mxH, dim=-1)
    prec = mxH if p.precession else torch.zeros_like(mxH)
    return c * (prec + p.alpha * mxmxH)


def rhs(p, m):
    return llg_rhs(p, m, heff(p, m))


def rk4_step(p, m0, dt, f=None):
    """One classical RK4 step with renormalisation of every stage input and of the result."""
    f = f or (lambda x: rhs(p, x))
    k1 = f(m0)
    m1 = normalize(m0 + 0.5 * dt * k1)
    k2 = f(m1)
    m2 = normalize(m0 + 0.5 * dt * k2)
    k3 = f(m2)
    m3 = normalize(m0 + dt * k3)
    k4 = f(m3)
    return normalize(m0 + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4))


def euler_step(p, m0, dt, f=None):
    """One forward Euler step, m1 = normalize(m0 + dt f(m0)) (Sec. II-D, III-E)."""
    f = f or (lambda x: rhs(p, x))
    return normalize(m0 + dt * f(m0))


def run(p, m, dt, nsteps, method="rk4"):
    m = normalize(as_t(m))
    step = rk4_step if method == "rk4" else euler_step
    for _ in range(nsteps):
        m = step(p, m, dt)
    return m


# --------------------------------------------------------------------------
# Energies (J)
# --------------------------------------------------------------------------

def exchange_energy_central(p, m):
    """Exchange energy V sum_cells A |grad m|^2 with every derivative a
    second-order central difference (m_{i+1} - m_{i-1}) / (2h) over the same
    ghost cells as the field (Eq. for e_exch in Sec. II-A with the central
    stencils of Sec. II-B).  This is the energy the paper tabulates; the
    exchange term of ``energies`` is the variational one (-mu0/2 Ms m.H_exch,
    face differences), whose gradient is the field."""
    mp = ghosted(p, m)
    gx = (mp[1:-1, 1:-1, 2:] - mp[1:-1, 1:-1, :-2]) / (2 * p.dx)
    gy = (mp[1:-1, 2:, 1:-1] - mp[1:-1, :-2, 1:-1]) / (2 * p.dy)
    gz = (mp[2:, 1:-1, 1:-1] - mp[:-2, 1:-1, 1:-1]) / (2 * p.dz)
    return float(p.V * p.A * ((gx ** 2).sum() + (gy ** 2).sum() + (gz ** 2).sum()))


def energies(p, m):
    """Demag, exchange, DMI: -mu0/2 V sum Ms m.H_term; anisotropy: V sum Ku[1-(e.m)^2];
    Zeeman: -mu0 V sum Ms m.H_bias (Sec. II-A energy densities, with the Ms factor
    of the demag density written out)."""
    t = field_terms(p, m)
    Ms = ms_field(p)
    V = p.V

    def quad(H):
        return float(-0.5 * MU0 * V * (Ms * (m * H).sum(-1)).sum())

    e = as_t(p.ku_axis)
    if e.ndim == 1:
        e = e.expand(m.shape)
    Ku = as_t(p.Ku).expand(p.shape)
    anis = float(V * (Ku * (1.0 - (m * e).sum(-1) ** 2)).sum())
    zee = float(-MU0 * V * (Ms * (m * t["zeeman"]).sum(-1)).sum())
    return {"demag": quad(t["demag"]), "exch": quad(t["exch"]), "anis": anis,
            "dmi": quad(t["dmi"]), "zeeman": zee}
