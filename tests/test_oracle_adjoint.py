"""Pins for the oracle's discrete adjoint: central finite differences of the
oracle's own forward map (CPU only)."""
import numpy as np
import pytest
import torch

from oracle import adjoint as adj
from oracle import micromag as mm


@pytest.fixture(scope="module")
def setup():
    rng = np.random.default_rng(21)
    shape = (1, 8, 10)
    Ms = rng.uniform(6e5, 1e6, size=shape)
    p = mm.Problem(10, 8, 1, 2e-9, 2e-9, 2e-9, Ms=Ms, A=1.3e-11, D=2e-3, dmi=True, alpha=0.3,
                   h_bias=(0.0, 0.0, 1e5), Ku=2e4, ku_axis=(0.2, 0.1, 1.0))
    m0 = rng.normal(size=shape + (3,)) * 1.3
    obj = lambda m: adj.patch_mean_mz(m, ((2, 6), (3, 7)))  # noqa: E731
    J, g_m, g_ms = adj.gradient(p, m0, 2e-14, 12, obj)
    return p, m0, obj, J, g_m, g_ms, rng


def test_gradient_wrt_m0_matches_central_differences(setup):
    p, m0, obj, J, g_m, g_ms, rng = setup
    for _ in range(3):
        d = rng.normal(size=m0.shape)
        fd = adj.central_fd(p, m0, 2e-14, 12, obj, direction_m=d, h=1e-6)
        an = float((g_m * torch.from_numpy(d)).sum())
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-12, (fd, an)
    # single entries
    for idx in [(0, 4, 5, 2), (0, 0, 0, 0), (0, 7, 9, 1)]:
        d = np.zeros(m0.shape)
        d[idx] = 1.0
        fd = adj.central_fd(p, m0, 2e-14, 12, obj, direction_m=d, h=1e-6)
        assert abs(fd - float(g_m[idx])) <= 1e-5 * float(g_m.abs().max()), (idx, fd, float(g_m[idx]))


def test_gradient_wrt_ms_matches_central_differences(setup):
    p, m0, obj, J, g_m, g_ms, rng = setup
    for _ in range(2):
        d = rng.normal(size=(1, 8, 10)) * 1e3
        fd = adj.central_fd(p, m0, 2e-14, 12, obj, direction_ms=d, h=1e-2)
        an = float((g_ms * torch.from_numpy(d)).sum())
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-14, (fd, an)


def test_gradient_is_tangent_to_the_initial_normalisation(setup):
    """J depends on m0 only through m0/|m0|, so dJ/dm0 is orthogonal to m0 in every cell."""
    p, m0, obj, J, g_m, g_ms, rng = setup
    dots = (g_m * torch.from_numpy(m0)).sum(-1)
    assert float(dots.abs().max()) <= 1e-12 * float(g_m.abs().max()) * np.abs(m0).max()


def test_dot_product_tangent_linear_vs_adjoint(setup):
    """<TLM d, w> = <d, ADJ w> for random d (in m0 and Ms) and w: the
    forward-mode tangent of the run and the step-wise reverse sweep are two
    independent derivatives of the same discrete map."""
    p, m0, obj, J, g_m, g_ms, rng = setup
    for _ in range(2):
        w = torch.from_numpy(rng.normal(size=m0.shape))
        dm = rng.normal(size=m0.shape)
        ds = rng.normal(size=(1, 8, 10)) * 1e4
        _, gw_m, gw_ms = adj.gradient(p, m0, 2e-14, 12, lambda m: (m * w).sum())
        tl = adj.tangent_linear(p, m0, 2e-14, 12, dm, ds)
        lhs = float((tl * w).sum())
        rhs = float((gw_m * torch.from_numpy(dm)).sum() + (gw_ms * torch.from_numpy(ds)).sum())
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs), (lhs, rhs)


@pytest.mark.parametrize("precession", [True, False])
def test_llg_vector_jacobian_products_closed_form(precession):
    """For f = c [m x H + alpha m x (m x H)], c = -gamma0/(1+alpha^2), and a
    cotangent v, the products the GPU adjoint kernel evaluates:
      d/dm: c [alpha ((m.H) v + (v.m) H - 2 (v.H) m) + H x v]
      d/dH: c [alpha ((v.m) m - (m.m) v) + v x m]
    (cross-product terms only with precession), against autograd of the
    oracle's llg_rhs; m need not be a unit vector."""
    rng = np.random.default_rng(23)
    p = mm.Problem(3, 2, 1, 2e-9, 2e-9, 2e-9, alpha=0.27, precession=precession)
    m = torch.from_numpy(rng.normal(size=(1, 2, 3, 3))).requires_grad_(True)
    H = torch.from_numpy(rng.normal(size=(1, 2, 3, 3)) * 1e4).requires_grad_(True)
    v = torch.from_numpy(rng.normal(size=(1, 2, 3, 3)))
    gm, gH = torch.autograd.grad(mm.llg_rhs(p, m, H), (m, H), grad_outputs=v)
    m_, H_ = m.detach(), H.detach()
    dot = lambda a, b: (a * b).sum(-1, keepdim=True)  # noqa: E731
    c = -p.gamma / (1 + p.alpha ** 2)
    ref_m = p.alpha * (dot(m_, H_) * v + dot(v, m_) * H_ - 2 * dot(v, H_) * m_)
    ref_H = p.alpha * (dot(v, m_) * m_ - dot(m_, m_) * v)
    if precession:
        ref_m = ref_m + torch.linalg.cross(H_, v, dim=-1)
        ref_H = ref_H + torch.linalg.cross(v, m_, dim=-1)
    assert torch.allclose(gm, c * ref_m, rtol=1e-12, atol=1e-12 * float((c * ref_m).abs().max()))
    assert torch.allclose(gH, c * ref_H, rtol=1e-12, atol=1e-12 * float((c * ref_H).abs().max()))


def test_renormalisation_vector_jacobian_product_closed_form():
    """d(u/|u|)^T v = (v - (n.v) n) / |u| with n = u/|u|."""
    rng = np.random.default_rng(24)
    u = torch.from_numpy(rng.normal(size=(4, 3))).requires_grad_(True)
    v = torch.from_numpy(rng.normal(size=(4, 3)))
    g, = torch.autograd.grad(mm.normalize(u), u, grad_outputs=v)
    r = u.detach().norm(dim=-1, keepdim=True)
    n = u.detach() / r
    assert torch.allclose(g, (v - (n * v).sum(-1, keepdim=True) * n) / r, rtol=1e-12, atol=1e-14)


def test_ms_gradient_formula_against_finite_differences():
    """The per-cell Ms term of the GPU adjoint: for a cotangent g of H_eff,
    d<g, H_eff(m; Ms)>/dMs_j = m_j . (-N * g)_j - (g_j / Ms_j) . H_local,j(m)
    (the demag source is Ms m; exchange, DMI and anisotropy scale as 1/Ms),
    checked by central differences of the oracle's field in each Ms_j."""
    rng = np.random.default_rng(25)
    shape = (2, 4, 3)
    Ms = rng.uniform(6e5, 1e6, size=shape)
    kw = dict(A=1.3e-11, D=1.5e-3, dmi=True, Ku=3e4, ku_axis=(0.2, 0.4, 1.0), h_bias=(1e4, 0.0, 2e4))
    p = mm.Problem(3, 4, 2, 2e-9, 2.5e-9, 3e-9, Ms=Ms, **kw)
    m = mm.normalize(torch.from_numpy(rng.normal(size=shape + (3,))))
    g = torch.from_numpy(rng.normal(size=shape + (3,)))
    t = mm.field_terms(p, m)
    H_local = t["exch"] + t["dmi"] + t["anis"]
    demag_of_g = torch.from_numpy(mm._convolve(p, g.numpy()))
    formula = (m * demag_of_g).sum(-1) - (g / torch.from_numpy(Ms)[..., None] * H_local).sum(-1)
    for j in [(0, 0, 0), (1, 3, 2), (0, 2, 1), (1, 1, 0)]:
        eps = 1e-3 * Ms[j]
        hs = []
        for sgn in (1.0, -1.0):
            Ms2 = Ms.copy()
            Ms2[j] += sgn * eps
            hs.append(float((g * mm.heff(mm.Problem(3, 4, 2, 2e-9, 2.5e-9, 3e-9, Ms=Ms2, **kw), m)).sum()))
        fd = (hs[0] - hs[1]) / (2 * eps)
        assert abs(fd - float(formula[j])) <= 1e-5 * abs(float(formula[j])) + 1e-12, (j, fd, float(formula[j]))
