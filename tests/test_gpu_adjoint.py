"""GPU discrete adjoint (mx_rk_forward_record / mx_rk_backward) vs the FP64
oracle's discrete adjoint and central finite differences.

Tolerance: 1e-3 relative (L2 over the whole gradient field, and per sampled
direction) -- the stated gradient tolerance for the FP32 path.
"""
import numpy as np
import pytest
import torch

from helpers import cfg_of, context, problem, rel_l2, t64
from oracle import adjoint as oadj
from oracle import micromag as mm

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-3


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def dev4(a):
    from paper_2602_12242_gb300.solver import to_dev4
    return to_dev4(a)


def run_case(c, Ms, m0_raw, nsteps, every, patch, dt):
    ctx = context(c, Ms=Ms)
    ctx.adjoint_reserve(nsteps, every)
    mT = ctx.rk_forward_record(dev4(m0_raw), dt)
    lam = torch.zeros_like(mT)
    (y0, y1), (x0, x1) = patch
    lam[:, y0:y1, x0:x1, 2] = 1.0 / ((y1 - y0) * (x1 - x0) * c["nz"])
    g, gms = ctx.rk_backward(lam)
    torch.cuda.synchronize()
    return ctx, mT, g[..., :3].double().cpu().numpy(), gms.double().cpu().numpy()


def test_adjoint_matches_oracle_discrete_adjoint():
    rng = np.random.default_rng(31)
    c = cfg_of(nx=24, ny=20, nz=1, D=2e-3, dmi=True, Ku=0.0, alpha=0.3, h_bias=(0.0, 0.0, 1e5))
    shape = (1, 20, 24)
    Ms = f32(rng.uniform(6e5, 1e6, size=shape))
    m0 = f32(rng.normal(size=shape + (3,)))
    patch = ((6, 14), (8, 16))
    dt, nsteps = 2e-14, 30
    ctx, mT, g, gms = run_case(c, Ms, m0, nsteps, 7, patch, dt)
    p = problem(c, Ms=Ms)
    J, g_ref, gms_ref = oadj.gradient(p, m0, dt, nsteps, lambda m: oadj.patch_mean_mz(m, patch))
    assert rel_l2(g, g_ref.numpy()) <= TOL_GRAD, rel_l2(g, g_ref.numpy())
    assert rel_l2(gms, gms_ref.numpy()) <= TOL_GRAD, rel_l2(gms, gms_ref.numpy())
    # the recorded forward equals the oracle's trajectory
    ref_T = oadj.forward_states(p, m0, dt, nsteps)[-1].numpy()
    assert np.abs(mT[..., :3].double().cpu().numpy() - ref_T).max() <= 1e-4


def test_adjoint_with_demag_off_and_anisotropy():
    rng = np.random.default_rng(32)
    c = cfg_of(nx=16, ny=12, nz=3, Ku=3e4, ku_axis=(0.3, -0.2, 1.0), alpha=0.2, h_bias=(2e4, 0.0, 5e4))
    shape = (3, 12, 16)
    Ms = f32(rng.uniform(6e5, 1e6, size=shape))
    m0 = f32(rng.normal(size=shape + (3,)))
    patch = ((2, 9), (3, 11))
    ctx = context(c, Ms=Ms, demag=False)
    ctx.adjoint_reserve(12, 5)
    mT = ctx.rk_forward_record(dev4(m0), 1e-14)
    lam = torch.zeros_like(mT)
    lam[:, 2:9, 3:11, 2] = 1.0 / (7 * 8 * 3)
    g, gms = ctx.rk_backward(lam)
    p = problem(c, Ms=Ms, demag=False)
    J, g_ref, gms_ref = oadj.gradient(p, m0, 1e-14, 12, lambda m: oadj.patch_mean_mz(m, patch))
    assert rel_l2(g[..., :3].double().cpu().numpy(), g_ref.numpy()) <= TOL_GRAD
    assert rel_l2(gms.double().cpu().numpy(), gms_ref.numpy()) <= TOL_GRAD


def test_adjoint_row_kernels_on_a_3d_grid_with_demag():
    """Demag on a few-row 3D grid (nz = 3, ragged rows): the recompute and the
    reverse sweep run as row kernels (z and y taken from the row index);
    gradients against the oracle's discrete adjoint."""
    rng = np.random.default_rng(35)
    c = cfg_of(nx=18, ny=10, nz=3, D=1e-3, dmi=True, Ku=2e4, ku_axis=(0.1, 0.4, 1.0), alpha=0.25,
               h_bias=(1e4, 0.0, 4e4))
    shape = (3, 10, 18)
    Ms = f32(rng.uniform(6e5, 1e6, size=shape))
    m0 = f32(rng.normal(size=shape + (3,)))
    patch = ((2, 8), (4, 14))
    ctx = context(c, Ms=Ms)
    assert ctx.kernel_name("x_inv_local") == "xr_kernel"
    ctx.adjoint_reserve(9, 4)
    mT = ctx.rk_forward_record(dev4(m0), 1e-14)
    lam = torch.zeros_like(mT)
    lam[:, 2:8, 4:14, 2] = 1.0 / (6 * 10 * 3)
    g, gms = ctx.rk_backward(lam)
    p = problem(c, Ms=Ms)
    J, g_ref, gms_ref = oadj.gradient(p, m0, 1e-14, 9, lambda m: oadj.patch_mean_mz(m, patch))
    assert rel_l2(g[..., :3].double().cpu().numpy(), g_ref.numpy()) <= TOL_GRAD
    assert rel_l2(gms.double().cpu().numpy(), gms_ref.numpy()) <= TOL_GRAD


def test_autograd_function_routes_both_gradients():
    from paper_2602_12242_gb300.autograd import rk4_run
    rng = np.random.default_rng(33)
    c = cfg_of(nx=20, ny=16, nz=1, D=1.5e-3, dmi=True, Ku=0.0, alpha=0.3, h_bias=(0.0, 0.0, 1e5))
    shape = (1, 16, 20)
    Ms = f32(rng.uniform(6e5, 1e6, size=shape))
    m0 = f32(rng.normal(size=shape + (3,)))
    ctx = context(c, Ms=Ms)
    ctx.adjoint_reserve(10, 4)
    m0_t = dev4(m0).requires_grad_(True)
    ms_t = torch.as_tensor(Ms, dtype=torch.float32, device="cuda").requires_grad_(True)
    mT = rk4_run(ctx, m0_t, 2e-14, ms_map=ms_t)
    J = mT[:, 4:12, 5:15, 2].mean()
    J.backward()
    p = problem(c, Ms=Ms)
    Jr, g_ref, gms_ref = oadj.gradient(p, m0, 2e-14, 10, lambda m: oadj.patch_mean_mz(m, ((4, 12), (5, 15))))
    assert abs(float(J.detach()) - Jr) <= 1e-5
    assert rel_l2(m0_t.grad[..., :3].double().cpu().numpy(), g_ref.numpy()) <= TOL_GRAD
    assert rel_l2(ms_t.grad.double().cpu().numpy(), gms_ref.numpy()) <= TOL_GRAD


def test_adjoint_errors():
    from paper_2602_12242_gb300 import MxError, _lib
    c = cfg_of(nx=8, ny=8, nz=1)
    ctx = context(c)
    lam = dev4(np.zeros((1, 8, 8, 3)))
    with pytest.raises(MxError) as ei:
        ctx.rk_backward(lam)
    assert ei.value.status == _lib.MX_ERR_INVALID_ARG
    with pytest.raises(MxError):
        ctx.adjoint_reserve(0, 1)


def _workload(nsteps, every):
    from paper_2602_12242_gb300 import inputs
    c = dict(inputs.CONFIGS["adjoint"])
    Ms, _, _ = inputs.material("adjoint")
    Ms = f32(Ms)
    m0 = f32(inputs.initial_m("adjoint"))
    patch = ((48, 80), (48, 80))  # central 32 x 32 of 128 x 128
    ctx, mT, g, gms = run_case(c, Ms, m0, nsteps, every, patch, c["dt"])
    return c, Ms, m0, patch, g, gms


def _check_against_oracle(c, Ms, m0, patch, g, gms, nsteps, ndirs):
    p = problem(c, Ms=Ms)
    obj = lambda m: oadj.patch_mean_mz(m, patch)  # noqa: E731
    J, g_ref, gms_ref = oadj.gradient(p, m0, c["dt"], nsteps, obj)
    assert rel_l2(g, g_ref.numpy()) <= TOL_GRAD, rel_l2(g, g_ref.numpy())
    assert rel_l2(gms, gms_ref.numpy()) <= TOL_GRAD, rel_l2(gms, gms_ref.numpy())
    # central differences (h = 1e-4) along unit-norm random directions of (m0, Ms/1e6)
    # and along single entries inside the objective's patch
    rng = np.random.default_rng(34)
    dirs = []
    for _ in range(ndirs):
        dm = rng.normal(size=m0.shape)
        ds = rng.normal(size=Ms.shape)
        nrm = np.sqrt((dm ** 2).sum() + (ds ** 2).sum())
        dirs.append((dm / nrm, 1e6 * ds / nrm))
    # a directional derivative can nearly cancel along a random direction, so
    # its error is bounded relative to |g_ref| |d| (Cauchy-Schwarz), the same
    # 1e-3 bar as the relative L2 check above
    # (in the coordinates (m0, Ms / 1e6) of the directions: gradient (g_m, 1e6 g_Ms))
    gnorm = float(np.sqrt((g_ref.numpy() ** 2).sum() + ((1e6 * gms_ref.numpy()) ** 2).sum()))
    for dm, ds in dirs:
        fd = oadj.central_fd(p, m0, c["dt"], nsteps, obj, direction_m=dm, direction_ms=ds, h=1e-4)
        an = float((g * dm).sum() + (0.0 if ds is None else (gms * ds).sum()))
        dnorm = float(np.sqrt((dm ** 2).sum() + ((ds * 1e-6) ** 2).sum()))
        assert abs(an - fd) <= TOL_GRAD * gnorm * dnorm, (an, fd, gnorm, dnorm)
    # single entries of m0 where the derivative is largest (far above the
    # differences' truncation and rounding noise): 1e-3 of the entry itself
    for k in np.argsort(-np.abs(g_ref.numpy()).ravel())[:2]:
        dm = np.zeros(m0.size)
        dm[k] = 1.0
        fd = oadj.central_fd(p, m0, c["dt"], nsteps, obj, direction_m=dm.reshape(m0.shape), h=1e-4)
        an = float(g.ravel()[k])
        assert abs(an - fd) <= TOL_GRAD * abs(fd), (k, an, fd)


def test_adjoint_workload_grid_200_steps():
    """The adjoint workload's grid and material (128x128x1, Ms map in [6e5, 1e6], DMI,
    bias 1e5 A/m along z), 200 RK4 steps with a checkpoint every 20."""
    c, Ms, m0, patch, g, gms = _workload(200, 20)
    _check_against_oracle(c, Ms, m0, patch, g, gms, 200, 1)


def test_adjoint_workload_2000_steps_matches_stored_oracle():
    """The adjoint workload at its stated length: 2000 RK4 steps, a checkpoint
    every 100.  The reference is the FP64 oracle's discrete adjoint and
    central differences of its forward map, computed by
    tests/golden/make_adjoint_2000.py (oracle only; about 20 CPU minutes):
    512 sampled entries and the 16 largest of dJ/dm0, 512 sampled cells of
    dJ/dMs, both full-field norms, and central differences along the two
    largest single entries and one random direction."""
    import json
    import os
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "adjoint_workload_2000.json")))
    c, Ms, m0, patch, g, gms = _workload(ref["nsteps"], 100)
    gi, gv = np.array(ref["g_index"]), np.array(ref["g_value"])
    si, sv = np.array(ref["gms_index"]), np.array(ref["gms_value"])
    assert rel_l2(g.ravel()[gi], gv) <= TOL_GRAD, rel_l2(g.ravel()[gi], gv)
    assert rel_l2(gms.ravel()[si], sv) <= TOL_GRAD, rel_l2(gms.ravel()[si], sv)
    assert abs(np.linalg.norm(g) - ref["g_norm"]) <= TOL_GRAD * ref["g_norm"]
    assert abs(np.linalg.norm(gms) - ref["gms_norm"]) <= TOL_GRAD * ref["gms_norm"]
    top = gi[-16:]
    assert np.all(np.abs(g.ravel()[top] - gv[-16:]) <= TOL_GRAD * np.abs(gv[-16:]))
    gnorm = float(np.sqrt(ref["g_norm"] ** 2 + (1e6 * ref["gms_norm"]) ** 2))
    for e in ref["fd"]:
        if "entry" in e:
            an = float(g.ravel()[e["entry"]])
            assert abs(an - e["fd"]) <= TOL_GRAD * abs(e["fd"]), (e, an)
        else:
            rd = np.random.default_rng(e["random_seed"])
            dm = rd.normal(size=g.shape)
            ds = rd.normal(size=gms.shape)
            nrm = np.sqrt((dm ** 2).sum() + (ds ** 2).sum())
            dm, ds = dm / nrm, 1e6 * ds / nrm  # unit norm in the coordinates (m0, Ms / 1e6)
            an = float((g * dm).sum() + (gms * ds).sum())
            assert abs(an - e["fd"]) <= TOL_GRAD * gnorm, (e, an)


@pytest.mark.slow
def test_adjoint_workload_full_2000_steps():
    """The full adjoint workload against the oracle's discrete adjoint computed
    in the test (every entry) and fresh central differences: 2000 RK4 steps,
    a checkpoint every 100 (about 30 CPU minutes)."""
    c, Ms, m0, patch, g, gms = _workload(2000, 100)
    _check_against_oracle(c, Ms, m0, patch, g, gms, 2000, 2)
