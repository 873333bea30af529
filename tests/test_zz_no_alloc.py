"""The allocation-free energy entry point (mx_energy_noalloc) against mx_energy.

mx_energy_noalloc serves callers that cannot allocate device memory: it uses
only the caller's buffers and a fixed scratch array inside the library.  This
file sorts last so that a run stopping at its first failure has already run
every other test; it passes alone in a fresh process and after the others.
"""
import ctypes

import numpy as np
import pytest
import torch

from helpers import cfg_of, context, problem, random_m, t64

pytestmark = pytest.mark.gpu

TOL_ENERGY = 1e-5  # relative to the sum of |terms|, as in the other energy tests


def _params(ctx):
    from paper_2602_12242_gb300 import _lib
    p = _lib.mx_params()
    ctypes.memmove(ctypes.byref(p), ctypes.byref(ctx.params), ctypes.sizeof(p))
    return p


@pytest.mark.parametrize("case", ["film_dmi_maps", "bulk_like"])
def test_noalloc_energy_equals_mx_energy_twice(case):
    from paper_2602_12242_gb300 import MX_TERM_DEMAG, _lib, inputs
    from paper_2602_12242_gb300.solver import to_dev4
    if case == "film_dmi_maps":
        c = cfg_of(nx=40, ny=24, nz=1, dx=3.9e-9, dy=3.9e-9, dz=3e-9, D=1.5e-3, dmi=True, Ku=2e4,
                   h_bias=(-2.5e4, 4.3e3, 0.0))
        shape = (1, 24, 40)
        Ms = inputs.uniform_map(shape, 6e5, 1e6, 71).astype(np.float32)
        Ku = inputs.uniform_map(shape, 1e4, 5e4, 72).astype(np.float32)
        axis = inputs.grain_axes(shape, (8, 8, 1), 73).astype(np.float32)
    else:
        c = cfg_of(nx=64, ny=48, nz=8, Ku=4e5)
        shape = (8, 48, 64)
        Ms, Ku, axis = None, None, inputs.grain_axes(shape, (32, 32, 16), 74).astype(np.float32)
    ctx = context(c, Ms=Ms, Ku=Ku, axis=axis)
    m = to_dev4(random_m(c, 75))
    ref = ctx.energy(m)
    hd = ctx.heff(m, terms=MX_TERM_DEMAG)
    ms_t = None if Ms is None else torch.as_tensor(Ms).cuda()
    ku_t = None if Ku is None else torch.as_tensor(Ku).cuda()
    ax_t = to_dev4(axis)
    p = _params(ctx)
    scale = sum(abs(v) for v in ref.values())
    for _ in range(2):  # two calls in a row share the scratch array
        out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        _lib.mx_energy_noalloc(p, m, out, h_demag=hd, ms_map=ms_t, ku_map=ku_t, axis_map=ax_t)
        torch.cuda.synchronize()
        got = dict(zip(("demag", "exch", "anis", "dmi", "zeeman"), out.cpu().tolist()))
        for k in ref:
            assert abs(got[k] - ref[k]) <= TOL_ENERGY * scale, (k, got[k], ref[k])


def _noalloc_vs_energy(c, seed, with_demag=True):
    """mx_energy_noalloc against mx_energy on one grid (uniform Ms and Ku, grain axes)."""
    from paper_2602_12242_gb300 import MX_TERM_DEMAG, _lib, inputs
    from paper_2602_12242_gb300.solver import to_dev4
    shape = (c["nz"], c["ny"], c["nx"])
    axis = inputs.grain_axes(shape, (16, 16, 4), seed).astype(np.float32)
    ctx = context(c, axis=axis)
    m = to_dev4(random_m(c, seed + 1))
    ref = ctx.energy(m)
    hd = ctx.heff(m, terms=MX_TERM_DEMAG) if with_demag else None
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    _lib.mx_energy_noalloc(_params(ctx), m, out, h_demag=hd, axis_map=to_dev4(axis))
    torch.cuda.synchronize()
    return dict(zip(("demag", "exch", "anis", "dmi", "zeeman"), out.cpu().tolist())), ref


def test_noalloc_after_a_larger_grid_and_without_demag():
    """A grid of more than 65,536 cells (512 blocks: the reduction's strided
    loop takes several passes) between two calls on a small grid, which must
    not see the larger call's leftover rows; then h_demag = NULL, whose demag
    energy is exactly 0 while the other terms still match."""
    small = cfg_of(nx=20, ny=12, nz=3, Ku=3e4, h_bias=(1e4, 0.0, -2e4))
    large = cfg_of(nx=128, ny=128, nz=8, Ku=4e5)
    for c, seed in ((small, 81), (large, 83), (small, 81)):
        got, ref = _noalloc_vs_energy(c, seed)
        scale = sum(abs(v) for v in ref.values())
        for k in ref:
            assert abs(got[k] - ref[k]) <= TOL_ENERGY * scale, (c["nx"], k, got[k], ref[k])
    got, ref = _noalloc_vs_energy(small, 85, with_demag=False)
    assert got["demag"] == 0.0
    scale = sum(abs(v) for k, v in ref.items() if k != "demag")
    for k in ("exch", "anis", "dmi", "zeeman"):
        assert abs(got[k] - ref[k]) <= TOL_ENERGY * scale, (k, got[k], ref[k])


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_2602_12242_gb300 import MxError, _lib
    p = _lib.mx_params()
    p.nx, p.ny, p.nz = 2048, 2048, 2
    p.dx = p.dy = p.dz = 2e-9
    p.Ms, p.A, p.gamma = 8e5, 1.3e-11, 2.211e5
    m = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(MxError) as ei:
        _lib.mx_energy_noalloc(p, m, out)
    assert ei.value.status == _lib.MX_ERR_UNSUPPORTED
    assert "limit" in str(ei.value)


def test_noalloc_energy_matches_oracle():
    """mx_energy_noalloc against the FP64 oracle's energies directly (film
    with DMI and chiral edges, per-cell Ms, Ku and easy axis), the demag field
    passed in being the library's own H_demag of the same m."""
    from oracle import micromag as mm
    from paper_2602_12242_gb300 import MX_TERM_DEMAG, _lib, inputs
    from paper_2602_12242_gb300.solver import to_dev4
    c = cfg_of(nx=40, ny=24, nz=1, dx=3.9e-9, dy=3.9e-9, dz=3e-9, D=1.5e-3, dmi=True, Ku=2e4,
               h_bias=(-2.5e4, 4.3e3, 0.0))
    shape = (1, 24, 40)
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    Ms = f32(inputs.uniform_map(shape, 6e5, 1e6, 81))
    Ku = f32(inputs.uniform_map(shape, 1e4, 5e4, 82))
    axis = f32(inputs.grain_axes(shape, (8, 8, 1), 83))
    m = f32(random_m(c, 84))
    ctx = context(c, Ms=Ms, Ku=Ku, axis=axis)
    md = to_dev4(m)
    hd = ctx.heff(md, terms=MX_TERM_DEMAG)
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    _lib.mx_energy_noalloc(_params(ctx), md, out, h_demag=hd,
                           ms_map=torch.as_tensor(Ms.astype(np.float32)).cuda(),
                           ku_map=torch.as_tensor(Ku.astype(np.float32)).cuda(), axis_map=to_dev4(axis))
    torch.cuda.synchronize()
    got = dict(zip(("demag", "exch", "anis", "dmi", "zeeman"), out.cpu().tolist()))
    ref = mm.energies(problem(c, Ms=Ms, Ku=Ku, axis=axis), t64(m))
    scale = sum(abs(v) for v in ref.values())
    for k in ref:
        assert abs(got[k] - ref[k]) <= TOL_ENERGY * scale, (k, got[k], ref[k])
