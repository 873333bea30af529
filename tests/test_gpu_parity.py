"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (FP32 path vs FP64 oracle):
  * tensor, real space (both FP64): 1e-10 of the largest entry;
  * tensor spectrum (FP32 store of an FP64 FFT): 1e-6 of the largest entry;
  * fields, dm/dt: relative L2 error <= 1e-5 per evaluation (the stated
    FP32-vs-FP64 tolerance on H_eff), max error <= 1e-4 of the largest value;
  * trajectories: max |m_gpu - m_ref| <= 1e-3.
The oracle is fed the same float32-rounded inputs as the GPU.
"""
import numpy as np
import pytest
import torch

from helpers import cfg_of, context, problem, random_m, rel_l2, rel_max, t64
from oracle import micromag as mm
from oracle import tensor as tn

pytestmark = pytest.mark.gpu

TOL_FIELD = 1e-5

CASES = {
    "cell1": cfg_of(nx=1, ny=1, nz=1),
    "odd3x5x2": cfg_of(nx=3, ny=5, nz=2, dx=2e-9, dy=3e-9, dz=1.5e-9),
    "film17x9": cfg_of(nx=17, ny=9, nz=1, dx=3.9e-9, dy=3.9e-9, dz=3e-9, Ku=0.0, D=1.5e-3, dmi=True,
                       h_bias=(-2.5e4, 4.3e3, 0.0)),
    "plain32x32x4": cfg_of(nx=32, ny=32, nz=4),
    "ragged37x21x5": cfg_of(nx=37, ny=21, nz=5, dx=2.2e-9, dy=1.9e-9, dz=2.5e-9, D=1e-3, dmi=True),
    "line100x3x2": cfg_of(nx=100, ny=3, nz=2),
    "column1x1x9": cfg_of(nx=1, ny=1, nz=9),
    # planes too large for the fused y/z kernel: separate y, z (+multiply), y passes
    "tall64x512x16": cfg_of(nx=64, ny=512, nz=16),
    "mid40x300x3": cfg_of(nx=40, ny=300, nz=3, dx=2.5e-9, dy=2e-9, dz=3e-9, D=1e-3, dmi=True),
    # four-CTA plane kernel: Py/4 = 64, 128, 512 with Pz = 16, 32 (nz < Pz/2), 4
    "quad70x100x6": cfg_of(nx=70, ny=100, nz=6),
    "quad50x200x9": cfg_of(nx=50, ny=200, nz=9, dx=2.5e-9, dy=2e-9, dz=3e-9, D=1e-3, dmi=True),
    "quad33x600x2": cfg_of(nx=33, ny=600, nz=2),
    # Px/2 = 1024: the widest x transforms (32 threads per line)
    "wide600x24x2": cfg_of(nx=600, ny=24, nz=2),
    # one z plane, Py/2 = 64, 256, 512 (single-z-plane y kernel sizes)
    "sheet30x40x1": cfg_of(nx=30, ny=40, nz=1, D=1e-3, dmi=True),
    "sheet40x200x1": cfg_of(nx=40, ny=200, nz=1),
    "sheet24x300x1": cfg_of(nx=24, ny=300, nz=1, dx=3.9e-9, dy=3.9e-9, dz=3e-9),
}
SMALL = [k for k in CASES if k not in ("tall64x512x16", "wide600x24x2", "sheet30x40x1", "sheet40x200x1",
                                       "sheet24x300x1", "quad70x100x6", "quad50x200x9", "quad33x600x2")]


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def gpu_m(a):
    from paper_2602_12242_gb300.solver import to_dev4
    return to_dev4(a)


def host(t):
    from paper_2602_12242_gb300.solver import from_dev4
    return from_dev4(t)


@pytest.mark.parametrize("name", SMALL)
def test_tensor_real_space_matches_oracle(name):
    c = CASES[name]
    ctx = context(c)
    got = ctx.demag_tensor_real().cpu().numpy()
    ref = tn.tensor_octant(c["nx"], c["ny"], c["nz"], c["dx"], c["dy"], c["dz"])
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["plain32x32x4"])
def test_tensor_spectrum_matches_oracle(name):
    """Power-of-two grid: the padded lengths equal the oracle's 2n, so the spectra compare directly."""
    c = CASES[name]
    ctx = context(c)
    Px, Py, Pz = ctx.padded_dims
    assert (Px, Py, Pz) == (2 * c["nx"], 2 * c["ny"], 2 * c["nz"])
    ref = -p_spectrum(problem(c)) / (Px * Py * Pz)
    got = ctx.demag_spectrum().cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()


def p_spectrum(p):
    Nh = mm.padded_tensor_spectrum(p)  # (6, Pz, Py, Px/2+1)
    assert np.abs(Nh.imag).max() <= 1e-12 * np.abs(Nh.real).max()
    Oz, Oy = Nh.shape[1] // 2 + 1, Nh.shape[2] // 2 + 1
    return Nh.real[:, :Oz, :Oy, :]


@pytest.mark.parametrize("name", list(CASES))
def test_demag_field_matches_oracle(name):
    from paper_2602_12242_gb300 import MX_TERM_DEMAG
    c = CASES[name]
    m = f32(random_m(c, 11))
    ctx = context(c)
    h = host(ctx.heff(gpu_m(m), terms=MX_TERM_DEMAG))
    ref = mm.demag_field(problem(c), t64(m)).numpy()
    assert rel_l2(h, ref) <= TOL_FIELD
    assert rel_max(h, ref) <= 1e-4


@pytest.mark.parametrize("name", SMALL)
def test_each_local_term_matches_oracle(name):
    from paper_2602_12242_gb300 import MX_TERM_ANIS, MX_TERM_DMI, MX_TERM_EXCH, MX_TERM_ZEEMAN
    c = CASES[name]
    m = f32(random_m(c, 12))
    ctx = context(c, demag=False)
    p = problem(c, demag=False)
    mt = t64(m)
    terms = {MX_TERM_EXCH: mm.exchange_field(p, mt), MX_TERM_ANIS: mm.anisotropy_field(p, mt),
             MX_TERM_DMI: mm.dmi_field(p, mt), MX_TERM_ZEEMAN: mm.zeeman_field(p, mt)}
    dm = gpu_m(m)
    for bit, ref in terms.items():
        ref = ref.numpy()
        h = host(ctx.heff(dm, terms=bit))
        if np.abs(ref).max() == 0.0:
            assert np.abs(h).max() == 0.0
        else:
            assert rel_l2(h, ref) <= TOL_FIELD, bit
            assert rel_max(h, ref) <= 1e-4, bit


@pytest.mark.parametrize("name", list(CASES))
def test_heff_and_llg_rhs_match_oracle(name):
    c = CASES[name]
    m = f32(random_m(c, 13))
    ctx = context(c)
    p = problem(c)
    dm = gpu_m(m)
    H = host(ctx.heff(dm))
    Href = mm.heff(p, t64(m))
    assert rel_l2(H, Href.numpy()) <= TOL_FIELD
    k = host(ctx.llg_rhs(dm))
    kref = mm.llg_rhs(p, t64(m), Href).numpy()
    assert rel_l2(k, kref) <= TOL_FIELD


def test_material_maps_match_oracle():
    from paper_2602_12242_gb300 import inputs
    c = cfg_of(nx=24, ny=20, nz=3, D=2e-3, dmi=True, Ku=3e4)
    shape = (3, 20, 24)
    Ms = f32(inputs.uniform_map(shape, 6e5, 1e6, 7))
    Ku = f32(inputs.uniform_map(shape, 1e4, 4e5, 8))
    axis = f32(inputs.grain_axes(shape, (8, 8, 2), 9))
    ctx = context(c, Ms=Ms, Ku=Ku, axis=axis)
    p = problem(c, Ms=Ms, Ku=Ku, axis=axis)
    m = f32(random_m(c, 14))
    H = host(ctx.heff(gpu_m(m)))
    assert rel_l2(H, mm.heff(p, t64(m)).numpy()) <= TOL_FIELD
    e = ctx.energy(gpu_m(m))
    eref = mm.energies(p, t64(m))
    scale = sum(abs(v) for v in eref.values())
    for k in eref:
        assert abs(e[k] - eref[k]) <= 1e-5 * scale, k


@pytest.mark.parametrize("name", ["plain32x32x4", "film17x9", "ragged37x21x5", "cell1"])
def test_energies_match_oracle(name):
    c = CASES[name]
    m = f32(random_m(c, 15))
    ctx = context(c)
    e = ctx.energy(gpu_m(m))
    eref = mm.energies(problem(c), t64(m))
    scale = sum(abs(v) for v in eref.values())
    for k in eref:
        assert abs(e[k] - eref[k]) <= 1e-5 * scale, (k, e[k], eref[k])


@pytest.mark.parametrize("method", ["rk4", "euler"])
def test_short_trajectory_matches_oracle(method):
    c = CASES["ragged37x21x5"]
    m0 = f32(random_m(c, 16))
    ctx = context(c)
    m = gpu_m(m0)
    dt = 1e-14
    n = 20
    ctx.rk_step(m, n, dt, method)
    ctx.sync()
    p = problem(c)
    ref = mm.run(p, t64(m0), dt, n, method).numpy()
    got = host(m)
    assert np.abs(got - ref).max() <= 1e-4
    assert np.abs(np.linalg.norm(got, axis=-1) - 1).max() <= 1e-6


@pytest.mark.parametrize("method", ["rk4", "euler"])
def test_relaxation_without_precession_matches_oracle(method):
    """The precession switch (damping term only, for relaxation to a state):
    dm/dt and a short run against the oracle with the same switch, DMI and
    chiral edges included."""
    c = CASES["ragged37x21x5"]
    m0 = f32(random_m(c, 17))
    ctx = context(c, precession=False)
    p = problem(c, precession=False)
    k = host(ctx.llg_rhs(gpu_m(m0)))
    kref = mm.llg_rhs(p, t64(m0), mm.heff(p, t64(m0))).numpy()
    assert rel_l2(k, kref) <= TOL_FIELD
    m = gpu_m(m0)
    ctx.rk_step(m, 20, 1e-14, method)
    ctx.sync()
    ref = mm.run(p, t64(m0), 1e-14, 20, method).numpy()
    assert np.abs(host(m) - ref).max() <= 1e-4


def test_plain_workload_200_rk4_steps_matches_oracle():
    """The plain workload: 32x32x4, random m, RK4 dt = 1e-14 s, 200 steps."""
    from paper_2602_12242_gb300 import inputs
    c = dict(inputs.CONFIGS["plain"])
    m0 = f32(inputs.initial_m("plain"))
    ctx = context(c)
    m = gpu_m(m0)
    ctx.rk_step(m, c["steps"], c["dt"])
    ctx.sync()
    ref = mm.run(problem(c), t64(m0), c["dt"], c["steps"]).numpy()
    err = np.abs(host(m) - ref).max()
    assert err <= 1e-3, err


def test_graph_replay_equals_direct_launches():
    """mx_rk_step (graph) and mx_profile_step (direct launches) give the same bits."""
    c = CASES["plain32x32x4"]
    m0 = f32(random_m(c, 17))
    ctx = context(c)
    a, b = gpu_m(m0), gpu_m(m0)
    ctx.rk_step(a, 5, 1e-14)
    ctx.profile_step(b, 5, 1e-14)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_errors_are_reported():
    from paper_2602_12242_gb300 import MX_TERM_ALL, MxError, _lib
    from paper_2602_12242_gb300.solver import Context
    c = CASES["odd3x5x2"]
    ctx = Context(c["nx"], c["ny"], c["nz"], c["dx"], c["dy"], c["dz"], build=False)
    m = gpu_m(f32(random_m(c, 18)))
    with pytest.raises(MxError) as ei:
        ctx.heff(m, terms=MX_TERM_ALL)
    assert ei.value.status == _lib.MX_ERR_NOT_BUILT
    ctx.build_demag_kernel()
    bad = m.clone()
    bad[0, 0, 0, 0] = float("nan")
    ctx.llg_rhs(bad)
    with pytest.raises(MxError) as ei:
        ctx.sync()
    assert ei.value.status == _lib.MX_ERR_NONFINITE
    ctx.sync()  # the flag was cleared
    with pytest.raises(MxError) as ei:
        ctx.rk_step(m, 1, -1.0)
    assert ei.value.status == _lib.MX_ERR_INVALID_ARG
    with pytest.raises(MxError) as ei:
        Context(5000, 4, 4, 1e-9, 1e-9, 1e-9, build=False)
    assert ei.value.status == _lib.MX_ERR_UNSUPPORTED


def test_film_workload_full_size_matches_oracle():
    """The thin-film workload at full size (512x128x1, DMI, chiral boundary), every cell."""
    from paper_2602_12242_gb300 import inputs
    c = dict(inputs.CONFIGS["film"])
    m = f32(inputs.initial_m("film"))
    ctx = context(c)
    p = problem(c)
    dm = gpu_m(m)
    H = host(ctx.heff(dm))
    Href = mm.heff(p, t64(m))
    assert rel_l2(H, Href.numpy()) <= TOL_FIELD
    k = host(ctx.llg_rhs(dm))
    assert rel_l2(k, mm.llg_rhs(p, t64(m), Href).numpy()) <= TOL_FIELD
    # one RK4 step of the workload
    ctx.rk_step(dm, 1, c["dt"])
    ctx.sync()
    ref = mm.rk4_step(p, t64(m), c["dt"]).numpy()
    assert np.abs(host(dm) - ref).max() <= 1e-5


def test_bulk_workload_full_size_sampled_direct_sum():
    """The bulk workload at full size (512x512x16, grains): demag field at sampled cells
    against the oracle's direct real-space sum over all 4.2M sources, local fields on
    sampled cells, and |m| = 1 after a step."""
    from paper_2602_12242_gb300 import inputs
    from paper_2602_12242_gb300 import MX_TERM_DEMAG
    c = dict(inputs.CONFIGS["bulk"])
    m = f32(inputs.initial_m("bulk"))
    Ms, Ku, axis = inputs.material("bulk")
    axis = f32(axis)
    ctx = context(c, Ms=Ms, Ku=Ku, axis=axis)
    p = problem(c, Ms=Ms, Ku=Ku, axis=axis)
    dm = gpu_m(m)
    Hd = host(ctx.heff(dm, terms=MX_TERM_DEMAG))
    targets = [(0, 0, 0), (15, 511, 511), (7, 256, 3), (8, 100, 400), (3, 511, 0), (12, 37, 290)]
    ref = mm.demag_field_at(p, t64(m), targets)
    got = np.array([Hd[t] for t in targets])
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-5 * scale, np.abs(got - ref).max() / scale
    # local terms on a sub-block (exchange + anisotropy + Zeeman), compared in the interior
    H = host(ctx.heff(dm)) - Hd
    sub = (slice(0, 16), slice(200, 232), slice(300, 340))
    pl = problem(dict(c, nx=40, ny=32, nz=16), Ms=Ms, Ku=Ku, axis=axis[sub], demag=False)
    Hl = mm.heff_local(pl, t64(m[sub])).numpy()
    assert rel_l2(H[sub][:, 1:-1, 1:-1], Hl[:, 1:-1, 1:-1]) <= TOL_FIELD
    ctx.rk_step(dm, 2, c["dt"])
    ctx.sync()
    nrm = np.linalg.norm(host(dm), axis=-1)
    assert np.abs(nrm - 1).max() <= 1e-6


@pytest.mark.parametrize("name", ["tall64x512x16", "mid40x300x3", "wide600x24x2", "ragged37x21x5", "film17x9", "cell1",
                                  "sheet30x40x1", "sheet40x200x1", "sheet24x300x1", "quad70x100x6", "quad50x200x9",
                                  "quad33x600x2"])
@pytest.mark.parametrize("path", ["generic", "plane", "plane_pair", "auto"])
def test_each_demag_schedule_matches_oracle(name, path):
    """Every schedule of the convolution (size-generic passes, per-kx plane path
    with the four-CTA or the two-CTA y/z kernel) gives the oracle's field;
    grids the plane path cannot take are refused."""
    from paper_2602_12242_gb300 import MX_TERM_DEMAG, MxError, _lib
    c = CASES[name]
    code = {"generic": _lib.MX_DEMAG_GENERIC, "plane": _lib.MX_DEMAG_PLANE, "plane_pair": _lib.MX_DEMAG_PLANE_PAIR,
            "auto": _lib.MX_DEMAG_AUTO}[path]
    try:
        ctx = context(c, demag_path=code)
    except MxError as e:
        assert path in ("plane", "plane_pair") and e.status == _lib.MX_ERR_UNSUPPORTED
        assert name in ("cell1", "film17x9") or c["nz"] == 1  # Py/2 < 16 or Pz < 4
        return
    # Py/4 >= 64 and Pz >= 4 take the four-CTA kernel unless the two-CTA one is forced
    Px, Py, Pz = ctx.padded_dims
    if path == "plane":
        assert ctx.kernel_name("yz_fused") == ("yzq_kernel" if Py >= 256 else "yzh_kernel")
    if path == "plane_pair":
        assert ctx.kernel_name("yz_fused") == "yzh_kernel"
    m = f32(random_m(c, 19))
    h = host(ctx.heff(gpu_m(m), terms=MX_TERM_DEMAG))
    ref = mm.demag_field(problem(c), t64(m)).numpy()
    assert rel_l2(h, ref) <= TOL_FIELD
    assert rel_max(h, ref) <= 1e-4


@pytest.mark.parametrize("name", ["ragged37x21x5", "mid40x300x3", "quad70x100x6", "quad50x200x9", "wide600x24x2"])
@pytest.mark.parametrize("method", ["rk4", "euler"])
def test_fused_inverse_x_local_stage_matches_oracle(name, method):
    """MX_DEMAG_PLANE_XLOCAL (the inverse x pass and the local stage in one
    kernel, H_demag kept in shared memory): short trajectories against the
    oracle and against the same steps with the separate passes, ragged rows
    (ny mod 8 != 0), odd nx and DMI with chiral edges included."""
    from paper_2602_12242_gb300 import _lib
    c = CASES[name]
    m0 = f32(random_m(c, 23))
    ctx = context(c, demag_path=_lib.MX_DEMAG_PLANE_XLOCAL)
    assert ctx.kernel_name("x_inv_local") == "xil_kernel"
    dt, n = 1e-14, 4
    m = gpu_m(m0)
    ctx.rk_step(m, n, dt, method)
    ctx.sync()
    got = host(m)
    ref = mm.run(problem(c), t64(m0), dt, n, method).numpy()
    assert np.abs(got - ref).max() <= 1e-4
    assert np.abs(np.linalg.norm(got, axis=-1) - 1).max() <= 1e-6
    sep = context(c, demag_path=_lib.MX_DEMAG_PLANE)
    assert sep.kernel_name("x_inv_local") == ""
    m2 = gpu_m(m0)
    sep.rk_step(m2, n, dt, method)
    sep.sync()
    assert np.abs(got - host(m2)).max() <= 1e-6


def test_fused_inverse_x_local_stage_bulk_workload():
    """The bulk workload at full size (512x512x16, grains): RK4 steps with the
    fused inverse x + local kernel equal the separate passes to FP32 rounding,
    the fused kernel is the one that runs, and |m| = 1 afterwards."""
    from paper_2602_12242_gb300 import _lib, inputs
    c = dict(inputs.CONFIGS["bulk"])
    m0 = f32(inputs.initial_m("bulk"))
    Ms, Ku, axis = inputs.material("bulk")
    out = []
    for path in (_lib.MX_DEMAG_PLANE_XLOCAL, _lib.MX_DEMAG_PLANE):
        ctx = context(c, Ms=Ms, Ku=Ku, axis=f32(axis), demag_path=path)
        m = gpu_m(m0)
        prof = ctx.profile_step(m, 2, c["dt"])
        if path == _lib.MX_DEMAG_PLANE_XLOCAL:
            assert prof["x_inv_local"][1] == 8 and "x_inv" not in prof and "local_stage" not in prof
        ctx.sync()
        out.append(host(m))
        del ctx
    assert np.abs(out[0] - out[1]).max() <= 1e-6
    assert np.abs(np.linalg.norm(out[0], axis=-1) - 1).max() <= 1e-6


@pytest.mark.parametrize("name", ["film17x9", "ragged37x21x5", "sheet30x40x1", "sheet24x300x1",
                                  "line100x3x2", "wide600x24x2"])
def test_row_kernel_rk4_matches_oracle(name):
    """Few-row grids run each RK4 stage as the y/z passes plus one row kernel
    (inverse x, local stage, the next stage's forward x): short trajectories
    against the oracle and against the size-generic separate passes."""
    from paper_2602_12242_gb300 import _lib
    c = CASES[name]
    m0 = f32(random_m(c, 29))
    ctx = context(c)
    assert ctx.kernel_name("x_inv_local") == "xr_kernel"
    dt, n = 1e-14, 5
    m = gpu_m(m0)
    prof = ctx.profile_step(m, n, dt)
    assert prof["x_inv_local"][1] == 4 * n and prof["x_fwd"][1] == 1 and "local_stage" not in prof
    ctx.sync()
    got = host(m)
    ref = mm.run(problem(c), t64(m0), dt, n, "rk4").numpy()
    assert np.abs(got - ref).max() <= 1e-4
    assert np.abs(np.linalg.norm(got, axis=-1) - 1).max() <= 1e-6
    gen = context(c, demag_path=_lib.MX_DEMAG_GENERIC)
    assert gen.kernel_name("x_inv_local") == ""
    m2 = gpu_m(m0)
    gen.rk_step(m2, n, dt)
    gen.sync()
    assert np.abs(got - host(m2)).max() <= 1e-6
