"""Explicit-explicit MRI step (Sec. II-C, III-C) on the GPU against the FP64
oracle's MRI step (oracle/mri.py): same fast/slow split, Knoth-Wolke on both
levels, fast step 0.1 of the slow step.  Tolerance as for the RK4 paths:
1e-5 on m after a few steps."""
import numpy as np
import pytest
import torch

from helpers import cfg_of, context, problem, random_m, t64
from oracle import mri as omri

pytestmark = pytest.mark.gpu


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


CASES = {
    "plain32x32x4": (cfg_of(nx=32, ny=32, nz=4), 5e-14, 4),
    "ragged37x21x5_dmi": (cfg_of(nx=37, ny=21, nz=5, dx=2.2e-9, dy=1.9e-9, dz=2.5e-9, D=1e-3, dmi=True), 5e-14, 4),
    "film40x24x1_dmi": (cfg_of(nx=40, ny=24, nz=1, dx=3.9e-9, dy=3.9e-9, dz=3e-9, Ku=0.0, D=1.5e-3, dmi=True,
                               h_bias=(-2.5e4, 4.3e3, 0.0), alpha=0.02), 2.5e-13, 4),
}


@pytest.mark.parametrize("name", list(CASES))
def test_mri_matches_oracle(name):
    from paper_2602_12242_gb300.solver import from_dev4, to_dev4
    c, dt, n = CASES[name]
    m0 = f32(random_m(c, 81)) if "film" not in name else f32(np.broadcast_to(
        np.array([1.0, 0.25, 0.1]) / np.linalg.norm([1.0, 0.25, 0.1]), (1, 24, 40, 3)).copy())
    ctx = context(c)
    m = to_dev4(m0)
    ctx.rk_step(m, n, dt, "mri")
    ctx.sync()
    ref = omri.run(problem(c), t64(m0), dt, n).numpy()
    got = from_dev4(m)
    assert np.abs(got - ref).max() <= 1e-5, np.abs(got - ref).max()
    assert np.abs(np.linalg.norm(got, axis=-1) - 1).max() <= 1e-6


def test_mri_fast_ratio_option_and_counts():
    """A coarser fast step (ratio 0.25: 2 + 2 + 1 fast steps) matches the oracle
    with the same ratio; one MRI step runs three demag convolutions."""
    from paper_2602_12242_gb300.solver import from_dev4, to_dev4
    c = cfg_of(nx=32, ny=32, nz=4)
    m0 = f32(random_m(c, 82))
    ctx = context(c, mri_fast_ratio=0.25)
    m = to_dev4(m0)
    ctx.rk_step(m, 2, 3e-14, "mri")
    ctx.sync()
    ref = omri.run(problem(c), t64(m0), 3e-14, 2, ratio=0.25).numpy()
    assert np.abs(from_dev4(m) - ref).max() <= 1e-5
    prof = ctx.profile_step(to_dev4(m0), 3, 3e-14, "mri")
    assert prof["mri_slow"][1] == 9 and prof["x_fwd"][1] == 9 and "local_stage" not in prof


def test_mri_graph_replay_equals_direct_launches():
    from paper_2602_12242_gb300.solver import to_dev4
    c = cfg_of(nx=32, ny=32, nz=4)
    m0 = f32(random_m(c, 83))
    ctx = context(c)
    a, b = to_dev4(m0), to_dev4(m0)
    ctx.rk_step(a, 3, 5e-14, "mri")
    ctx.profile_step(b, 3, 5e-14, "mri")
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_bad_fast_ratio_is_refused():
    from paper_2602_12242_gb300 import MxError, _lib
    with pytest.raises(MxError) as ei:
        context(cfg_of(nx=8, ny=8, nz=1), mri_fast_ratio=2.0)
    assert ei.value.status == _lib.MX_ERR_INVALID_ARG
