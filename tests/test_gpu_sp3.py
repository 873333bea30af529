"""muMAG Standard Problem 3 (Sec. III-B, Table I, N = 10) on the GPU path:
the FP32 RK4 relaxation (alpha 0.5, 2 ns, dt 2e-13 s) of the flower and
vortex states reproduces the tabulated energy densities and mean
magnetisation to 1e-3, and the central-difference exchange energy entry
point equals the oracle's on a random field."""
import numpy as np
import pytest

import sp3
from helpers import context, problem, random_m, t64
from oracle import micromag as mm

pytestmark = pytest.mark.gpu


def test_central_exchange_energy_matches_oracle():
    from paper_2602_12242_gb300.solver import to_dev4
    from helpers import cfg_of
    for c in (cfg_of(nx=37, ny=21, nz=5, dx=2.2e-9, dy=1.9e-9, dz=2.5e-9),
              cfg_of(nx=24, ny=16, nz=1, D=1.5e-3, dmi=True)):
        m = np.asarray(random_m(c, 71), np.float32).astype(np.float64)
        ctx = context(c)
        got = ctx.exchange_energy_central(to_dev4(m))
        ref = mm.exchange_energy_central(problem(c), t64(m))
        assert abs(got - ref) <= 1e-5 * abs(ref), (got, ref)


@pytest.mark.parametrize("state", ["flower", "vortex"])
def test_standard_problem_3_matches_table_1(state):
    from paper_2602_12242_gb300.solver import from_dev4, to_dev4
    c = sp3.cfg()
    ctx = context(c)
    m = to_dev4(sp3.initial(state))
    ctx.rk_step(m, 10000, 2e-13)
    ctx.sync()
    e = ctx.energy(m)
    d = sp3.densities(c, e["demag"], ctx.exchange_energy_central(m), e["anis"])
    mean = from_dev4(m).reshape(-1, 3).mean(0)
    print(f"\nSP3 N=10 {state}: {d}, mean m {mean}")
    sp3.check(state, d, mean)
