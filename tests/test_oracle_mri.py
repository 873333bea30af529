"""Pins for the oracle's explicit-explicit MRI step (Sec. II-C, III-C): the
Knoth-Wolke tableau's third-order conditions, reduction to the single-rate
method when the fast part vanishes, the fast-step count, and third-order
convergence of the coupled method against a fine RK4 reference."""
import numpy as np
import torch

from oracle import micromag as mm
from oracle import mri


def test_knoth_wolke_tableau_is_third_order():
    A, b, c = np.array(mri.KW3_A), np.array(mri.KW3_B), np.array(mri.KW3_C)
    assert np.allclose(A.sum(1), c, atol=1e-15)
    assert abs(b.sum() - 1) < 1e-15
    assert abs(b @ c - 1 / 2) < 1e-15
    assert abs(b @ c ** 2 - 1 / 3) < 1e-15
    assert abs(b @ A @ c - 1 / 6) < 1e-15


def test_knoth_wolke_step_converges_at_third_order_on_a_rotation():
    """v' = w x v (exact solution: rotation), no renormalisation."""
    w = torch.tensor([0.3, -0.2, 1.1], dtype=torch.float64)
    v0 = torch.tensor([1.0, 0.2, -0.4], dtype=torch.float64)
    T = 2.0
    th = float(w.norm()) * T
    k = w / w.norm()
    exact = v0 * np.cos(th) + torch.linalg.cross(k, v0) * np.sin(th) + k * (k @ v0) * (1 - np.cos(th))
    errs = []
    for n in (16, 32, 64):
        v = v0.clone()
        for _ in range(n):
            v = mri.kw3_step(lambda x: torch.linalg.cross(w, x), v, T / n, renorm=False)
        errs.append(float((v - exact).abs().max()))
    assert 7.0 < errs[0] / errs[1] < 9.0 and 7.0 < errs[1] / errs[2] < 9.0, errs


def test_fast_step_counts():
    """Stage intervals 1/3, 5/12, 1/4 of the slow step at a 0.1 fast ratio."""
    c = mri.KW3_C + (1.0,)
    assert [mri.fast_steps(c[i] - c[i - 1], 0.1) for i in (1, 2, 3)] == [4, 5, 3]


def _problem(A=1.3e-11):
    return mm.Problem(6, 5, 2, 2e-9, 2e-9, 2e-9, Ms=8e5, A=A, Ku=5e4, ku_axis=(0.2, 0.1, 1.0), alpha=0.3,
                      h_bias=(1e4, 0.0, 3e4))


def _m0():
    rng = np.random.default_rng(3)
    return mm.normalize(torch.from_numpy(rng.normal(size=(2, 5, 6, 3)) * 0.3 + np.array([0.0, 0.0, 1.0])))


def test_without_fast_part_it_is_the_single_rate_method():
    """A = 0: the inner problems integrate a constant forcing exactly, so the
    step is one Knoth-Wolke step of the slow right-hand side."""
    p = _problem(A=0.0)
    m = _m0()
    h = 5e-13
    got = mri.mri_step(p, m, h, renorm=False)
    ref = mri.kw3_step(lambda x: mri.slow_rhs(p, x), m, h, renorm=False)
    assert float((got - ref).abs().max()) <= 1e-13


def test_split_adds_up_to_the_full_right_hand_side():
    p = _problem()
    m = _m0()
    assert float((mri.fast_rhs(p, m) + mri.slow_rhs(p, m) - mm.rhs(p, m)).abs().max()) <= 1e-6 * float(
        mm.rhs(p, m).abs().max())


def test_coupled_method_converges_at_third_order():
    p = _problem()
    m0 = _m0()
    T = 2e-12
    ref = mm.run(p, m0, T / 2000, 2000)
    errs = []
    for n in (4, 8, 16):
        m = m0.clone()
        for _ in range(n):
            m = mri.mri_step(p, m, T / n)
        errs.append(float((m - ref).abs().max()))
    assert 6.0 < errs[0] / errs[1] < 11.0 and 6.0 < errs[1] / errs[2] < 11.0, errs


def test_evaluation_counts_against_table_2():
    """Table II (Sec. III-C): RK4 evaluates the full right-hand side (demag and
    exchange) 4 times per step; the MRI step evaluates demag 3 times, and
    over the 1.25e-13 s interval RK4 needs 5 steps against MRI's 1.  Exchange
    per MRI step: 12 fast Knoth-Wolke steps x 3 stages = 36 here; the table
    prints 37 (the reading of the fast step count is the one difference)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table2_eval_counts.json")))
    p = _problem()
    m = _m0()
    calls = {"fast": 0, "slow": 0, "full": 0}

    def counted(name, f):
        def g_(x):
            calls[name] += 1
            return f(x)
        return g_

    mri.mri_step(p, m, 1e-13, fast=counted("fast", lambda x: mri.fast_rhs(p, x)),
                 slow=counted("slow", lambda x: mri.slow_rhs(p, x)))
    assert calls["slow"] == g["mri"]["demag_per_step"] == 3
    assert calls["fast"] == 36 == g["mri"]["exchange_per_step"] - 1
    mm.rk4_step(p, m, 1e-14, f=counted("full", lambda x: mm.rhs(p, x)))
    assert calls["full"] == g["rk4"]["demag_per_step"] == g["rk4"]["exchange_per_step"]
    steps = {k: round(g["interval_s"] / g[k]["max_dt_s"]) for k in ("rk4", "mri")}
    assert steps == {"rk4": g["rk4"]["steps"], "mri": g["mri"]["steps"]}
    assert steps["rk4"] * calls["full"] == g["rk4"]["total_demag"]
    assert steps["mri"] * calls["slow"] == g["mri"]["total_demag"]
