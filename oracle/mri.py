"""Oracle: explicit-explicit multirate infinitesimal (MRI) time step.

TEST INFRASTRUCTURE ONLY (plain FP64 CPU; the product never imports it).

Partition (Sec. III-C): the fast part of the LLG right-hand side is the one
driven by the exchange field, the slow part the one driven by every other
term (demag, anisotropy, DMI, Zeeman); the LLG right-hand side is linear in H,
so the two parts add up to Eq. 1.  Both levels use the three-stage,
third-order explicit Runge-Kutta method of Knoth and Wolke (1998),
    A = [[0, 0, 0], [1/3, 0, 0], [-3/16, 15/16, 0]], b = [1/6, 3/10, 8/15],
    c = [0, 1/3, 3/4],
with a fast step of 0.1 of the slow step (Sec. III-C).

Coupling (the multirate infinitesimal step of Knoth and Wolke, in the form
of Wensch, Knoth and Galant 2009, the explicit MRI scheme of Sec. II-C):
with c_4 = 1 and row 4 of A equal to b, the slow stages are Y_1 = y_n and,
for i = 2, 3, 4, the solution at the end of an interval of length
(c_i - c_{i-1}) h of
    v' = f_fast(v) + r_i,   v(0) = Y_{i-1},
    r_i = sum_{j<i} (a_ij - a_{i-1,j}) f_slow(Y_j) / (c_i - c_{i-1}),
so y_{n+1} = Y_4 and one step costs three slow evaluations.  The inner
problem is integrated with ceil((c_i - c_{i-1}) / ratio) equal Knoth-Wolke
steps (ratio = 0.1: 4 + 5 + 3 = 12 fast steps, 36 fast evaluations).
With ``renorm`` every fast stage input and every fast step result is
renormalised (Sec. II-B: after each step or stage evaluation).
"""
import math

import torch

from . import micromag as mm

KW3_A = ((0.0, 0.0, 0.0), (1.0 / 3.0, 0.0, 0.0), (-3.0 / 16.0, 15.0 / 16.0, 0.0))
KW3_B = (1.0 / 6.0, 3.0 / 10.0, 8.0 / 15.0)
KW3_C = (0.0, 1.0 / 3.0, 3.0 / 4.0)


def fast_rhs(p, m):
    """LLG right-hand side of the exchange field alone."""
    return mm.llg_rhs(p, m, mm.exchange_field(p, m))


def slow_rhs(p, m):
    """LLG right-hand side of demag + anisotropy + DMI + Zeeman."""
    t = mm.field_terms(p, m)
    return mm.llg_rhs(p, m, t["demag"] + t["anis"] + t["dmi"] + t["zeeman"])


def kw3_step(f, v, h, renorm=True):
    """One Knoth-Wolke step of v' = f(v)."""
    nrm = mm.normalize if renorm else (lambda x: x)
    k = []
    for i in range(3):
        u = v + h * sum(KW3_A[i][j] * k[j] for j in range(i)) if i else v
        k.append(f(nrm(u) if i else u))
    return nrm(v + h * sum(KW3_B[j] * k[j] for j in range(3)))


def fast_steps(interval, ratio):
    """Number of equal fast steps for a stage interval (in units of h)."""
    return max(1, math.ceil(interval / ratio - 1e-9))


def mri_step(p, m, h, ratio=0.1, renorm=True, fast=None, slow=None):
    """One explicit-explicit MRI step of length h."""
    fast = fast or (lambda x: fast_rhs(p, x))
    slow = slow or (lambda x: slow_rhs(p, x))
    a = KW3_A + (KW3_B,)
    c = KW3_C + (1.0,)
    Y = [m]
    F = []
    for i in range(1, 4):
        F.append(slow(Y[i - 1]))
        dc = c[i] - c[i - 1]
        r = sum((a[i][j] - a[i - 1][j]) * F[j] for j in range(i)) / dc
        n = fast_steps(dc, ratio)
        v = Y[i - 1]
        for _ in range(n):
            v = kw3_step(lambda x: fast(x) + r, v, dc * h / n, renorm)
        Y.append(v)
    return Y[3]


def run(p, m, h, nsteps, ratio=0.1, renorm=True):
    m = mm.normalize(mm.as_t(m)) if renorm else mm.as_t(m)
    for _ in range(nsteps):
        m = mri_step(p, m, h, ratio, renorm)
    return m
