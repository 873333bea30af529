"""muMAG Standard Problem 3 set-up of Sec. III-B shared by the oracle and GPU
tests: the cube, the two initial states and the energy densities in units of
K_m."""
import json
import math
import os

import numpy as np

MU0 = 4e-7 * math.pi
MS, A = 8.0e5, 1.005154e-11
KM = 0.5 * MU0 * MS ** 2
LEX = math.sqrt(2.0 * A / (MU0 * MS ** 2))
GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "sp3_table1_n10.json")))


def cfg(n=GOLDEN["N"], L=GOLDEN["L_over_lex"]):
    h = L * LEX / n
    return dict(nx=n, ny=n, nz=n, dx=h, dy=h, dz=h, Ms=MS, A=A, Ku=0.1 * KM, ku_axis=(0.0, 0.0, 1.0), D=0.0,
                dmi=False, alpha=0.5, gamma=2.211e5, h_bias=(0.0, 0.0, 0.0))


def initial(name, n=GOLDEN["N"]):
    m = np.zeros((n, n, n, 3))
    if name == "flower":
        m[...] = 1.0 / math.sqrt(3.0)
    else:
        m[:, :, : n // 2, 0] = 1.0
        m[:, :, n // 2:, 0] = -1.0
    return m


def densities(c, e_demag, e_exch_central, e_anis):
    V = c["nx"] * c["ny"] * c["nz"] * c["dx"] * c["dy"] * c["dz"]
    return {"e_demag": e_demag / (KM * V), "e_exch": e_exch_central / (KM * V), "e_anis": e_anis / (KM * V)}


def check(name, d, mean_m, tol=1e-3):
    """Energy densities and the mean magnetisation component against Table I."""
    g = GOLDEN[name]
    for k in ("e_demag", "e_exch", "e_anis"):
        assert abs(d[k] - g[k]) <= tol, (name, k, d[k], g[k])
    if name == "flower":
        assert abs(mean_m[2] - g["m_z"]) <= tol, (name, mean_m)
    else:
        assert abs(abs(mean_m[1]) - g["m_y"]) <= tol, (name, mean_m)
