"""Write adjoint_workload_2000.json: the FP64 oracle's discrete-adjoint gradient
of the adjoint workload (128 x 128 x 1 cells, Ms map in [6e5, 1e6], DMI,
bias 1e5 A/m along z; J = mean m_z over the central 32 x 32 patch after 2000
RK4 steps of 2e-14 s), sampled, with central differences (h = 1e-4) of the
oracle's forward map along a few directions.

Only ``oracle/`` and the seeded input generators are called; nothing here
touches the CUDA path.  Inputs are rounded to float32 first, as the GPU sees
them.  Run from the repository root:

    python tests/golden/make_adjoint_2000.py

(about 20 minutes of FP64 CPU work).
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import adjoint as oadj  # noqa: E402
from oracle import micromag as mm  # noqa: E402
from paper_2602_12242_gb300 import inputs  # noqa: E402

NSTEPS = 2000
PATCH = ((48, 80), (48, 80))  # central 32 x 32 of 128 x 128
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "adjoint_workload_2000.json")


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def main():
    c = dict(inputs.CONFIGS["adjoint"])
    Ms, _, _ = inputs.material("adjoint")
    Ms = f32(Ms)
    m0 = f32(inputs.initial_m("adjoint"))
    p = mm.Problem(c["nx"], c["ny"], c["nz"], c["dx"], c["dy"], c["dz"], Ms=Ms, A=c["A"], Ku=c["Ku"],
                   ku_axis=c["ku_axis"], D=c["D"], alpha=c["alpha"], gamma=c["gamma"], h_bias=c["h_bias"],
                   dmi=c["dmi"], demag=True, precession=True)
    obj = lambda m: oadj.patch_mean_mz(m, PATCH)  # noqa: E731
    t0 = time.time()
    J, g, gms = oadj.gradient(p, m0, c["dt"], NSTEPS, obj)
    g, gms = g.numpy(), gms.numpy()
    t1 = time.time()
    rng = np.random.default_rng(2000)
    # sampled cells: 512 uniform, plus the 16 largest |g| entries
    flat = rng.choice(g.size, size=512, replace=False)
    top = np.argsort(-np.abs(g).ravel())[:16]
    cells = rng.choice(gms.size, size=512, replace=False)
    # central differences: the two largest-|g| single entries, one random direction of (m0, Ms / 1e6)
    fd = []
    for k in top[:2]:
        dm = np.zeros(g.size)
        dm[k] = 1.0
        v = oadj.central_fd(p, m0, c["dt"], NSTEPS, obj, direction_m=dm.reshape(g.shape), direction_ms=None, h=1e-4)
        fd.append({"entry": int(k), "fd": v})
    rd = np.random.default_rng(2001)
    dm = rd.normal(size=g.shape)
    ds = rd.normal(size=gms.shape)
    nrm = np.sqrt((dm ** 2).sum() + (ds ** 2).sum())
    dm, ds = dm / nrm, 1e6 * ds / nrm
    v = oadj.central_fd(p, m0, c["dt"], NSTEPS, obj, direction_m=dm, direction_ms=ds, h=1e-4)
    fd.append({"random_seed": 2001, "fd": v})
    t2 = time.time()
    out = {
        "_about": "FP64 oracle (oracle.adjoint.gradient / central_fd) on the adjoint workload, written by "
                  "tests/golden/make_adjoint_2000.py; gradient w.r.t. the raw initial m (dJ/dm0) and the "
                  "per-cell Ms map (dJ/dMs) after 2000 RK4 steps; samples, full-field norms and central "
                  "differences (h = 1e-4). The random direction of the last fd entry is "
                  "np.random.default_rng(2001): normal m0 part then normal Ms part, jointly normalised, "
                  "Ms part times 1e6.",
        "nsteps": NSTEPS, "patch": PATCH, "dt": c["dt"], "J": J,
        "g_norm": float(np.linalg.norm(g)), "gms_norm": float(np.linalg.norm(gms)),
        "g_index": [int(i) for i in np.concatenate([flat, top])],
        "g_value": [float(v) for v in g.ravel()[np.concatenate([flat, top])]],
        "gms_index": [int(i) for i in cells],
        "gms_value": [float(v) for v in gms.ravel()[cells]],
        "fd": fd,
        "cpu_seconds": {"gradient": round(t1 - t0, 1), "fd": round(t2 - t1, 1)},
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT, out["cpu_seconds"])


if __name__ == "__main__":
    main()
