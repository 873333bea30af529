"""Oracle: FP64 snapshots of a workload's RK4 trajectory, and the divergence
of another run's snapshots from them (the FP32-vs-FP64 divergence curve).

TEST INFRASTRUCTURE ONLY (plain FP64 CPU; the product never imports it).

  python -m oracle.trajectory run film --steps 20000 --every 1000 --out film_fp64.npz
  python -m oracle.trajectory compare film_fp64.npz film_fp32.npz

The run is ``micromag.rk4_step`` (classical RK4, renormalised after every
stage, Sec. II-B) from the workload's seeded initial state; the initial state,
maps and parameters come from the shared input generators.
"""
import argparse
import sys

import numpy as np
import torch

from . import micromag as mm


def problem(name):
    from paper_2602_12242_gb300 import inputs
    c = inputs.CONFIGS[name]
    Ms, Ku, axis = inputs.material(name)
    return mm.Problem(c["nx"], c["ny"], c["nz"], c["dx"], c["dy"], c["dz"], Ms=Ms, A=c["A"], Ku=Ku, ku_axis=axis,
                      D=c["D"], alpha=c["alpha"], gamma=c["gamma"], h_bias=c["h_bias"], dmi=c["dmi"]), c


def run(name, steps, every, log=None):
    from paper_2602_12242_gb300 import inputs
    p, c = problem(name)
    m = mm.normalize(torch.from_numpy(np.ascontiguousarray(inputs.initial_m(name))))
    snaps, at = [m.numpy().copy()], [0]
    for s in range(1, steps + 1):
        m = mm.rk4_step(p, m, c["dt"])
        if s % every == 0 or s == steps:
            snaps.append(m.numpy().copy())
            at.append(s)
            if log:
                log(f"step {s}")
    return np.stack(snaps), np.array(at)


def compare(ref, other):
    """Rows (step, max_i |m_i - m_ref,i|, rms) over the common snapshot steps."""
    rows = []
    for k, s in enumerate(ref["step"]):
        j = np.nonzero(other["step"] == s)[0]
        if len(j) == 0:
            continue
        d = np.linalg.norm(other["m"][j[0]].astype(np.float64) - ref["m"][k], axis=-1)
        rows.append((int(s), float(d.max()), float(np.sqrt((d ** 2).mean()))))
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    r = sub.add_parser("run")
    r.add_argument("workload")
    r.add_argument("--steps", type=int, default=20000)
    r.add_argument("--every", type=int, default=1000)
    r.add_argument("--out", required=True)
    c = sub.add_parser("compare")
    c.add_argument("ref")
    c.add_argument("other")
    a = ap.parse_args(argv)
    if a.cmd == "run":
        snaps, at = run(a.workload, a.steps, a.every, log=lambda s: print(s, file=sys.stderr, flush=True))
        np.savez_compressed(a.out, m=snaps, step=at)
    else:
        print("| step | max_i abs(m - m_FP64) | rms |")
        print("|---|---|---|")
        for s, mx, rms in compare(np.load(a.ref), np.load(a.other)):
            print(f"| {s} | {mx:.3e} | {rms:.3e} |")


if __name__ == "__main__":
    main()
