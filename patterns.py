"""Reports of the method's patterns against the plain FP32 path on one GPU.

  python patterns.py [--pairs N] [--epochs E] [--insteps S] [--out FILE]

learned: the conv-net surrogate trained on (m, H_demag) pairs from the FFT
  path on the learned workload (64x64x4 cells, smooth textures); held-out
  error, time per demag evaluation and per RK4 step against the FFT, and an
  in-loop run with the FFT as judge (every --judge steps) and fallback (error
  above 1e-2), with the drift of m against the FFT-only trajectory.
adjoint: time of the recorded forward plus the reverse sweep against the
  plain forward run for the adjoint workload (128x128x1, 2000 RK4 steps,
  a checkpoint every 100).

  python patterns.py --trajectory film --steps 20000 --every 1000 --npz FILE

trajectory: snapshots of m every --every RK4 steps of a workload from its
  seeded initial state (for the FP32-vs-FP64 divergence curve).

  python patterns.py --fft-mode-timing

fft-mode timing: per-kernel time of the bulk RK4 step with FP32 x transforms
  and with the split-BF16 DFT-as-GEMM first x stage.

  python patterns.py --fno [--train-sims N] [--frames F] [--epochs E] [--batch B] [--out FILE]

fno: the Fourier-neural-operator surrogate and the conv net trained on the
  same SP4 film pairs (160x40x1 cells of 3.125 nm; S-state, then random
  in-plane fields of 25-40 mT, F snapshots over 1 ns each); held-out demag
  error, <m>(t) over 1 ns under the two SP4 fields with each network as the
  demag backend against the FFT run, and times.

  python patterns.py --fno-timing

fno timing: per-call time of FNO inference (1 field, 128 fields) and of one
  training step of 128 fields on the SP4 film grid.

  python patterns.py --mri

mri: time to solution of RK4 and of the explicit-explicit MRI step on the SP4
  film with the stiffened 0.78125 nm grid (640x160x4), MRI at 5x the RK4 step,
  both against a fine RK4 reference.
"""
import argparse
import json
import time

import numpy as np
import torch

import os
import sys

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from paper_2602_12242_gb300 import _lib as L  # noqa: E402
from paper_2602_12242_gb300 import inputs  # noqa: E402
from paper_2602_12242_gb300.solver import Context, to_dev4  # noqa: E402
from paper_2602_12242_gb300.surrogate import (FourierSurrogate, Surrogate, init_fno_params, init_params, make_dataset, normalizer_stats,
                        run_in_loop, time_batched, time_demag, train)


def _rk_time(ctx, m, n, dt):
    ctx.rk_step(m, 2, dt)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctx.rk_step(m, n, dt)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def learned_report(pairs, epochs, batch, insteps, judge, holdout=64, log=print):
    cfg = dict(inputs.CONFIGS["learned"])
    ctx = Context.from_config(cfg)
    t0 = time.perf_counter()
    M, H = make_dataset(ctx, pairs + holdout, seed0=inputs.SEEDS["learned"])
    t_data = time.perf_counter() - t0
    net = Surrogate(cfg["nx"], cfg["ny"], cfg["nz"], max_batch=batch)
    net.set_params(torch.as_tensor(init_params(11)))
    net.set_normalizer(normalizer_stats(M[:pairs], H[:pairs]))
    pred0 = net.forward(M[pairs:pairs + 1][0])
    err_untrained = L.mx_rel_l2(ctx.h, pred0, H[pairs])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = train(net, M[:pairs], H[:pairs], epochs=epochs, batch=batch, log=log)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    errs = []
    for i in range(pairs, pairs + holdout):
        errs.append(L.mx_rel_l2(ctx.h, net.forward(M[i]), H[i]))
    m_test = M[pairs].clone()
    tdem = time_demag(ctx, net, m_test)
    tbatch = time_batched(ctx, net, M[pairs:pairs + holdout])
    # RK4 step time with each backend
    m1 = M[pairs].clone()
    t_fft = _rk_time(ctx, m1, 100, cfg["dt"])
    L.mx_set_demag_surrogate(ctx.h, net.h)
    m2 = M[pairs].clone()
    t_sur = _rk_time(ctx, m2, 100, cfg["dt"])
    L.mx_set_demag_surrogate(ctx.h, None)
    # in-loop runs from a held-out texture
    ref = M[pairs + 1].clone()
    ctx.rk_step(ref, insteps, cfg["dt"])
    judged = M[pairs + 1].clone()
    res = run_in_loop(ctx, net, judged, insteps, cfg["dt"], judge, threshold=1e-2)
    free = M[pairs + 1].clone()
    res_free = run_in_loop(ctx, net, free, insteps, cfg["dt"], judge, threshold=float("inf"))
    drift_free = float((free[..., :3] - ref[..., :3]).abs().max())
    drift_judged = float((judged[..., :3] - ref[..., :3]).abs().max())
    return {
        "workload": "learned 64x64x4, smooth textures sigma 8 cells",
        "pairs": pairs, "holdout": holdout, "epochs": epochs, "batch": batch,
        "dataset_s": t_data, "train_s": t_train,
        "train_samples_per_s": pairs * epochs / t_train,
        "loss_first_last": [losses[0], losses[-1]],
        "holdout_rel_l2_mean": float(np.mean(errs)), "holdout_rel_l2_max": float(np.max(errs)),
        "untrained_rel_l2": err_untrained,
        "demag_eval_ms": tdem, "batched_demag_ms_per_field": tbatch,
        "rk4_step_ms": {"fft": t_fft, "surrogate": t_sur},
        "in_loop": {"steps": insteps, "judge_every": judge, "threshold": 1e-2,
                    "fallback_step": res["fallback_step"], "first_errors": res["errors"][:5],
                    "free_run_errors": res_free["errors"][:: max(1, len(res_free["errors"]) // 10)],
                    "max_drift_m_free_run": drift_free, "max_drift_m_judged_run": drift_judged},
    }


SP4_FILM = dict(nx=160, ny=40, nz=1, dx=3.125e-9, dy=3.125e-9, dz=3.125e-9, Ms=8e5, A=1.3e-11, Ku=0.0,
                ku_axis=(0.0, 0.0, 1.0), D=0.0, dmi=False, alpha=0.02, gamma=2.211e5, h_bias=(0.0, 0.0, 0.0))
MU0 = 4e-7 * np.pi


def sp4_s_state(dt=1e-13):
    """The S-state of Sec. III-D: m = (1, 0, 0), alpha 0.5, a (1e5, 1e5, 1e5) A/m
    field for 20 ps, ramped linearly to zero over 10 ps (in 1 ps steps), then
    1 ns of relaxation without field (RK4)."""
    cfg = dict(SP4_FILM, alpha=0.5)
    ctx = Context.from_config(cfg)
    m0 = np.zeros((1, cfg["ny"], cfg["nx"], 3))
    m0[..., 0] = 1.0
    m = to_dev4(m0)
    ctx.set_bias((1e5, 1e5, 1e5))
    ctx.rk_step(m, int(round(20e-12 / dt)), dt)
    for q in range(10):
        f = 1e5 * (1.0 - (q + 0.5) / 10.0)
        ctx.set_bias((f, f, f))
        ctx.rk_step(m, int(round(1e-12 / dt)), dt)
    ctx.set_bias((0.0, 0.0, 0.0))
    ctx.rk_step(m, int(round(1e-9 / dt)), dt)
    ctx.sync()
    ctx.close()
    return m


def sp4_fields(n, seed):
    """n bias fields of Sec. II-D: magnitude uniform in 25-40 mT, direction
    uniform on the sphere projected into the film plane [A/m]."""
    r = inputs.rng(seed)
    v = r.normal(size=(n, 3))
    v[:, 2] = 0.0
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    mag = r.uniform(25e-3, 40e-3, size=n) / MU0
    return v * mag[:, None]


def sp4_dataset(ctx, s_state, fields, T=1e-9, frames=20, dt=1e-13):
    """(m, H_demag) pairs: from the S-state, each field drives the film for T
    (RK4, alpha 0.02); a snapshot every T/frames."""
    n = len(fields) * frames
    M = torch.empty((n,) + tuple(s_state.shape), dtype=torch.float32, device="cuda")
    H = torch.empty_like(M)
    every = int(round(T / frames / dt))
    q = 0
    for f in fields:
        ctx.set_bias(tuple(float(v) for v in f))
        m = s_state.clone()
        for _ in range(frames):
            ctx.rk_step(m, every, dt)
            M[q] = m
            ctx.heff(m, out=H[q], terms=L.MX_TERM_DEMAG)
            q += 1
    torch.cuda.synchronize()
    return M, H


def mean_m_curve(ctx, m, steps, every, dt, net=None):
    """<m> every `every` RK4 steps (the net, if given, as the demag backend)."""
    out = []
    if net is not None:
        net.attach(ctx.h)
    try:
        for _ in range(steps // every):
            ctx.rk_step(m, every, dt)
            out.append(m[..., :3].double().mean(dim=(0, 1, 2)))
    finally:
        if net is not None:
            net.detach(ctx.h)
    ctx.sync()
    return torch.stack(out).cpu().numpy()


def fno_report(train_sims=96, val_sims=8, frames=100, epochs=100, batch=32, modes=12, log=print):
    """The FNO surrogate (Sec. II-D) and the conv net trained on the same SP4
    film pairs (160 x 40 x 1, 3.125 nm): held-out demag error, in-loop <m>(t)
    under the two SP4 fields against the FFT run, and times."""
    dt = 1e-13
    t0 = time.perf_counter()
    s_state = sp4_s_state(dt)
    ctx = Context.from_config(dict(SP4_FILM))
    fields = sp4_fields(train_sims + val_sims, 2602)
    M, H = sp4_dataset(ctx, s_state, fields, frames=frames, dt=dt)
    t_data = time.perf_counter() - t0
    ntr = train_sims * frames
    stats = normalizer_stats(M[:ntr], H[:ntr])
    nets = {
        "fno": FourierSurrogate(SP4_FILM["nx"], SP4_FILM["ny"], modes, max_batch=batch),
        "cnn": Surrogate(SP4_FILM["nx"], SP4_FILM["ny"], 1, max_batch=batch),
    }
    nets["fno"].set_params(torch.as_tensor(init_fno_params(modes, 12)))
    nets["cnn"].set_params(torch.as_tensor(init_params(11)))
    out = {"workload": "SP4 film 160x40x1 (3.125 nm), S-state + random in-plane fields 25-40 mT",
           "train_pairs": ntr, "val_pairs": val_sims * frames, "epochs": epochs, "batch": batch, "modes": modes,
           "dataset_s": t_data, "params": {k: n.n_params for k, n in nets.items()}}
    ms = (20, 40, 60)
    sp4 = {"field1": (-19576.0, 3422.0, 0.0), "field2": (-28259.0, -5013.0, 0.0)}
    curves = {}
    for f, hb in sp4.items():
        ctx.set_bias(hb)
        curves[(f, "fft")] = mean_m_curve(ctx, s_state.clone(), 10000, 100, dt)
    for name, net in nets.items():
        net.set_normalizer(stats)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        losses = train(net, M[:ntr], H[:ntr], epochs=epochs, batch=batch, milestones=ms, log=None)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t1
        errs = [L.mx_rel_l2(ctx.h, net.forward(M[i]), H[i]) for i in range(ntr, M.shape[0])]
        r = {"train_s": t_train, "train_samples_per_s": ntr * epochs / t_train,
             "loss_first_last": [losses[0], losses[-1]],
             "val_rel_l2_mean": float(np.mean(errs)), "val_rel_l2_max": float(np.max(errs)),
             "demag_eval_ms": time_demag(ctx, net, M[ntr].clone()),
             "batched_demag_ms_per_field": time_batched(ctx, net, M[ntr:ntr + batch])}
        for f, hb in sp4.items():
            ctx.set_bias(hb)
            c = mean_m_curve(ctx, s_state.clone(), 10000, 100, dt, net)
            ref = curves[(f, "fft")]
            r[f] = {"max_abs_mean_m_err": [float(v) for v in np.abs(c - ref).max(axis=0)],
                    "mean_m_at_1ns": [float(v) for v in c[-1]], "fft_mean_m_at_1ns": [float(v) for v in ref[-1]]}
        out[name] = r
        if log:
            log(f"{name}: {json.dumps(r)}")
    return out


def fno_timing(batch=128, modes=12, reps=20):
    """Per-call times of the FNO on the SP4 film grid with seeded parameters
    and fields: inference of one field, inference of `batch` fields, and one
    training step (loss, gradient and Adam) of `batch` fields."""
    nx, ny = SP4_FILM["nx"], SP4_FILM["ny"]
    net = FourierSurrogate(nx, ny, modes, max_batch=batch)
    net.set_params(torch.as_tensor(init_fno_params(modes, 12)))
    net.set_normalizer([0.0, 0.0, 0.0, 0.5, 0.5, 0.5, 0.0, 0.0, 0.0, 1e5, 1e5, 1e5])
    M = torch.stack([to_dev4(inputs.smooth_texture((1, ny, nx), 8.0, 7000 + i)) for i in range(batch)])
    Ht = torch.empty_like(M)
    h1 = torch.empty_like(M[:1])
    out = {"grid": f"{nx}x{ny}x1", "modes": modes, "batch": batch}
    runs = {"infer_1": lambda: net.forward_into(M[:1], h1, 1),
            "infer_batch": lambda: net.forward_into(M, Ht, batch),
            "train_step_batch": lambda: (net.loss_grad(M, Ht, want_grad=False), net.adam_step(1e-4, 1e-4))}
    for name, fn in runs.items():
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        out[name + "_ms"] = e0.elapsed_time(e1) / reps
    out["infer_ms_per_field_batch"] = out["infer_batch_ms"] / batch
    out["train_samples_per_s"] = batch / (out["train_step_batch_ms"] * 1e-3)
    net.close()
    return out


def adjoint_report(nsteps=2000, every=100):
    cfg = dict(inputs.CONFIGS["adjoint"])
    Ms, _, _ = inputs.material("adjoint")
    ctx = Context.from_config(cfg, Ms=Ms)
    m0 = to_dev4(inputs.initial_m("adjoint"))
    m = m0.clone()
    t_plain = _rk_time(ctx, m, nsteps, cfg["dt"]) * nsteps
    ctx.adjoint_reserve(nsteps, every)
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record()
    mT = ctx.rk_forward_record(m0, cfg["dt"])
    e1.record()
    lam = torch.zeros_like(mT)
    lam[:, 48:80, 48:80, 2] = 1.0 / (32 * 32)
    g, gms = ctx.rk_backward(lam)
    e2.record()
    torch.cuda.synchronize()
    return {"workload": f"adjoint 128x128x1, {nsteps} RK4 steps, checkpoint every {every}",
            "plain_forward_ms": t_plain, "recorded_forward_ms": e0.elapsed_time(e1),
            "backward_ms": e1.elapsed_time(e2),
            "gradient_cost_over_plain_forward": e0.elapsed_time(e2) / t_plain,
            "grad_m0_norm": float(g[..., :3].norm()), "grad_ms_norm": float(gms.norm())}


def fft_mode_timing(name="bulk", steps=20):
    """Per-kernel microseconds per launch of one workload's RK4 step with the
    FP32 x transforms and with the split-BF16 DFT-as-GEMM first x stage."""
    cfg = dict(inputs.CONFIGS[name])
    Ms, Ku, axis = inputs.material(name)
    out = {}
    for label, mode in (("fp32", L.MX_FFT_FP32), ("split_bf16", L.MX_FFT_SPLIT_BF16)):
        ctx = Context.from_config(cfg, Ms=Ms, Ku=Ku, ku_axis=axis, fft_mode=mode)
        m = to_dev4(inputs.initial_m(name))
        prof = ctx.profile_step(m, steps, cfg["dt"])
        ctx.sync()
        out[label] = {k: round(1e3 * v[0] / v[1], 2) for k, v in prof.items()}
        ctx.close()
    return out


def mri_report(T=5e-11, dt_rk4=2e-14, mri_factor=5, ref_factor=4):
    """Time to solution of RK4 and of the explicit-explicit MRI step over the
    same interval T on the SP4 film with the stiffened 0.78125 nm grid of
    Sec. III-C (640 x 160 x 4 cubic cells, Ms 8e5, A 1.3e-11, alpha 0.02,
    field (-24.6, 4.3, 0) mT, initial m along (1, 0.25, 0.1) plus 1% seeded
    noise): RK4 at dt_rk4, MRI at mri_factor x dt_rk4, both against RK4 at
    dt_rk4 / ref_factor."""
    h = 0.78125e-9
    mu0 = 4e-7 * np.pi
    cfg = dict(nx=640, ny=160, nz=4, dx=h, dy=h, dz=h, Ms=8e5, A=1.3e-11, Ku=0.0, ku_axis=(0.0, 0.0, 1.0), D=0.0,
               dmi=False, alpha=0.02, gamma=2.211e5, h_bias=(-24.6e-3 / mu0, 4.3e-3 / mu0, 0.0))
    m0 = inputs.near_uniform((4, 160, 640), (1.0, 0.25, 0.1), 0.01, 7)
    out = {"grid": "640x160x4, 0.78125 nm", "T_s": T}
    runs = {"rk4_ref": ("rk4", dt_rk4 / ref_factor), "rk4": ("rk4", dt_rk4), "mri": ("mri", dt_rk4 * mri_factor)}
    res = {}
    for name, (method, dt) in runs.items():
        ctx = Context.from_config(cfg)
        m = to_dev4(m0)
        n = int(round(T / dt))
        ctx.rk_step(m, 1, dt, method)  # capture the step graph outside the timed region
        torch.cuda.synchronize()
        m = to_dev4(m0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.rk_step(m, n, dt, method)
        e1.record()
        torch.cuda.synchronize()
        ctx.sync()
        res[name] = m[..., :3].double().clone()
        out[name] = {"dt_s": dt, "steps": n, "ms": round(e0.elapsed_time(e1), 2)}
        ctx.close()
    for name in ("rk4", "mri"):
        out[name]["max_err_vs_ref"] = float((res[name] - res["rk4_ref"]).abs().max())
    out["mri_speedup_vs_rk4"] = round(out["rk4"]["ms"] / out["mri"]["ms"], 3)
    return out


def trajectory(name, steps, every, perturb=False):
    """m (float32, (n_snap, nz, ny, nx, 3)) at steps 0, every, 2 every, ... of
    a workload's RK4 run from its seeded initial state, and those step counts.
    With ``perturb`` every component of m0 is scaled by 1 +- 2^-24 (seeded
    signs): the run's own sensitivity to rounding-level changes."""
    cfg = dict(inputs.CONFIGS[name])
    Ms, Ku, axis = inputs.material(name)
    ctx = Context.from_config(cfg, Ms=Ms, Ku=Ku, ku_axis=axis)
    m0 = inputs.initial_m(name)
    if perturb:
        m0 = m0 * (1.0 + 2.0 ** -24 * inputs.rng(99).choice([-1.0, 1.0], size=m0.shape))
    m = to_dev4(m0)
    snaps, at = [m[..., :3].cpu().numpy().copy()], [0]
    done = 0
    while done < steps:
        k = min(every, steps - done)
        ctx.rk_step(m, k, cfg["dt"])
        done += k
        snaps.append(m[..., :3].cpu().numpy().copy())
        at.append(done)
    ctx.sync()
    ctx.close()
    return np.stack(snaps), np.array(at)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--trajectory", default=None, choices=list(inputs.CONFIGS))
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--every", type=int, default=1000)
    ap.add_argument("--npz", default=None)
    ap.add_argument("--perturb", action="store_true")
    ap.add_argument("--fft-mode-timing", action="store_true")
    ap.add_argument("--mri", action="store_true")
    ap.add_argument("--fno", action="store_true")
    ap.add_argument("--fno-timing", action="store_true")
    ap.add_argument("--train-sims", type=int, default=96)
    ap.add_argument("--frames", type=int, default=100)
    ap.add_argument("--pairs", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=100)
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--insteps", type=int, default=5000)
    ap.add_argument("--judge", type=int, default=100)
    ap.add_argument("--skip-adjoint", action="store_true")
    ap.add_argument("--adjoint-only", action="store_true")
    ap.add_argument("--adj-steps", type=int, default=2000)
    ap.add_argument("--adj-every", type=int, default=100)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    if a.adjoint_only:
        print(json.dumps(adjoint_report(a.adj_steps, a.adj_every)), flush=True)
        return
    if a.mri:
        print(json.dumps(mri_report()), flush=True)
        return
    if a.fno_timing:
        print(json.dumps(fno_timing()), flush=True)
        return
    if a.fno:
        s = json.dumps(fno_report(train_sims=a.train_sims, frames=a.frames, epochs=a.epochs, batch=a.batch))
        print(s, flush=True)
        if a.out:
            with open(a.out, "w") as f:
                f.write(s + "\n")
        return
    if a.fft_mode_timing:
        print(json.dumps(fft_mode_timing()), flush=True)
        return
    if a.trajectory:
        snaps, at = trajectory(a.trajectory, a.steps, a.every, a.perturb)
        np.savez_compressed(a.npz or f"{a.trajectory}_fp32.npz", m=snaps, step=at)
        return
    rep = {"learned": learned_report(a.pairs, a.epochs, a.batch, a.insteps, a.judge)}
    if not a.skip_adjoint:
        rep["adjoint"] = adjoint_report()
    s = json.dumps(rep)
    print(s, flush=True)
    if a.out:
        with open(a.out, "w") as f:
            f.write(s + "\n")


if __name__ == "__main__":
    main()
