"""Benchmark: cell-steps/s of the full H_eff + LLG RK4 step on one GB300.

Default workload: the bulk grid, 512x512x16 cells of 2 nm (padded
1024x1024x32), random m, 32x32x16 grains of random easy axis, RK4 with
dt = 1e-14 s.  Its working set (~0.9 GB) is far larger than L2, so no L2 flush
is needed between steps.  A step is one RK4 step: four evaluations of the
demag convolution and the fused local kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mx|reference]
                  [--workload bulk|film|plain] [--no-cpu-baseline]

Prints one JSON line.  Under torchrun (N > 1) every rank runs an independent
replica (the method on one grid does not shard without an exchange step);
value is the sum over ranks of cells x steps divided by the slowest rank's
time.  ``--impl reference`` times the plain FP64 CPU oracle instead (the
reference arm): each of its steps is one RK4 step of a bounded crop of the
workload on the host cores.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "bulk": "bulk 512x512x16 (2 nm cells, grains), RK4 dt 1e-14 s",
    "film": "film 512x128x1 (3.9x3.9x3 nm, DMI 1.5e-3 chiral), RK4 dt 5e-14 s",
    "plain": "plain 32x32x4 (2 nm), RK4 dt 1e-14 s",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mx", choices=["mx", "reference"])
    ap.add_argument("--workload", default="bulk", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# distributed plumbing
# ----------------------------------------------------------------------------
def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (args.impl == "mx" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world, device=None):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# workload setup
# ----------------------------------------------------------------------------
def workload(name):
    from paper_2602_12242_gb300 import inputs
    cfg = dict(inputs.CONFIGS[name])
    m0 = inputs.initial_m(name)
    Ms, Ku, axis = inputs.material(name)
    return cfg, m0, Ms, Ku, axis


def algorithmic_bytes(cfg, P, ms_map=False, ku_map=False, axis_map=False):
    """Algorithmic HBM bytes per launch of each kernel (FP32 spectra, float4
    fields; a per-cell Ms map adds 4 B/cell to the x pass and the local
    kernel, a Ku map 4 B/cell and an easy-axis map (float4) 16 B/cell to the
    local kernel)."""
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    Px, Py, Pz = P
    Hx = Px // 2 + 1 if Px > 1 else 1
    nc = nx * ny * nz
    w1 = 3 * nz * ny * Hx * 8           # spectrum after the x pass
    w2 = 3 * nz * Py * Hx * 8           # after the y pass
    tensor = (6 if Pz > 1 else 4) * (Pz // 2 + 1) * (Py // 2 + 1) * Hx * 4
    maps = (4 if ms_map else 0) + (4 if ku_map else 0) + (16 if axis_map else 0)
    return {
        "x_fwd": nc * (16 + (4 if ms_map else 0)) + w1,
        "y_fwd": w1 + w2,
        "z_mul": 2 * w2 + tensor,
        "y_inv": w2 + w1,
        "yz_fused": 2 * w1 + tensor,
        "x_inv": w1 + nc * 16,
        # RK4 stage average: (64 + 96 + 96 + 80) / 4 bytes per cell, plus the maps
        "local_stage": nc * (84 + maps),
        # inverse x fused with the local stage: H_demag neither stored nor read
        "x_inv_local": w1 + nc * (68 + maps),
        "normalize": nc * 32,
        "copy": nc * 32,
    }


CSRC = os.path.join(ROOT, "paper_2602_12242_gb300", "csrc")
# translation unit that defines each kernel of the traffic table
KERNEL_TU = {"yzq_kernel": "demag_quad.cu", "yzh_kernel": "demag_plane.cu", "xfk_kernel": "demag_plane.cu",
             "xik_kernel": "demag_plane.cu", "xil_kernel": "demag_plane.cu", "xr_kernel": "demag_fast.cu",
             "local_kernel": "local.cu"}


def kernel_sources(kernel):
    """The kernel's translation unit and every local header it includes,
    directly or through other headers (paths relative to the repository)."""
    todo, seen = [os.path.join(CSRC, KERNEL_TU[kernel])], set()
    while todo:
        f = os.path.normpath(todo.pop())
        if f in seen:
            continue
        seen.add(f)
        for inc in re.findall(r'^\s*#include\s+"([^"]+)"', open(f).read(), flags=re.M):
            todo.append(os.path.join(os.path.dirname(f), inc))
    return sorted(os.path.relpath(f, ROOT) for f in seen)


def _code_text(path):
    """A source file without its comments and with whitespace collapsed, so
    that comment and layout edits leave the digest alone."""
    text = re.sub(r"//[^\n]*|/\*.*?\*/", " ", open(path).read(), flags=re.S)
    return " ".join(text.split())


def source_digest(kernel=None):
    """sha256 (first 16 hex digits) of the code a kernel is compiled from
    (file names and their text without comments); without a kernel, of every
    file under csrc/ byte for byte."""
    h = hashlib.sha256()
    if kernel is None:
        for f in sorted(os.listdir(CSRC)):
            h.update(open(os.path.join(CSRC, f), "rb").read())
    else:
        for rel in kernel_sources(kernel):
            h.update(rel.encode())
            h.update(_code_text(os.path.join(ROOT, rel)).encode())
    return h.hexdigest()[:16]


def load_traffic(workload_name, kernel):
    """dram bytes per launch of `kernel` from a committed ncu summary, if the
    kernel sources have not changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        e = d.get(workload_name, {}).get(kernel)
        if e and e.get("source_digest") == source_digest(kernel):
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def run_mx(args, rank, world, local, name, with_extras=True):
    import torch
    from paper_2602_12242_gb300.solver import Context, to_dev4

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    cfg, m0, Ms, Ku, axis = workload(name)
    ctx = Context.from_config(cfg, Ms=Ms, Ku=Ku, ku_axis=axis)
    m = to_dev4(m0, dev)
    dt = cfg["dt"]
    nc = cfg["nx"] * cfg["ny"] * cfg["nz"]
    K, W = args.steps, args.warmup
    stream = torch.cuda.current_stream()

    ctx.rk_step(m, W, dt)  # warm-up (also captures the step graph)
    ctx.sync()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.4)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.rk_step(m, K, dt)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    ctx.sync()
    ms_max = max_over_ranks(ms, world, dev)
    value = world * nc * K / (ms_max * 1e-3)
    res = {"ms": ms_max, "value": value, "clocks": clk, "launches_per_step": None}
    if not with_extras:
        ctx.close()
        return res

    # kernel times with direct launches, same steps (event pair per launch)
    prof = ctx.profile_step(m, K, dt)
    ctx.sync()
    P = ctx.padded_dims
    ab = algorithmic_bytes(cfg, P, ms_map=not np.isscalar(Ms), ku_map=not np.isscalar(Ku),
                           axis_map=np.asarray(axis).ndim > 1)
    launches = sum(c for (_, c) in prof.values())
    per_step = (launches - 1) / K  # one normalisation per call
    res["launches_per_step"] = per_step
    res["gpu_launches"] = int(round(per_step * K)) + 1
    names = ctx.kernel_names()
    if names.get("x_inv_local") == "xr_kernel":
        # the row kernel also writes the next stage's spectrum (3 stages of 4)
        ab["x_inv_local"] += 3 * (ab["x_inv"] - cfg["nx"] * cfg["ny"] * cfg["nz"] * 16) // 4
    dom = max(prof, key=lambda k: prof[k][0])
    tot = sum(v[0] for v in prof.values())
    kern = {k: {"kernel": names.get(k, k), "ms_total": round(v[0], 4), "launches": v[1],
                "share": round(v[0] / tot, 4),
                "us_per_launch": round(1e3 * v[0] / v[1], 3),
                "gbs": round(ab.get(k, 0) / (1e-3 * v[0] / v[1]) / 1e9, 1)} for k, v in prof.items()}
    res["kernels"] = kern
    peak, src = peaks()
    achieved = ab[dom] / (1e-3 * prof[dom][0] / prof[dom][1]) / 1e9
    res["roofline"] = {"bound": "hbm", "kernel": names.get(dom, dom), "slot": dom, "achieved": round(achieved, 1),
                       "peak": peak, "peak_source": src, "unit": "GB/s", "frac": round(achieved / peak, 4),
                       "traffic": load_traffic(name, names.get(dom, dom)),
                       "algorithmic_bytes_per_launch": ab[dom]}
    demag = [k for k in prof if k in ("x_fwd", "y_fwd", "z_mul", "y_inv", "yz_fused", "x_inv")]
    dbytes = sum(ab[k] * prof[k][1] for k in demag)
    dms = sum(prof[k][0] for k in demag)
    res["demag_conv_gbs"] = round(dbytes / (dms * 1e-3) / 1e9, 1)
    res["step_ms_direct"] = round(tot / K, 4)

    # end to end through the public API with host buffers: H2D of m from pinned
    # memory, one RK4 step, D2H of the new m, every step
    host = m.cpu().pin_memory()
    out = torch.empty_like(host).pin_memory()
    ctx.rk_step(m, 1, dt)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(K):
        m.copy_(host, non_blocking=True)
        ctx.rk_step(m, 1, dt)
        out.copy_(m, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - t0
    e2e_ms = max_over_ranks(max(f0.elapsed_time(f1), wall * 1e3), world, dev)
    res["e2e"] = {"value": world * nc * K / (e2e_ms * 1e-3), "unit": "cell-steps/s",
                  "h2d_bytes_per_step": int(host.numel() * 4), "d2h_bytes_per_step": int(out.numel() * 4)}
    ctx.close()
    return res


# ----------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ----------------------------------------------------------------------------
def oracle_problem(cfg, Ms, Ku, axis, crop):
    from oracle import micromag as mm
    nx, ny, nz = crop
    sl = (slice(0, nz), slice(0, ny), slice(0, nx))
    Ms_c = Ms if np.isscalar(Ms) else np.asarray(Ms)[sl]
    Ku_c = Ku if np.isscalar(Ku) else np.asarray(Ku)[sl]
    ax_c = axis if (isinstance(axis, tuple) or np.asarray(axis).ndim == 1) else np.asarray(axis)[sl]
    return mm.Problem(nx, ny, nz, cfg["dx"], cfg["dy"], cfg["dz"], Ms=Ms_c, A=cfg["A"], Ku=Ku_c, ku_axis=ax_c,
                      D=cfg["D"], alpha=cfg["alpha"], gamma=cfg["gamma"], h_bias=cfg["h_bias"], dmi=cfg["dmi"])


def time_oracle(name, crop, steps):
    import torch
    from oracle import micromag as mm
    cfg, m0, Ms, Ku, axis = workload(name)
    p = oracle_problem(cfg, Ms, Ku, axis, crop)
    nx, ny, nz = crop
    m = mm.normalize(torch.from_numpy(np.ascontiguousarray(m0[:nz, :ny, :nx])))
    mm.padded_tensor_spectrum(p)  # tensor build is set-up, not timed
    t0 = time.perf_counter()
    for _ in range(steps):
        m = mm.rk4_step(p, m, cfg["dt"])
    dt = time.perf_counter() - t0
    return nx * ny * nz * steps / dt, dt, torch.get_num_threads()


def crop_for(name, budget_steps):
    from paper_2602_12242_gb300 import inputs
    c = inputs.CONFIGS[name]
    nx, ny, nz = c["nx"], c["ny"], c["nz"]
    if name != "bulk":
        return (nx, ny, nz)
    # about one second of FP64 CPU work per RK4 step on a bounded crop
    side = 512 if budget_steps <= 2 else (256 if budget_steps <= 10 else (128 if budget_steps <= 60 else 64))
    return (side, side, nz)


def cpu_model():
    """Host CPU description from /proc/cpuinfo (x86 'model name', Arm implementer/part)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return "unknown"
    for key in ("model name", "Model"):
        for line in info:
            if line.startswith(key):
                return line.split(":", 1)[1].strip()
    impl = [l.split(":", 1)[1].strip() for l in info if l.startswith("CPU implementer")]
    part = [l.split(":", 1)[1].strip() for l in info if l.startswith("CPU part")]
    return f"implementer {impl[0]} part {part[0]}" if impl and part else "unknown"


def cpu_baseline(name):
    import torch
    crop = crop_for(name, 2)
    if name == "bulk":
        crop = (256, 256, 16)
    value, secs, threads = time_oracle(name, crop, 2)
    # the same oracle on one core, on a smaller crop of the same workload
    crop1 = (64, 64, crop[2]) if name == "bulk" else crop
    nthreads = torch.get_num_threads()
    torch.set_num_threads(1)
    try:
        value1, secs1, _ = time_oracle(name, crop1, 2)
    finally:
        torch.set_num_threads(nthreads)
    return {"value": value, "unit": "cell-steps/s", "cores": threads, "kind": "oracle",
            "sample": f"2 RK4 steps of the FP64 oracle on a {crop[0]}x{crop[1]}x{crop[2]} crop of the "
                      f"{name} workload ({secs:.1f} s, torch CPU FFT, {threads} threads)",
            "single_core": {"value": value1, "sample": f"2 RK4 steps on a {crop1[0]}x{crop1[1]}x{crop1[2]} crop, "
                                                       f"1 thread ({secs1:.1f} s)"},
            "host": {"cpu_count": os.cpu_count(), "cpu_model": cpu_model()}}


def run_reference(args, rank, world):
    name = args.workload
    if rank != 0:
        return None
    crop = crop_for(name, args.steps + args.warmup)
    from paper_2602_12242_gb300 import inputs
    c = inputs.CONFIGS[name]
    if args.warmup:
        time_oracle(name, crop, 1)
    value, secs, threads = time_oracle(name, crop, args.steps)
    line = {"metric": "cell-steps/s (full H_eff+LLG RK4 step)", "value": value, "unit": "cell-steps/s",
            "impl": "reference", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": {"workload": WORKLOADS[name], "cells": c["nx"] * c["ny"] * c["nz"],
                       "sample_crop": list(crop), "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": "cell-steps/s", "cores": threads, "kind": "oracle",
                             "sample": f"each step: one RK4 step of the FP64 oracle on a "
                                       f"{crop[0]}x{crop[1]}x{crop[2]} crop of the {name} workload"},
            "e2e": {"value": value, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


def main():
    args = parse()
    rank, world, local = dist_init(args)
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    name = args.workload
    from paper_2602_12242_gb300 import inputs
    c = inputs.CONFIGS[name]
    res = run_mx(args, rank, world, local, name)
    secondary = None
    if not args.no_secondary and name == "bulk":
        sec = run_mx(args, rank, world, local, "film", with_extras=False)
        secondary = {"workload": WORKLOADS["film"], "value": sec["value"], "unit": "cell-steps/s",
                     "ms_per_step": sec["ms"] / args.steps}
    if rank != 0:
        return
    line = {
        "metric": "cell-steps/s (full H_eff+LLG RK4 step)",
        "value": res["value"], "unit": "cell-steps/s", "cell_stages_per_s": 4 * res["value"],
        "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
        "config": {"workload": WORKLOADS[name], "cells": c["nx"] * c["ny"] * c["nz"],
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "no flush: working set ~0.9 GB > 129 MB L2" if name == "bulk" else "L2-resident"},
        "roofline": res["roofline"],
        "demag_conv_gbs": res["demag_conv_gbs"],
        "e2e": res["e2e"],
        "gpu_launches": res["gpu_launches"],
        "clocks": res["clocks"],
        "kernels": res["kernels"],
        "step_ms_direct_launch": res["step_ms_direct"],
    }
    if secondary:
        line["secondary"] = secondary
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(name)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
