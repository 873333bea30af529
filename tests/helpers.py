"""Shared test helpers: build the oracle problem and the CUDA context from one config."""
import numpy as np
import torch

from oracle import micromag as mm
from paper_2602_12242_gb300 import inputs

BASE = dict(nx=8, ny=8, nz=2, dx=2e-9, dy=2e-9, dz=2e-9, Ms=8e5, A=1.3e-11, Ku=5e3, ku_axis=(0.0, 0.0, 1.0),
            D=0.0, dmi=False, alpha=0.5, gamma=2.211e5, h_bias=(0.0, 0.0, 1e4))


def cfg_of(**kw):
    c = dict(BASE)
    c.update(kw)
    return c


def problem(cfg, Ms=None, Ku=None, axis=None, demag=True, precession=True):
    return mm.Problem(cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["dy"], cfg["dz"],
                      Ms=cfg["Ms"] if Ms is None else Ms, A=cfg["A"], Ku=cfg["Ku"] if Ku is None else Ku,
                      ku_axis=cfg["ku_axis"] if axis is None else axis, D=cfg["D"], alpha=cfg["alpha"],
                      gamma=cfg["gamma"], h_bias=cfg["h_bias"], dmi=cfg["dmi"], demag=demag,
                      precession=precession)


def context(cfg, Ms=None, Ku=None, axis=None, demag=True, demag_path=0, fft_mode=0, **kw):
    from paper_2602_12242_gb300.solver import Context
    c = dict(cfg)
    return Context.from_config(c, Ms=Ms, Ku=Ku, ku_axis=axis, demag=demag, demag_path=demag_path,
                               fft_mode=fft_mode, **kw)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_max(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def random_m(cfg, seed):
    return inputs.unit_random((cfg["nz"], cfg["ny"], cfg["nx"]), seed)


def t64(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
