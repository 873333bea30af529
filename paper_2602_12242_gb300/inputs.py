"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the method itself: it only draws seeded
random fields (numpy PCG64) and states the workload parameters.  Every field
is returned as float64 with shape (nz, ny, nx, 3) (cell (i, j, k) at
``[k, j, i]``), or (nz, ny, nx) for scalar maps.

Workloads (stand-ins for the paper's thin-film problem of Sec. III-C and the
bulk cubes of the scaling study in Sec. III-E; no external data is used):
  plain    32x32x4 cells of 2 nm, random unit m
  film     512x128x1 cells of 3.9x3.9x3 nm, near-uniform m with noise, DMI
  bulk     512x512x16 cells of 2 nm, random m, 32x32x16 grains of random easy axis
  adjoint  128x128x1 cells of 2 nm, per-cell Ms map, DMI
  learned  64x64x4 cells of 2 nm, smooth random textures (Gaussian filter, 8 cells)
"""
import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def unit_random(shape, seed):
    """Unit vectors uniform on the sphere: normalised standard normal triples."""
    nz, ny, nx = shape
    return _unit(rng(seed).standard_normal((nz, ny, nx, 3)))


def near_uniform(shape, direction, noise, seed):
    """normalize(direction/|direction| + N(0, noise^2) per component)."""
    nz, ny, nx = shape
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return _unit(d + noise * rng(seed).standard_normal((nz, ny, nx, 3)))


def grain_axes(shape, grain, seed):
    """Per-cell easy axis, constant on axis-aligned blocks of ``grain`` = (gx, gy, gz)
    cells, each block's axis uniform on the sphere."""
    nz, ny, nx = shape
    gx, gy, gz = grain
    bz, by, bx = -(-nz // gz), -(-ny // gy), -(-nx // gx)
    axes = _unit(rng(seed).standard_normal((bz, by, bx, 3)))
    k = np.arange(nz) // gz
    j = np.arange(ny) // gy
    i = np.arange(nx) // gx
    return axes[np.ix_(k, j, i)].copy()


def uniform_map(shape, lo, hi, seed):
    return rng(seed).uniform(lo, hi, size=shape)


def smooth_texture(shape, sigma, seed):
    """White N(0,1) noise per component, periodic Gaussian filter of width
    ``sigma`` cells applied in Fourier space, then normalised per cell."""
    nz, ny, nx = shape
    w = rng(seed).standard_normal((3, nz, ny, nx))
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.fftfreq(nx)[None, None, :]
    g = np.exp(-2.0 * (np.pi * sigma) ** 2 * (kx ** 2 + ky ** 2 + kz ** 2))
    f = np.real(np.fft.ifftn(np.fft.fftn(w, axes=(1, 2, 3)) * g, axes=(1, 2, 3)))
    return _unit(np.moveaxis(f, 0, -1))


# Workload parameters (SI units).  "gamma" is gamma0 = mu0 |gamma| in m/(A s).
CONFIGS = {
    "plain": dict(nx=32, ny=32, nz=4, dx=2e-9, dy=2e-9, dz=2e-9, Ms=8.0e5, A=1.3e-11,
                  Ku=5e3, ku_axis=(0.0, 0.0, 1.0), D=0.0, dmi=False, alpha=0.5,
                  gamma=2.211e5, h_bias=(0.0, 0.0, 1e4), dt=1e-14, steps=200),
    "film": dict(nx=512, ny=128, nz=1, dx=3.9e-9, dy=3.9e-9, dz=3e-9, Ms=8.0e5, A=1.3e-11,
                 Ku=0.0, ku_axis=(0.0, 0.0, 1.0), D=1.5e-3, dmi=True, alpha=0.02,
                 gamma=2.211e5, h_bias=(-2.5e4, 4.3e3, 0.0), dt=5e-14, steps=20000),
    "bulk": dict(nx=512, ny=512, nz=16, dx=2e-9, dy=2e-9, dz=2e-9, Ms=1.1e6, A=1.5e-11,
                 Ku=4e5, ku_axis="grains", D=0.0, dmi=False, alpha=0.1,
                 gamma=2.211e5, h_bias=(0.0, 0.0, 0.0), dt=1e-14, steps=1000),
    "adjoint": dict(nx=128, ny=128, nz=1, dx=2e-9, dy=2e-9, dz=2e-9, Ms="map", A=1.3e-11,
                    Ku=0.0, ku_axis=(0.0, 0.0, 1.0), D=2e-3, dmi=True, alpha=0.3,
                    gamma=2.211e5, h_bias=(0.0, 0.0, 1e5), dt=2e-14, steps=2000),
    "learned": dict(nx=64, ny=64, nz=4, dx=2e-9, dy=2e-9, dz=2e-9, Ms=8.0e5, A=1.3e-11,
                    Ku=5e3, ku_axis=(0.0, 0.0, 1.0), D=0.0, dmi=False, alpha=0.5,
                    gamma=2.211e5, h_bias=(0.0, 0.0, 1e4), dt=1e-14, steps=5000),
}

SEEDS = {"plain": 1, "film": 2, "bulk": 3, "bulk_grains": 33, "adjoint": 4,
         "adjoint_ms": 44, "learned": 5000}


def initial_m(name, shape=None):
    c = CONFIGS[name]
    shape = shape or (c["nz"], c["ny"], c["nx"])
    if name == "film":
        return near_uniform(shape, (1.0, 0.25, 0.1), 0.01, SEEDS["film"])
    if name == "learned":
        return smooth_texture(shape, 8.0, SEEDS["learned"])
    return unit_random(shape, SEEDS[name])


def material(name, shape=None):
    """(Ms, Ku, ku_axis) for a workload; maps where the workload has them."""
    c = CONFIGS[name]
    shape = shape or (c["nz"], c["ny"], c["nx"])
    Ms = c["Ms"]
    if Ms == "map":
        Ms = uniform_map(shape, 6e5, 1e6, SEEDS["adjoint_ms"])
    axis = c["ku_axis"]
    if isinstance(axis, str):
        axis = grain_axes(shape, (32, 32, 16), SEEDS["bulk_grains"])
    return Ms, c["Ku"], axis
