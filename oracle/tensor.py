"""Oracle demag tensor: Python side of ``newell.c``.

TEST INFRASTRUCTURE ONLY (the plain FP64 CPU oracle; the product never
imports this package).

Paper Sec. II-B (FFT demag on a grid of twice the problem size, after
Nakatani et al. and Hayashi et al.) and the demag equation of Sec. II-A.
The tensor here follows the sign convention H_d(r_i) = -sum_j N(r_i - r_j) M_j,
so that a cube's self-term is 1/3 on each diagonal entry.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)

COMPONENTS = ("xx", "yy", "zz", "xy", "xz", "yz")
# Parity of each component under X -> -X, Y -> -Y, Z -> -Z: the diagonal ones
# are even in every axis; N_xy is odd in X and Y, even in Z, and so on.
PARITY = {
    "xx": (1, 1, 1), "yy": (1, 1, 1), "zz": (1, 1, 1),
    "xy": (-1, -1, 1), "xz": (-1, 1, -1), "yz": (1, -1, -1),
}


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        for fn in ("mxo_newell_f64", "mxo_tensor_at"):
            getattr(L, fn).argtypes = [_D] * 6 + [_PD]
            getattr(L, fn).restype = None
        L.mxo_newell_q.argtypes = [_D] * 6 + [_PD]
        L.mxo_newell_q.restype = ctypes.c_int
        L.mxo_quad_f64.argtypes = [_D] * 6 + [ctypes.c_int, _PD]
        L.mxo_quad_f64.restype = None
        L.mxo_tensor_octant.argtypes = [ctypes.c_int] * 3 + [_D] * 3 + [_PD]
        L.mxo_tensor_octant.restype = None
        L.mxo_has_quad.restype = ctypes.c_int
        L.mxo_set_switch.argtypes = [_D]
        L.mxo_get_switch.restype = _D
        _lib = L
    return _lib


def _call6(fn, *args):
    out = (_D * 6)()
    r = fn(*args, out)
    return np.array(out[:]), r


def newell_closed_form(X, Y, Z, dx, dy, dz):
    """Newell's closed form in double precision (all six components)."""
    return _call6(lib().mxo_newell_f64, X, Y, Z, dx, dy, dz)[0]


def newell_binary128(X, Y, Z, dx, dy, dz):
    """Newell's closed form in binary128 (None where unavailable)."""
    v, ok = _call6(lib().mxo_newell_q, X, Y, Z, dx, dy, dz)
    return v if ok else None


def quadrature(X, Y, Z, dx, dy, dz, n):
    """Gauss-Legendre quadrature of the defining integral, n points per half-axis."""
    out = (_D * 6)()
    lib().mxo_quad_f64(X, Y, Z, dx, dy, dz, int(n), out)
    return np.array(out[:])


def tensor_at(X, Y, Z, dx, dy, dz):
    """The oracle's tensor at one offset (closed form near, quadrature far)."""
    return _call6(lib().mxo_tensor_at, X, Y, Z, dx, dy, dz)[0]


def has_binary128():
    return bool(lib().mxo_has_quad())


def tensor_octant(nx, ny, nz, dx, dy, dz):
    """Tensor at offsets (i dx, j dy, k dz), 0 <= i < nx etc.

    Returns an array of shape (6, nz, ny, nx), components xx,yy,zz,xy,xz,yz.
    """
    out = np.empty((6, nz, ny, nx), dtype=np.float64)
    lib().mxo_tensor_octant(int(nx), int(ny), int(nz), float(dx), float(dy), float(dz),
                            out.ctypes.data_as(_PD))
    return out


def tensor_full(nx, ny, nz, dx, dy, dz):
    """Tensor on all signed offsets -(n-1)..(n-1) per axis.

    Shape (6, 2nz-1, 2ny-1, 2nx-1); index [c, Z + nz - 1, Y + ny - 1, X + nx - 1].
    Built from the octant with each component's parity in X, Y and Z.
    """
    oc = tensor_octant(nx, ny, nz, dx, dy, dz)
    full = np.zeros((6, 2 * nz - 1, 2 * ny - 1, 2 * nx - 1))
    ix = np.abs(np.arange(-(nx - 1), nx))
    iy = np.abs(np.arange(-(ny - 1), ny))
    iz = np.abs(np.arange(-(nz - 1), nz))
    sx = np.sign(np.arange(-(nx - 1), nx)) + (np.arange(-(nx - 1), nx) == 0)
    sy = np.sign(np.arange(-(ny - 1), ny)) + (np.arange(-(ny - 1), ny) == 0)
    sz = np.sign(np.arange(-(nz - 1), nz)) + (np.arange(-(nz - 1), nz) == 0)
    for c, name in enumerate(COMPONENTS):
        px, py, pz = PARITY[name]
        block = oc[c][np.ix_(iz, iy, ix)]
        fx = sx if px < 0 else np.ones_like(sx)
        fy = sy if py < 0 else np.ones_like(sy)
        fz = sz if pz < 0 else np.ones_like(sz)
        full[c] = block * fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
    return full
