"""mx_create's argument checks, which return before any device call (CPU only):
empty and oversized grids, non-physical parameters, unknown options."""
import ctypes
import math

import pytest


@pytest.fixture(scope="module")
def L():
    from paper_2602_12242_gb300 import _lib, build
    build.build()
    return _lib


def params(L, **kw):
    p = L.mx_params()
    base = dict(nx=8, ny=8, nz=2, dx=2e-9, dy=2e-9, dz=2e-9, Ms=8e5, A=1.3e-11, Ku=0.0, D=0.0, alpha=0.5,
                gamma=2.211e5, dmi_interfacial=0, precession=1, demag=1)
    base.update(kw)
    for k, v in base.items():
        setattr(p, k, v)
    return p


CASES = [
    ("empty x", dict(nx=0), "MX_ERR_UNSUPPORTED"),
    ("empty z", dict(nz=0), "MX_ERR_UNSUPPORTED"),
    ("negative y", dict(ny=-3), "MX_ERR_UNSUPPORTED"),
    ("over 2048 cells", dict(nx=2049), "MX_ERR_UNSUPPORTED"),
    ("zero cell size", dict(dy=0.0), "MX_ERR_INVALID_ARG"),
    ("zero Ms", dict(Ms=0.0), "MX_ERR_INVALID_ARG"),
    ("negative A", dict(A=-1e-11), "MX_ERR_INVALID_ARG"),
    ("negative alpha", dict(alpha=-0.1), "MX_ERR_INVALID_ARG"),
    ("zero gamma", dict(gamma=0.0), "MX_ERR_INVALID_ARG"),
    ("NaN Ku", dict(Ku=math.nan), "MX_ERR_INVALID_ARG"),
    ("NaN D", dict(D=math.nan), "MX_ERR_INVALID_ARG"),
    ("chiral boundary without exchange", dict(dmi_interfacial=1, D=1e-3, A=0.0), "MX_ERR_INVALID_ARG"),
    ("demag path", dict(demag_path=7), "MX_ERR_INVALID_ARG"),
    ("fft mode", dict(fft_mode=9), "MX_ERR_INVALID_ARG"),
    ("MRI ratio above 1", dict(mri_fast_ratio=1.5), "MX_ERR_INVALID_ARG"),
    ("MRI ratio NaN", dict(mri_fast_ratio=math.nan), "MX_ERR_INVALID_ARG"),
]


@pytest.mark.parametrize("name,kw,status", CASES, ids=[c[0] for c in CASES])
def test_create_refuses(L, name, kw, status):
    h = ctypes.c_void_p()
    got = L.lib().mx_create(ctypes.byref(h), ctypes.byref(params(L, **kw)))
    assert got == getattr(L, status), (name, got, L.lib().mx_last_error())
    assert not h.value
    assert L.lib().mx_last_error()


NOALLOC_CASES = [
    ("axis far beyond 2048", dict(nx=1 << 22, ny=1 << 22, nz=1 << 22), {}, "MX_ERR_UNSUPPORTED"),
    ("one axis over 2048", dict(nx=4096, ny=1, nz=1), {}, "MX_ERR_UNSUPPORTED"),
    ("cells over the scratch limit", dict(nx=2048, ny=2048, nz=2), {}, "MX_ERR_UNSUPPORTED"),
    ("empty grid", dict(nx=0), {}, "MX_ERR_UNSUPPORTED"),
    ("zero Ms", dict(Ms=0.0), {}, "MX_ERR_INVALID_ARG"),
    ("misaligned Ms map", {}, dict(ms_map=2), "MX_ERR_INVALID_ARG"),
    ("misaligned Ku map", {}, dict(ku_map=1), "MX_ERR_INVALID_ARG"),
    ("misaligned m", {}, dict(m=8), "MX_ERR_INVALID_ARG"),
    ("NULL m", {}, dict(m=None), "MX_ERR_INVALID_ARG"),
]


@pytest.mark.parametrize("name,kw,ptrs,status", NOALLOC_CASES, ids=[c[0] for c in NOALLOC_CASES])
def test_energy_noalloc_refuses_before_any_device_call(L, name, kw, ptrs, status):
    """mx_energy_noalloc's checks use no device: host buffers stand in for the
    device pointers (never dereferenced), offsets make them misaligned."""
    buf = (ctypes.c_double * 64)()
    base = ctypes.addressof(buf)
    base += (-base) % 16

    def at(off):
        return ctypes.c_void_p(None if off is None else base + off)

    args = dict(m=0, h_demag=None, ms_map=None, ku_map=None, axis_map=None)
    args.update(ptrs)
    p = params(L, **kw)
    got = L.lib().mx_energy_noalloc(ctypes.byref(p), at(args["m"]), at(args["h_demag"]), at(args["ms_map"]),
                                    at(args["ku_map"]), at(args["axis_map"]), at(256), ctypes.c_void_p(None))
    assert got == getattr(L, status), (name, got, L.lib().mx_last_error())
    assert L.lib().mx_last_error()


def test_wait_timeout_hook_refuses_a_null_context(L):
    assert L.lib().mx_inject_wait_timeout(ctypes.c_void_p(None), 1) == L.MX_ERR_INVALID_ARG
