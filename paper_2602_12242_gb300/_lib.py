"""ctypes binding of libmx (include/mx.h): argument marshalling only.

Every computation runs in the CUDA library; this module only converts
arguments.  Loading fails loudly if ``_build/libmx.so`` is missing: there is
no CPU fallback.

Field tensors are torch CUDA float32 tensors of shape (nz, ny, nx, 4),
contiguous (x, y, z, unused per cell); scalar maps are (nz, ny, nx) float32.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmx.so")

MX_OK, MX_ERR_INVALID_ARG, MX_ERR_CUDA, MX_ERR_OOM, MX_ERR_NOT_BUILT, MX_ERR_NONFINITE, MX_ERR_TIMEOUT, \
    MX_ERR_UNSUPPORTED = range(8)
STATUS_NAMES = {0: "MX_OK", 1: "MX_ERR_INVALID_ARG", 2: "MX_ERR_CUDA", 3: "MX_ERR_OOM", 4: "MX_ERR_NOT_BUILT",
                5: "MX_ERR_NONFINITE", 6: "MX_ERR_TIMEOUT", 7: "MX_ERR_UNSUPPORTED"}
MX_TERM_DEMAG, MX_TERM_EXCH, MX_TERM_ANIS, MX_TERM_DMI, MX_TERM_ZEEMAN = 1, 2, 4, 8, 16
MX_TERM_ALL = 31
MX_RK4, MX_EULER, MX_MRI = 0, 1, 2
MX_DEMAG_AUTO, MX_DEMAG_GENERIC, MX_DEMAG_PLANE, MX_DEMAG_PLANE_PAIR, MX_DEMAG_PLANE_XLOCAL = 0, 1, 2, 3, 4
MX_FFT_FP32, MX_FFT_SPLIT_BF16 = 0, 1


class MxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class mx_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("Ms", ctypes.c_double), ("A", ctypes.c_double), ("Ku", ctypes.c_double),
                ("D", ctypes.c_double), ("alpha", ctypes.c_double), ("gamma", ctypes.c_double),
                ("ku_axis", ctypes.c_double * 3), ("h_bias", ctypes.c_double * 3),
                ("dmi_interfacial", ctypes.c_int), ("precession", ctypes.c_int), ("demag", ctypes.c_int),
                ("demag_path", ctypes.c_int), ("fft_mode", ctypes.c_int), ("mri_fast_ratio", ctypes.c_double)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
# name -> (restype, argtypes)
SIGNATURES = {
    "mx_last_error": (ctypes.c_char_p, []),
    "mx_version": (ctypes.c_char_p, []),
    "mx_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(mx_params)]),
    "mx_destroy": (_I, [_P]),
    "mx_set_ms_map": (_I, [_P, _P, _P]),
    "mx_set_anis_map": (_I, [_P, _P, _P, _P]),
    "mx_set_bias": (_I, [_P, ctypes.POINTER(_D)]),
    "mx_build_demag_kernel": (_I, [_P, _P]),
    "mx_heff": (_I, [_P, _P, _P, _I, _P]),
    "mx_llg_rhs": (_I, [_P, _P, _P, _P]),
    "mx_rk_step": (_I, [_P, _P, _I, _D, _I, _P]),
    "mx_energy": (_I, [_P, _P, ctypes.POINTER(_D), _P]),
    "mx_exchange_energy_central": (_I, [_P, _P, ctypes.POINTER(_D), _P]),
    "mx_sync": (_I, [_P, _P]),
    "mx_padded_dims": (_I, [_P, ctypes.POINTER(_I)]),
    "mx_demag_tensor_real": (_I, [_P, _P, _P]),
    "mx_demag_spectrum": (_I, [_P, _P, _P]),
    "mx_profile_step": (_I, [_P, _P, _I, _D, _I, _P, ctypes.POINTER(_D), ctypes.POINTER(_I), _I,
                             ctypes.POINTER(_I)]),
    "mx_kernel_slot": (ctypes.c_char_p, [_I]),
    "mx_inject_wait_timeout": (_I, [_P, _I]),
    "mx_kernel_name": (ctypes.c_char_p, [_P, _I]),
    "mx_energy_noalloc": (_I, [ctypes.POINTER(mx_params), _P, _P, _P, _P, _P, _P, _P]),
    "mx_cnn_num_params": (_I, []),
    "mx_cnn_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I]),
    "mx_cnn_destroy": (_I, [_P]),
    "mx_cnn_set_params": (_I, [_P, _P, _P]),
    "mx_cnn_get_params": (_I, [_P, _P, _P]),
    "mx_cnn_set_normalizer": (_I, [_P, ctypes.POINTER(_D)]),
    "mx_cnn_forward": (_I, [_P, _P, _P, _I, _P]),
    "mx_cnn_loss_grad": (_I, [_P, _P, _P, _I, _P, _P, _P]),
    "mx_cnn_sync": (_I, [_P, _P]),
    "mx_cnn_adam_step": (_I, [_P, _D, _D, _P]),
    "mx_set_demag_surrogate": (_I, [_P, _P]),
    "mx_fno_num_params": (_I, [_I]),
    "mx_fno_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _I]),
    "mx_fno_destroy": (_I, [_P]),
    "mx_fno_set_params": (_I, [_P, _P, _P]),
    "mx_fno_get_params": (_I, [_P, _P, _P]),
    "mx_fno_set_normalizer": (_I, [_P, ctypes.POINTER(_D)]),
    "mx_fno_forward": (_I, [_P, _P, _P, _I, _P]),
    "mx_fno_loss_grad": (_I, [_P, _P, _P, _I, _P, _P, _P]),
    "mx_fno_adam_step": (_I, [_P, _D, _D, _P]),
    "mx_set_demag_fno": (_I, [_P, _P]),
    "mx_rel_l2": (_I, [_P, _P, _P, ctypes.POINTER(_D), _P]),
    "mx_adjoint_reserve": (_I, [_P, _I, _I]),
    "mx_rk_forward_record": (_I, [_P, _P, _P, _D, _P]),
    "mx_rk_backward": (_I, [_P, _P, _P, _P, _P]),
}

_lib = None


def lib():
    """Load libmx.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libmx.so not found at {LIB_PATH}: run __graft_entry__.build() "
                              "(the CUDA library is required; there is no CPU path)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status):
    if status != MX_OK:
        raise MxError(status, lib().mx_last_error().decode())


def ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ----------------------------------------------------------------------------
# Functions with the C names.
# ----------------------------------------------------------------------------

def mx_create(params):
    h = ctypes.c_void_p()
    check(lib().mx_create(ctypes.byref(h), ctypes.byref(params)))
    return h


def mx_destroy(ctx):
    check(lib().mx_destroy(ctx))


def mx_set_ms_map(ctx, ms, stream=None):
    check(lib().mx_set_ms_map(ctx, ptr(ms), stream_handle(stream)))


def mx_set_anis_map(ctx, ku, axis, stream=None):
    check(lib().mx_set_anis_map(ctx, ptr(ku), ptr(axis), stream_handle(stream)))


def mx_set_bias(ctx, h):
    arr = (_D * 3)(*[float(v) for v in h])
    check(lib().mx_set_bias(ctx, arr))


def mx_build_demag_kernel(ctx, stream=None):
    check(lib().mx_build_demag_kernel(ctx, stream_handle(stream)))


def mx_heff(ctx, m, h, terms=MX_TERM_ALL, stream=None):
    check(lib().mx_heff(ctx, ptr(m), ptr(h), int(terms), stream_handle(stream)))


def mx_llg_rhs(ctx, m, dmdt, stream=None):
    check(lib().mx_llg_rhs(ctx, ptr(m), ptr(dmdt), stream_handle(stream)))


def mx_rk_step(ctx, m, nsteps, dt, method=MX_RK4, stream=None):
    check(lib().mx_rk_step(ctx, ptr(m), int(nsteps), float(dt), int(method), stream_handle(stream)))


def mx_energy(ctx, m, stream=None):
    out = (_D * 5)()
    check(lib().mx_energy(ctx, ptr(m), out, stream_handle(stream)))
    return list(out)


def mx_exchange_energy_central(ctx, m, stream=None):
    out = _D()
    check(lib().mx_exchange_energy_central(ctx, ptr(m), ctypes.byref(out), stream_handle(stream)))
    return out.value


def mx_sync(ctx, stream=None):
    check(lib().mx_sync(ctx, stream_handle(stream)))


def mx_padded_dims(ctx):
    out = (_I * 3)()
    check(lib().mx_padded_dims(ctx, out))
    return tuple(out)


def mx_demag_tensor_real(ctx, out, stream=None):
    check(lib().mx_demag_tensor_real(ctx, ptr(out), stream_handle(stream)))


def mx_demag_spectrum(ctx, out, stream=None):
    check(lib().mx_demag_spectrum(ctx, ptr(out), stream_handle(stream)))


def mx_profile_step(ctx, m, nsteps, dt, method=MX_RK4, stream=None, max_kernels=32):
    ms = (_D * max_kernels)()
    cnt = (_I * max_kernels)()
    n = _I()
    check(lib().mx_profile_step(ctx, ptr(m), int(nsteps), float(dt), int(method), stream_handle(stream),
                                ms, cnt, max_kernels, ctypes.byref(n)))
    return {lib().mx_kernel_slot(q).decode(): (ms[q], cnt[q]) for q in range(n.value) if cnt[q] > 0}


def mx_inject_wait_timeout(ctx, on):
    check(lib().mx_inject_wait_timeout(ctx, int(bool(on))))


def mx_kernel_names(ctx, max_kernels=32):
    """{slot: kernel this context launches in it} for every timing slot."""
    out, q = {}, 0
    while q < max_kernels:
        slot = lib().mx_kernel_slot(q).decode()
        if not slot:
            break
        out[slot] = lib().mx_kernel_name(ctx, q).decode()
        q += 1
    return out


def mx_adjoint_reserve(ctx, nsteps, checkpoint_every):
    check(lib().mx_adjoint_reserve(ctx, int(nsteps), int(checkpoint_every)))


def mx_rk_forward_record(ctx, m0_raw, m_final, dt, stream=None):
    check(lib().mx_rk_forward_record(ctx, ptr(m0_raw), ptr(m_final), float(dt), stream_handle(stream)))


def mx_rk_backward(ctx, lam_final, grad_m0, grad_ms=None, stream=None):
    check(lib().mx_rk_backward(ctx, ptr(lam_final), ptr(grad_m0), ptr(grad_ms), stream_handle(stream)))


def mx_energy_noalloc(params, m, e_out, h_demag=None, ms_map=None, ku_map=None, axis_map=None, stream=None):
    """Energies into the caller's DEVICE buffer e_out (5 float64) without any
    device allocation inside the library (see include/mx.h)."""
    check(lib().mx_energy_noalloc(ctypes.byref(params), ptr(m), ptr(h_demag), ptr(ms_map), ptr(ku_map),
                                  ptr(axis_map), ptr(e_out), stream_handle(stream)))


def mx_cnn_num_params():
    return int(lib().mx_cnn_num_params())


def mx_cnn_create(nx, ny, nz, max_batch):
    h = ctypes.c_void_p()
    check(lib().mx_cnn_create(ctypes.byref(h), int(nx), int(ny), int(nz), int(max_batch)))
    return h


def mx_cnn_destroy(net):
    check(lib().mx_cnn_destroy(net))


def mx_cnn_set_params(net, params, stream=None):
    check(lib().mx_cnn_set_params(net, ptr(params), stream_handle(stream)))


def mx_cnn_get_params(net, params, stream=None):
    check(lib().mx_cnn_get_params(net, ptr(params), stream_handle(stream)))


def mx_cnn_set_normalizer(net, stats):
    arr = (_D * 12)(*[float(v) for v in stats])
    check(lib().mx_cnn_set_normalizer(net, arr))


def mx_cnn_forward(net, m, h, batch, stream=None):
    check(lib().mx_cnn_forward(net, ptr(m), ptr(h), int(batch), stream_handle(stream)))


def mx_cnn_loss_grad(net, m, h_target, batch, loss_out=None, grad_out=None, stream=None):
    check(lib().mx_cnn_loss_grad(net, ptr(m), ptr(h_target), int(batch), ptr(loss_out), ptr(grad_out),
                                 stream_handle(stream)))


def mx_cnn_sync(net, stream=None):
    check(lib().mx_cnn_sync(net, stream_handle(stream)))


def mx_cnn_adam_step(net, lr, weight_decay, stream=None):
    check(lib().mx_cnn_adam_step(net, float(lr), float(weight_decay), stream_handle(stream)))


def mx_set_demag_surrogate(ctx, net):
    check(lib().mx_set_demag_surrogate(ctx, net))


def mx_fno_num_params(modes):
    return int(lib().mx_fno_num_params(int(modes)))


def mx_fno_create(nx, ny, modes, max_batch):
    h = _P()
    check(lib().mx_fno_create(ctypes.byref(h), int(nx), int(ny), int(modes), int(max_batch)))
    return h


def mx_fno_destroy(net):
    check(lib().mx_fno_destroy(net))


def mx_fno_set_params(net, params, stream=None):
    check(lib().mx_fno_set_params(net, ptr(params), stream_handle(stream)))


def mx_fno_get_params(net, params, stream=None):
    check(lib().mx_fno_get_params(net, ptr(params), stream_handle(stream)))


def mx_fno_set_normalizer(net, stats):
    arr = (_D * 12)(*[float(v) for v in stats])
    check(lib().mx_fno_set_normalizer(net, arr))


def mx_fno_forward(net, m, h, batch, stream=None):
    check(lib().mx_fno_forward(net, ptr(m), ptr(h), int(batch), stream_handle(stream)))


def mx_fno_loss_grad(net, m, h_target, batch, loss_out=None, grad_out=None, stream=None):
    check(lib().mx_fno_loss_grad(net, ptr(m), ptr(h_target), int(batch), ptr(loss_out), ptr(grad_out),
                                 stream_handle(stream)))


def mx_fno_adam_step(net, lr, weight_decay, stream=None):
    check(lib().mx_fno_adam_step(net, float(lr), float(weight_decay), stream_handle(stream)))


def mx_set_demag_fno(ctx, net):
    check(lib().mx_set_demag_fno(ctx, net))


def mx_rel_l2(ctx, a, b, stream=None):
    out = _D()
    check(lib().mx_rel_l2(ctx, ptr(a), ptr(b), ctypes.byref(out), stream_handle(stream)))
    return out.value
