"""Context object over the C ABI (argument marshalling only).

``Context`` owns one ``mx_ctx`` and exposes the entry points of include/mx.h
as methods on torch CUDA tensors.  No arithmetic of the method happens here.
"""
import numpy as np
import torch

from . import _lib as L


def to_dev4(a, device="cuda"):
    """(nz, ny, nx, 3) array -> contiguous float32 CUDA tensor (nz, ny, nx, 4)."""
    a = torch.as_tensor(np.asarray(a, dtype=np.float32))
    out = torch.zeros(a.shape[:-1] + (4,), dtype=torch.float32)
    out[..., :3] = a
    return out.to(device).contiguous()


def from_dev4(t):
    """(nz, ny, nx, 4) CUDA tensor -> (nz, ny, nx, 3) float64 numpy array."""
    return t[..., :3].double().cpu().numpy()


def save_state(path, m, t=0.0, step=0, meta=None):
    """Checkpoint of a run: the xyz of the float4 field m (any device; the
    FP32 values are stored exactly; the w slot, which mx_rk_step does not
    read, is not kept), the simulated time t [s], the step count and a
    JSON-serialisable dict of run metadata, in one .npz file."""
    import json
    np.savez(path, m=m[..., :3].float().cpu().numpy(), t=np.float64(t), step=np.int64(step),
             meta=np.array(json.dumps(meta or {})))


def load_state(path, device="cuda"):
    """(m, t, step, meta) from save_state; m as a float4 tensor on `device`."""
    import json
    with np.load(path) as d:
        m = to_dev4(d["m"], device)
        return m, float(d["t"]), int(d["step"]), json.loads(str(d["meta"]))


_METHODS = {"rk4": L.MX_RK4, "euler": L.MX_EULER, "mri": L.MX_MRI}


class Context:
    """One simulation grid: parameters, demag kernel and workspaces on one GPU."""

    def __init__(self, nx, ny, nz, dx, dy, dz, Ms=8e5, A=1.3e-11, Ku=0.0, D=0.0, alpha=0.5,
                 gamma=2.211e5, ku_axis=(0.0, 0.0, 1.0), h_bias=(0.0, 0.0, 0.0), dmi=False,
                 precession=True, demag=True, demag_path=0, fft_mode=0, mri_fast_ratio=0.0, build=True,
                 stream=None):
        p = L.mx_params()
        p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
        p.dx, p.dy, p.dz = float(dx), float(dy), float(dz)
        p.Ms, p.A, p.Ku, p.D = float(Ms), float(A), float(Ku), float(D)
        p.alpha, p.gamma = float(alpha), float(gamma)
        p.ku_axis[:] = [float(v) for v in ku_axis]
        p.h_bias[:] = [float(v) for v in h_bias]
        p.dmi_interfacial, p.precession, p.demag = int(bool(dmi)), int(bool(precession)), int(bool(demag))
        p.demag_path = int(demag_path)
        p.fft_mode = int(fft_mode)
        p.mri_fast_ratio = float(mri_fast_ratio)
        self.params = p
        self.shape = (int(nz), int(ny), int(nx))
        self.h = None
        self.h = L.mx_create(p)
        if build and demag:
            self.build_demag_kernel(stream)

    @classmethod
    def from_config(cls, cfg, Ms=None, Ku=None, ku_axis=None, **kw):
        c = dict(cfg)
        ms = c["Ms"] if Ms is None else Ms
        axis = c["ku_axis"] if ku_axis is None else ku_axis
        ms_scalar = float(ms) if np.isscalar(ms) else float(np.mean(ms))
        axis_scalar = axis if (not isinstance(axis, np.ndarray) or axis.ndim == 1) else (0.0, 0.0, 1.0)
        ku = c["Ku"] if Ku is None else Ku
        ku_scalar = float(ku) if np.isscalar(ku) else 0.0
        ctx = cls(c["nx"], c["ny"], c["nz"], c["dx"], c["dy"], c["dz"], Ms=ms_scalar, A=c["A"], Ku=ku_scalar,
                  D=c["D"], alpha=c["alpha"], gamma=c["gamma"], ku_axis=axis_scalar, h_bias=c["h_bias"],
                  dmi=c["dmi"], build=False, **kw)
        if not np.isscalar(ms):
            ctx.set_ms_map(torch.as_tensor(np.asarray(ms, np.float32)).cuda())
        ku_map = None if np.isscalar(ku) else torch.as_tensor(np.asarray(ku, np.float32)).cuda()
        ax_map = None
        if isinstance(axis, np.ndarray) and axis.ndim > 1:
            ax_map = to_dev4(axis)
        if ku_map is not None or ax_map is not None:
            # a scalar Ku stays scalar (the library reads p.Ku where no Ku map is set)
            ctx.set_anis_map(ku_map, ax_map)
        if ctx.params.demag:
            ctx.build_demag_kernel()
        return ctx

    def close(self):
        if self.h is not None:
            L.mx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- setup ---------------------------------------------------------------
    def build_demag_kernel(self, stream=None):
        L.mx_build_demag_kernel(self.h, stream)

    def _check_map(self, t, rec):
        """A per-cell map: contiguous CUDA float32 of shape (nz, ny, nx) (+ (4,) for float4 records)."""
        shape = self.shape + rec
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != shape:
            raise ValueError(f"expected contiguous CUDA float32 tensor of shape {shape}")

    def set_ms_map(self, ms, stream=None):
        if ms is not None:
            ms = ms.contiguous()
            self._check_map(ms, ())
        L.mx_set_ms_map(self.h, ms, stream)
        if stream is None:
            torch.cuda.current_stream().synchronize()

    def set_anis_map(self, ku, axis, stream=None):
        if ku is not None:
            ku = ku.contiguous()
            self._check_map(ku, ())
        if axis is not None:
            axis = axis.contiguous()
            self._check_map(axis, (4,))
        L.mx_set_anis_map(self.h, ku, axis, stream)
        if stream is None:
            torch.cuda.current_stream().synchronize()

    def set_bias(self, h):
        L.mx_set_bias(self.h, h)

    @property
    def padded_dims(self):
        return L.mx_padded_dims(self.h)

    # -- hot path ------------------------------------------------------------
    def _check(self, t):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != self.shape + (4,):
            raise ValueError(f"expected contiguous CUDA float32 tensor of shape {self.shape + (4,)}")

    def heff(self, m, out=None, terms=L.MX_TERM_ALL, stream=None):
        self._check(m)
        out = torch.empty_like(m) if out is None else out
        self._check(out)
        L.mx_heff(self.h, m, out, terms, stream)
        return out

    def llg_rhs(self, m, out=None, stream=None):
        self._check(m)
        out = torch.empty_like(m) if out is None else out
        self._check(out)
        L.mx_llg_rhs(self.h, m, out, stream)
        return out

    def rk_step(self, m, nsteps, dt, method="rk4", stream=None):
        self._check(m)
        L.mx_rk_step(self.h, m, nsteps, dt, _METHODS[method], stream)
        return m

    def energy(self, m, stream=None):
        self._check(m)
        e = L.mx_energy(self.h, m, stream)
        return dict(zip(("demag", "exch", "anis", "dmi", "zeeman"), e))

    def exchange_energy_central(self, m, stream=None):
        """Exchange energy with central-difference gradients (the tabulated form)."""
        self._check(m)
        return L.mx_exchange_energy_central(self.h, m, stream)

    def sync(self, stream=None):
        L.mx_sync(self.h, stream)

    def demag_tensor_real(self):
        nz, ny, nx = self.shape
        out = torch.empty((6, nz, ny, nx), dtype=torch.float64, device="cuda")
        L.mx_demag_tensor_real(self.h, out)
        torch.cuda.current_stream().synchronize()
        return out

    def demag_spectrum(self):
        Px, Py, Pz = self.padded_dims
        Hx = Px // 2 + 1 if Px > 1 else 1
        out = torch.empty((6, Pz // 2 + 1, Py // 2 + 1, Hx), dtype=torch.float32, device="cuda")
        L.mx_demag_spectrum(self.h, out)
        torch.cuda.current_stream().synchronize()
        return out

    def kernel_names(self):
        """{timing slot: the kernel this context launches in it}."""
        return L.mx_kernel_names(self.h)

    def kernel_name(self, slot):
        """The kernel launched in timing slot `slot` (an index or a slot name)."""
        names = self.kernel_names()
        if isinstance(slot, int):
            slot = list(names)[slot]
        return names[slot]

    def profile_step(self, m, nsteps, dt, method="rk4", stream=None):
        self._check(m)
        return L.mx_profile_step(self.h, m, nsteps, dt, _METHODS[method], stream)

    # -- adjoint ---------------------------------------------------------------
    def adjoint_reserve(self, nsteps, checkpoint_every):
        L.mx_adjoint_reserve(self.h, nsteps, checkpoint_every)
        self._adj = (int(nsteps), int(checkpoint_every))

    def rk_forward_record(self, m0_raw, dt, stream=None):
        self._check(m0_raw)
        out = torch.empty_like(m0_raw)
        L.mx_rk_forward_record(self.h, m0_raw, out, dt, stream)
        return out

    def rk_backward(self, lam_final, want_ms=True, stream=None):
        self._check(lam_final)
        g = torch.empty_like(lam_final)
        gms = torch.empty(self.shape, dtype=torch.float32, device=lam_final.device) if want_ms else None
        L.mx_rk_backward(self.h, lam_final.contiguous(), g, gms, stream)
        return g, gms
