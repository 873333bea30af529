"""Learned demag surrogate: network handle, dataset, training loop and the
in-loop driver with the FFT demag as judge and fallback.

All arithmetic of the networks (forward, loss, backward, Adam) and of the
micromagnetic path runs in libmx (mx_cnn_*, mx_fno_*, mx_heff, mx_rk_step,
mx_rel_l2);
this module only moves tensors, draws seeded inputs and runs the control flow
of training (batching, learning-rate schedule) and of the judge.
"""
import time

import numpy as np
import torch

from . import _lib as L
from . import inputs
from .solver import to_dev4


CHANNELS = (3, 32, 64, 32, 3)


def _fields(shape, max_batch, *ts):
    """Batch size of float4 field tensors of one grid (nz, ny, nx): (B, nz, ny,
    nx, 4) or one (nz, ny, nx, 4) field; contiguous CUDA float32, 1 <= B <=
    max_batch.  The library takes plain pointers, so the sizes are checked here."""
    one = tuple(shape) + (4,)
    b = None
    for t in ts:
        ok = t.dtype == torch.float32 and t.is_cuda and t.is_contiguous()
        tb = 1 if tuple(t.shape) == one else (t.shape[0] if t.dim() == 5 and tuple(t.shape[1:]) == one else None)
        if not ok or tb is None or (b is not None and tb != b) or not 1 <= tb <= max_batch:
            raise ValueError(f"expected contiguous CUDA float32 fields of shape (B,) + {one}, 1 <= B <= {max_batch}")
        b = tb
    return b


def init_params(seed):
    """Seeded initial parameters: each layer's weights and biases uniform in
    +-1/sqrt(fan_in) (fan_in = 27 * input channels), in the library's order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for l in range(4):
        cin, cout = CHANNELS[l], CHANNELS[l + 1]
        bound = 1.0 / np.sqrt(cin * 27)
        parts.append(rng.uniform(-bound, bound, size=cout * cin * 27))
        parts.append(rng.uniform(-bound, bound, size=cout))
    return np.concatenate(parts).astype(np.float32)


class Surrogate:
    """The 3 -> 32 -> 64 -> 32 -> 3 conv net of libmx for one grid."""

    def __init__(self, nx, ny, nz, max_batch=1):
        self.shape = (int(nz), int(ny), int(nx))
        self.max_batch = int(max_batch)
        self.h = None
        self.h = L.mx_cnn_create(nx, ny, nz, max_batch)
        self.n_params = L.mx_cnn_num_params()

    def close(self):
        if self.h is not None:
            L.mx_cnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        flat = torch.as_tensor(flat, dtype=torch.float32, device="cuda").contiguous()
        assert flat.numel() == self.n_params
        L.mx_cnn_set_params(self.h, flat)

    def get_params(self):
        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        L.mx_cnn_get_params(self.h, out)
        torch.cuda.current_stream().synchronize()
        return out

    def set_normalizer(self, stats):
        self.stats = [float(v) for v in stats]
        L.mx_cnn_set_normalizer(self.h, self.stats)

    def forward(self, m):
        m = m.contiguous()
        b = _fields(self.shape, self.max_batch, m)
        h = torch.empty_like(m)
        L.mx_cnn_forward(self.h, m, h, b)
        return h

    def loss_grad(self, m, h_target, want_grad=True):
        m, h_target = m.contiguous(), h_target.contiguous()
        b = _fields(self.shape, self.max_batch, m, h_target)
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        grad = torch.empty(self.n_params, dtype=torch.float32, device="cuda") if want_grad else None
        L.mx_cnn_loss_grad(self.h, m, h_target, b, loss, grad)
        return loss, grad

    def adam_step(self, lr, weight_decay):
        L.mx_cnn_adam_step(self.h, lr, weight_decay)

    def forward_into(self, m, h, batch):
        if _fields(self.shape, self.max_batch, m, h) < batch:
            raise ValueError("batch larger than the tensors")
        L.mx_cnn_forward(self.h, m, h, batch)

    def attach(self, ctx_h):
        """Make this net the demag backend of a context (None: detach)."""
        L.mx_set_demag_surrogate(ctx_h, self.h)

    @staticmethod
    def detach(ctx_h):
        L.mx_set_demag_surrogate(ctx_h, None)


def init_fno_params(modes, seed):
    """Seeded initial parameters of the Fourier neural operator, in the
    library's order: pointwise weights and biases uniform in +-1/sqrt(fan_in),
    spectral filters (real and imaginary parts) uniform in [0, 1/(32*32))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []

    def lin(cout, cin):
        bound = 1.0 / np.sqrt(cin)
        parts.append(rng.uniform(-bound, bound, size=cout * cin))
        parts.append(rng.uniform(-bound, bound, size=cout))

    lin(32, 3)
    for _ in range(4):
        parts.append(rng.uniform(0.0, 1.0 / (32 * 32), size=2 * modes * modes * 32 * 32 * 2))
        lin(32, 32)
    lin(128, 32)
    lin(3, 128)
    return np.concatenate(parts).astype(np.float32)


class FourierSurrogate:
    """The 2D Fourier neural operator of libmx for one film grid (nz = 1)."""

    def __init__(self, nx, ny, modes=12, max_batch=1):
        self.shape = (1, int(ny), int(nx))
        self.modes = int(modes)
        self.max_batch = int(max_batch)
        self.h = None
        self.h = L.mx_fno_create(nx, ny, modes, max_batch)
        self.n_params = L.mx_fno_num_params(modes)

    def close(self):
        if self.h is not None:
            L.mx_fno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        flat = torch.as_tensor(flat, dtype=torch.float32, device="cuda").contiguous()
        assert flat.numel() == self.n_params
        L.mx_fno_set_params(self.h, flat)

    def get_params(self):
        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        L.mx_fno_get_params(self.h, out)
        torch.cuda.current_stream().synchronize()
        return out

    def set_normalizer(self, stats):
        self.stats = [float(v) for v in stats]
        L.mx_fno_set_normalizer(self.h, self.stats)

    def forward(self, m):
        m = m.contiguous()
        b = _fields(self.shape, self.max_batch, m)
        h = torch.empty_like(m)
        L.mx_fno_forward(self.h, m, h, b)
        return h

    def forward_into(self, m, h, batch):
        if _fields(self.shape, self.max_batch, m, h) < batch:
            raise ValueError("batch larger than the tensors")
        L.mx_fno_forward(self.h, m, h, batch)

    def loss_grad(self, m, h_target, want_grad=True):
        m, h_target = m.contiguous(), h_target.contiguous()
        b = _fields(self.shape, self.max_batch, m, h_target)
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        grad = torch.empty(self.n_params, dtype=torch.float32, device="cuda") if want_grad else None
        L.mx_fno_loss_grad(self.h, m, h_target, b, loss, grad)
        return loss, grad

    def adam_step(self, lr, weight_decay):
        L.mx_fno_adam_step(self.h, lr, weight_decay)

    def attach(self, ctx_h):
        L.mx_set_demag_fno(ctx_h, self.h)

    @staticmethod
    def detach(ctx_h):
        L.mx_set_demag_fno(ctx_h, None)


def make_dataset(ctx, n, seed0=5000, sigma=8.0, chunk=256):
    """n seeded smooth-noise textures (normalised) and their FFT demag fields.

    Returns CUDA tensors M, H of shape (n, nz, ny, nx, 4)."""
    nz, ny, nx = ctx.shape
    M = torch.empty((n, nz, ny, nx, 4), dtype=torch.float32, device="cuda")
    H = torch.empty_like(M)
    for i in range(n):
        M[i] = to_dev4(inputs.smooth_texture((nz, ny, nx), sigma, seed0 + i))
        ctx.heff(M[i], out=H[i], terms=L.MX_TERM_DEMAG)
    torch.cuda.synchronize()
    return M, H


def normalizer_stats(M, H):
    """Per-component mean and standard deviation of inputs and targets (data preparation)."""
    m = M[..., :3].reshape(-1, 3).double()
    h = H[..., :3].reshape(-1, 3).double()
    st = [m.mean(0), m.std(0, unbiased=False), h.mean(0), h.std(0, unbiased=False)]
    return [float(v) for s in st for v in s.tolist()]


def train(net, M, H, epochs, batch, lr=1e-3, weight_decay=1e-4, milestones=(20, 40, 60), gamma=0.5, seed=0,
          log=None):
    """Adam with a step schedule (x gamma at each milestone epoch); returns the
    mean training loss of every epoch."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = M.shape[0]
    losses = []
    for ep in range(epochs):
        lr_ep = lr * gamma ** sum(ep >= mst for mst in milestones)
        perm = torch.as_tensor(rng.permutation(n), device=M.device)
        tot, cnt = torch.zeros(1, device=M.device), 0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            loss, _ = net.loss_grad(M.index_select(0, idx), H.index_select(0, idx), want_grad=False)
            net.adam_step(lr_ep, weight_decay)
            tot += loss
            cnt += 1
        losses.append(float(tot) / max(cnt, 1))
        if log:
            log(f"epoch {ep} lr {lr_ep:.2e} loss {losses[-1]:.4e}")
    return losses


def run_in_loop(ctx, net, m, nsteps, dt, judge_every, threshold=1e-2):
    """RK4 with the surrogate as demag backend; every `judge_every` steps the
    FFT demag judges the surrogate's field (relative L2); above `threshold`
    the run falls back to the FFT demag for its remaining steps.

    Returns dict(errors=[...], fallback_step=int or None)."""
    errors, fallback = [], None
    hs = torch.empty_like(m)
    hf = torch.empty_like(m)
    net.attach(ctx.h)
    try:
        done = 0
        while done < nsteps:
            k = min(judge_every, nsteps - done)
            ctx.rk_step(m, k, dt)
            done += k
            if fallback is None:
                ctx.heff(m, out=hs, terms=L.MX_TERM_DEMAG)
                net.detach(ctx.h)
                ctx.heff(m, out=hf, terms=L.MX_TERM_DEMAG)
                err = L.mx_rel_l2(ctx.h, hs, hf)
                errors.append((done, err))
                if err > threshold:
                    fallback = done
                else:
                    net.attach(ctx.h)
    finally:
        net.detach(ctx.h)
    ctx.sync()
    return {"errors": errors, "fallback_step": fallback}


def time_batched(ctx, net, M, reps=10):
    """Per-field time [ms] of demag fields for a batch of fields: the FFT
    convolution one field after another, and one batched surrogate forward
    (the net's max_batch fields at once)."""
    b = min(net.max_batch, M.shape[0])
    h = torch.empty_like(M[:b])
    out = {}
    for name in ("fft", "surrogate"):
        for _ in range(2):
            if name == "fft":
                for i in range(b):
                    ctx.heff(M[i], out=h[i], terms=L.MX_TERM_DEMAG)
            else:
                net.forward_into(M[:b].contiguous(), h, b)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            if name == "fft":
                for i in range(b):
                    ctx.heff(M[i], out=h[i], terms=L.MX_TERM_DEMAG)
            else:
                net.forward_into(M[:b].contiguous(), h, b)
        e1.record()
        torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1) / (reps * b)
    out["batch"] = b
    return out


def time_demag(ctx, net, m, reps=50):
    """Mean time [ms] of one demag evaluation by the FFT convolution and by the surrogate."""
    h = torch.empty_like(m)
    out = {}
    for name in ("fft", "surrogate"):
        if name == "fft":
            net.detach(ctx.h)
        else:
            net.attach(ctx.h)
        for _ in range(3):
            ctx.heff(m, out=h, terms=L.MX_TERM_DEMAG)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            ctx.heff(m, out=h, terms=L.MX_TERM_DEMAG)
        e1.record()
        torch.cuda.synchronize()
        out[name] = e0.elapsed_time(e1) / reps
    net.detach(ctx.h)
    return out
