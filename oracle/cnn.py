"""Oracle: the learned demag surrogate (a small 3D conv net) in FP64.

TEST INFRASTRUCTURE ONLY (plain CPU; the product never imports it).

The paper's ML module (Sec. II-D) replaces the FFT demag with a network
trained offline on (M, H_demag) pairs from the conventional solver, with a
per-channel Gaussian normaliser of inputs and targets, Adam (lr 1e-3, weight
decay 1e-4), a step learning-rate schedule and a SmoothL1 ("MAE") loss.  The
network here is the 3D conv net of the workload: 3 -> 32 -> 64 -> 32 -> 3
channels, 3x3x3 kernels with zero padding 1, exact-erf GELU after the first
three convolutions.  torch's conv3d in float64 is the convolution primitive
(pinned against explicit loops); gradients come from torch autograd (pinned
against finite differences).

Optional rounding hook ``rnd`` reproduces the places where a BF16 pipeline
rounds (inputs, weights, hidden activations), so a BF16 implementation can be
compared with the same rounded operands.
"""
import math

import numpy as np
import torch
import torch.nn.functional as F

CHANNELS = (3, 32, 64, 32, 3)
DT = torch.float64


def param_shapes():
    shapes = []
    for l in range(4):
        cin, cout = CHANNELS[l], CHANNELS[l + 1]
        shapes.append((cout, cin, 3, 3, 3))
        shapes.append((cout,))
    return shapes


def num_params():
    return sum(int(np.prod(s)) for s in param_shapes())


def unflatten(flat):
    flat = torch.as_tensor(flat, dtype=DT)
    out, o = [], 0
    for s in param_shapes():
        n = int(np.prod(s))
        out.append(flat[o:o + n].reshape(s))
        o += n
    return out


def flatten(params):
    return torch.cat([p.reshape(-1) for p in params])


def init_params(seed):
    """Kaiming-uniform-like init (uniform in +-1/sqrt(fan_in)), seeded."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for l in range(4):
        cin, cout = CHANNELS[l], CHANNELS[l + 1]
        bound = 1.0 / math.sqrt(cin * 27)
        parts.append(rng.uniform(-bound, bound, size=cout * cin * 27))
        parts.append(rng.uniform(-bound, bound, size=cout))
    return np.concatenate(parts)


def gelu(x):
    return 0.5 * x * (1.0 + torch.erf(x / math.sqrt(2.0)))


def ident(x):
    return x


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned in float64."""
    return x.to(torch.float32).to(torch.bfloat16).to(DT)


def forward(params, x, rnd=ident):
    """x: (B, 3, nz, ny, nx) normalised input -> (B, 3, nz, ny, nx) normalised output."""
    a = rnd(x)
    for l in range(4):
        W, b = params[2 * l], params[2 * l + 1]
        acc = F.conv3d(a, rnd(W), b, padding=1)
        a = rnd(gelu(acc)) if l < 3 else acc
    return a


def conv3d_loops(x, W, b):
    """Direct 3x3x3 zero-padded convolution by loops (pin for F.conv3d)."""
    B, cin, nz, ny, nx = x.shape
    cout = W.shape[0]
    xp = np.zeros((B, cin, nz + 2, ny + 2, nx + 2))
    xp[:, :, 1:-1, 1:-1, 1:-1] = x
    out = np.zeros((B, cout, nz, ny, nx))
    for bb in range(B):
        for co in range(cout):
            for k in range(nz):
                for j in range(ny):
                    for i in range(nx):
                        s = b[co]
                        for ci in range(cin):
                            for dz in range(3):
                                for dy in range(3):
                                    for dx in range(3):
                                        s += W[co, ci, dz, dy, dx] * xp[bb, ci, k + dz, j + dy, i + dx]
                        out[bb, co, k, j, i] = s
    return out


def smooth_l1(pred, target):
    """Mean SmoothL1 with beta = 1: 0.5 d^2 where |d| < 1, |d| - 0.5 elsewhere."""
    d = pred - target
    ad = d.abs()
    return torch.where(ad < 1.0, 0.5 * d * d, ad - 0.5).mean()


def loss_and_grad(flat, x, target, rnd=ident):
    params = [p.clone().requires_grad_(True) for p in unflatten(flat)]
    L = smooth_l1(forward(params, x, rnd), target)
    grads = torch.autograd.grad(L, params)
    return float(L.detach()), flatten(grads).detach()


def adam_step(flat, grad, m, v, t, lr, wd, beta1=0.9, beta2=0.999, eps=1e-8):
    """Adam with L2-coupled weight decay (the decay is added to the gradient)."""
    flat, grad, m, v = (torch.as_tensor(a, dtype=DT) for a in (flat, grad, m, v))
    g = grad + wd * flat
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return flat - lr * mhat / (vhat.sqrt() + eps), m, v


class Normalizer:
    """Per-channel Gaussian normaliser (mean and standard deviation per component)."""

    def __init__(self, data):
        # data: (..., 3)
        d = torch.as_tensor(data, dtype=DT).reshape(-1, 3)
        self.mean = d.mean(0)
        self.std = d.std(0, unbiased=False)

    def encode(self, a):
        return (torch.as_tensor(a, dtype=DT) - self.mean) / self.std

    def decode(self, a):
        return torch.as_tensor(a, dtype=DT) * self.std + self.mean


def to_ncdhw(a):
    """(B, nz, ny, nx, 3) -> (B, 3, nz, ny, nx)."""
    return torch.as_tensor(a, dtype=DT).permute(0, 4, 1, 2, 3).contiguous()


def from_ncdhw(a):
    return a.permute(0, 2, 3, 4, 1).contiguous()
