"""Oracle: the Fourier-neural-operator demag surrogate (Sec. II-D) in FP64.

TEST INFRASTRUCTURE ONLY (plain CPU; the product never imports it).

Sec. II-D replaces the FFT demag of a thin film by a two-dimensional Fourier
neural operator (Li et al., "Fourier neural operator for parametric partial
differential equations"): a lifting layer 3 -> 32 channels, four spectral
convolution layers that keep the lowest 12 modes per dimension with
complex-valued learned filters, and a projection back to 3 channels, trained
with Adam (lr 1e-3, weight decay 1e-4, step schedule) on a SmoothL1 loss of
per-channel Gaussian-normalised inputs and targets.

Reading of the layers (the paper names them; the details follow Li et al.):
  v_0     = P x + p                                    (per cell, 3 -> 32)
  v_{l+1} = act_l( K_l v_l + W_l v_l + w_l ),  l = 0..3, act = exact-erf GELU
            for l < 3, identity after the last layer
  K_l v   = irfft2( R_l . rfft2(v) restricted to the kept modes ), kept modes:
            ky in [0, K) and [H-K, H) (the two low-frequency corners of the
            full transform along y), kx in [0, K) (the half spectrum along x);
            per kept mode, R_l is a complex 32 x 32 matrix acting on channels:
            Y_o = sum_i X_i R_l[mode, i, o]
  y       = Q2 gelu(Q1 v_4 + q1) + q2                  (per cell, 32 -> 128 -> 3)
Fields are (B, C, H, W) with H = ny (rows) and W = nx (columns) of a film.
torch's FP64 rfft2 / irfft2 are the transform primitives (pinned against the
closed form of the truncated transform pair by explicit sums); gradients come
from torch autograd (pinned against finite differences).

Parameter vector (flat, this order): P (32, 3), p (32), then per layer
R (2K, K, 32, 32, 2) [mode row (low corner then high corner), kx, in, out,
re/im], W (32, 32) [out, in], w (32); then Q1 (128, 32), q1 (128),
Q2 (3, 128), q2 (3).
"""
import math

import numpy as np
import torch

WIDTH = 32
HIDDEN = 128
LAYERS = 4
DT = torch.float64


def param_shapes(K):
    shapes = [(WIDTH, 3), (WIDTH,)]
    for _ in range(LAYERS):
        shapes += [(2 * K, K, WIDTH, WIDTH, 2), (WIDTH, WIDTH), (WIDTH,)]
    shapes += [(HIDDEN, WIDTH), (HIDDEN,), (3, HIDDEN), (3,)]
    return shapes


def num_params(K):
    return sum(int(np.prod(s)) for s in param_shapes(K))


def unflatten(flat, K):
    flat = torch.as_tensor(flat, dtype=DT)
    out, o = [], 0
    for s in param_shapes(K):
        n = int(np.prod(s))
        out.append(flat[o:o + n].reshape(s))
        o += n
    assert o == flat.numel()
    return out


def flatten(params):
    return torch.cat([p.reshape(-1) for p in params])


def init_params(K, seed):
    """Seeded initial parameters: pointwise weights and biases uniform in
    +-1/sqrt(fan_in); spectral filters uniform in [0, 1/(32*32)) for both the
    real and imaginary parts (the scale of Li et al.'s initialisation)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []

    def lin(cout, cin):
        bound = 1.0 / math.sqrt(cin)
        parts.append(rng.uniform(-bound, bound, size=cout * cin))
        parts.append(rng.uniform(-bound, bound, size=cout))

    lin(WIDTH, 3)
    for _ in range(LAYERS):
        parts.append(rng.uniform(0.0, 1.0 / (WIDTH * WIDTH), size=2 * K * K * WIDTH * WIDTH * 2))
        lin(WIDTH, WIDTH)
    lin(HIDDEN, WIDTH)
    lin(3, HIDDEN)
    return np.concatenate(parts)


def gelu(x):
    return 0.5 * x * (1.0 + torch.erf(x / math.sqrt(2.0)))


def kept_rows(H, K):
    """Row (ky) indices of the kept modes, in the order of R's first axis."""
    return list(range(K)) + list(range(H - K, H))


def spectral_conv(v, R, K):
    """K v for v (B, C, H, W) and R (2K, K, C, C, 2)."""
    B, C, H, W = v.shape
    assert 2 * K <= H and 2 * K <= W, "the kept modes need 2K <= H and 2K <= W"
    X = torch.fft.rfft2(v)  # (B, C, H, W//2+1)
    rows = kept_rows(H, K)
    Xk = X[:, :, rows, :K]  # (B, C, 2K, K)
    Rc = torch.complex(R[..., 0], R[..., 1])  # (2K, K, Cin, Cout)
    Y = torch.einsum("bimn,mnio->bomn", Xk, Rc)
    out = torch.zeros(B, R.shape[3], H, W // 2 + 1, dtype=torch.complex128)
    out[:, :, rows, :K] = Y
    return torch.fft.irfft2(out, s=(H, W))


def pointwise(v, Wt, b):
    """Per-cell linear map: (B, Cin, H, W) -> (B, Cout, H, W)."""
    return torch.einsum("oi,bihw->bohw", Wt, v) + b.view(1, -1, 1, 1)


def forward(params, x, K):
    """x: (B, 3, H, W) normalised magnetisation -> (B, 3, H, W) normalised field."""
    P, p = params[0], params[1]
    v = pointwise(x, P, p)
    for l in range(LAYERS):
        R, Wt, w = params[2 + 3 * l: 5 + 3 * l]
        u = spectral_conv(v, R, K) + pointwise(v, Wt, w)
        v = gelu(u) if l < LAYERS - 1 else u
    Q1, q1, Q2, q2 = params[-4:]
    return pointwise(gelu(pointwise(v, Q1, q1)), Q2, q2)


def smooth_l1(pred, target):
    """Mean SmoothL1 with beta = 1: 0.5 d^2 where |d| < 1, |d| - 0.5 elsewhere."""
    d = pred - target
    ad = d.abs()
    return torch.where(ad < 1.0, 0.5 * d * d, ad - 0.5).mean()


def loss_and_grad(flat, x, target, K):
    params = [p.clone().requires_grad_(True) for p in unflatten(flat, K)]
    L = smooth_l1(forward(params, x, K), target)
    grads = torch.autograd.grad(L, params)
    return float(L.detach()), flatten(grads).detach()


def spectral_conv_direct(v, R, K):
    """The truncated transform pair written out as explicit sums (pin for
    spectral_conv; tiny grids only):
      X[ky,kx,i] = sum_{y,x} v[i,y,x] exp(-2 pi i (ky y / H + kx x / W))
      Y[ky,kx,o] = sum_i X[ky,kx,i] R[ky,kx,i,o]
      out[o,y,x] = (1 / (H W)) sum_{kept} c_kx Re(Y[ky,kx,o] exp(+2 pi i (ky y / H + kx x / W)))
    with c_0 = 1 and c_kx = 2 for kx > 0 (the half spectrum stands for its
    conjugate mirror; only the real part of the kx = 0 column survives)."""
    v = np.asarray(v, dtype=np.float64)
    B, C, H, W = v.shape
    Rc = np.asarray(R[..., 0]) + 1j * np.asarray(R[..., 1])
    Cout = Rc.shape[3]
    out = np.zeros((B, Cout, H, W))
    rows = kept_rows(H, K)
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    for b in range(B):
        for m, ky in enumerate(rows):
            for kx in range(K):
                ph = 2.0 * np.pi * (ky * yy / H + kx * xx / W)
                X = np.array([np.sum(v[b, i] * np.exp(-1j * ph)) for i in range(C)])
                Y = X @ Rc[m, kx]
                ck = 1.0 if kx == 0 else 2.0
                for o in range(Cout):
                    out[b, o] += ck * np.real(Y[o] * np.exp(1j * ph)) / (H * W)
    return out


def adjoint_filters(R):
    """R' with R'[mode, o, i] = conj(R[mode, i, o]): the spectral convolution
    with R' is the transpose of the one with R (<K_R a, b> = <a, K_R' b>)."""
    Rt = R.transpose(2, 3).clone()
    Rt[..., 1] = -Rt[..., 1]
    return Rt


def to_nchw(a):
    """(B, ny, nx, 3) -> (B, 3, ny, nx)."""
    return torch.as_tensor(a, dtype=DT).permute(0, 3, 1, 2).contiguous()


def from_nchw(a):
    return a.permute(0, 2, 3, 1).contiguous()
