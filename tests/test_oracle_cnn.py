"""Pins for the oracle's conv-net surrogate (CPU only)."""
import math

import numpy as np
import torch

from oracle import cnn


def test_conv3d_primitive_matches_explicit_loops():
    rng = np.random.default_rng(41)
    x = rng.normal(size=(2, 3, 3, 4, 5))
    W = rng.normal(size=(4, 3, 3, 3, 3))
    b = rng.normal(size=4)
    ref = cnn.conv3d_loops(x, W, b)
    got = torch.nn.functional.conv3d(torch.from_numpy(x), torch.from_numpy(W), torch.from_numpy(b), padding=1)
    assert np.abs(got.numpy() - ref).max() < 1e-12


def test_gelu_closed_values():
    x = torch.tensor([0.0, 1.0, -1.0, 3.0], dtype=torch.float64)
    ref = [0.0, 0.5 * (1 + math.erf(1 / math.sqrt(2))), -0.5 * (1 - math.erf(1 / math.sqrt(2))),
           1.5 * (1 + math.erf(3 / math.sqrt(2)))]
    assert torch.allclose(cnn.gelu(x), torch.tensor(ref, dtype=torch.float64), atol=1e-15)


def test_smooth_l1_branches():
    p = torch.tensor([0.0, 0.5, 3.0], dtype=torch.float64)
    t = torch.zeros(3, dtype=torch.float64)
    assert abs(float(cnn.smooth_l1(p, t)) - (0.0 + 0.125 + 2.5) / 3) < 1e-15


def test_network_gradient_matches_central_differences():
    rng = np.random.default_rng(42)
    flat = torch.from_numpy(cnn.init_params(7))
    x = torch.from_numpy(rng.normal(size=(2, 3, 2, 4, 4)))
    tgt = torch.from_numpy(rng.normal(size=(2, 3, 2, 4, 4)))
    L, g = cnn.loss_and_grad(flat, x, tgt)
    for idx in rng.choice(flat.numel(), size=6, replace=False).tolist() + [flat.numel() - 1]:
        h = 1e-6
        fp, fm = flat.clone(), flat.clone()
        fp[idx] += h
        fm[idx] -= h
        Lp = float(cnn.smooth_l1(cnn.forward(cnn.unflatten(fp), x), tgt))
        Lm = float(cnn.smooth_l1(cnn.forward(cnn.unflatten(fm), x), tgt))
        fd = (Lp - Lm) / (2 * h)
        # central-difference noise floor: eps * L / h ~ 1e-10
        assert abs(fd - float(g[idx])) <= 1e-6 * abs(fd) + 2e-10, (idx, fd, float(g[idx]))


def test_adam_first_step_by_hand():
    """First step: m = (1-b1) g, v = (1-b2) g^2, bias corrections give m_hat = g,
    v_hat = g^2, so the update is lr * g / (|g| + eps) per parameter."""
    th = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64)
    g = torch.tensor([0.3, -0.1, 0.0], dtype=torch.float64)
    wd, lr = 1e-4, 1e-3
    new, m, v = cnn.adam_step(th, g, torch.zeros(3), torch.zeros(3), 1, lr, wd)
    gg = g + wd * th
    ref = th - lr * gg / (gg.abs() + 1e-8)
    assert torch.allclose(new, ref, atol=1e-15)


def test_bf16_rounding_is_nearest():
    x = torch.tensor([1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, 1.0], dtype=torch.float64)
    r = cnn.bf16_round(x)
    assert r.tolist() == [1.0, 1.0 + 2 ** -7, 1.0]  # ties to even, then round up


def test_normalizer_round_trip():
    a = np.random.default_rng(43).normal(size=(5, 4, 3)) * [1, 2, 3] + [0.1, -1, 2]
    n = cnn.Normalizer(a)
    e = n.encode(a).reshape(-1, 3)
    assert torch.allclose(e.mean(0), torch.zeros(3, dtype=torch.float64), atol=1e-12)
    assert torch.allclose(e.std(0, unbiased=False), torch.ones(3, dtype=torch.float64), atol=1e-12)
    assert torch.allclose(n.decode(n.encode(a)), torch.as_tensor(a), atol=1e-12)


def test_input_gradient_is_a_convolution_with_flipped_transposed_weights():
    """dL/dx of y = conv3d(x, W) (3x3x3, zero padding 1) equals conv3d(dL/dy, W')
    with W'[ci][co][dz][dy][dx] = W[co][ci][2-dz][2-dy][2-dx]: the layout the
    GPU backward pass packs its weights in."""
    rng = np.random.default_rng(44)
    x = torch.from_numpy(rng.normal(size=(2, 3, 3, 5, 4))).requires_grad_(True)
    W = torch.from_numpy(rng.normal(size=(4, 3, 3, 3, 3)))
    g = torch.from_numpy(rng.normal(size=(2, 4, 3, 5, 4)))
    (torch.nn.functional.conv3d(x, W, padding=1) * g).sum().backward()
    Wf = W.flip(2, 3, 4).transpose(0, 1).contiguous()
    ref = torch.nn.functional.conv3d(g, Wf, padding=1)
    assert torch.allclose(x.grad, ref, atol=1e-12)
