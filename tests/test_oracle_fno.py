"""Pins for the oracle's Fourier-neural-operator surrogate (CPU only)."""
import numpy as np
import pytest
import torch

from oracle import fno


def rand_R(rng, K, cin, cout):
    return torch.from_numpy(rng.normal(size=(2 * K, K, cin, cout, 2)))


@pytest.mark.parametrize("H,W,K", [(6, 5, 2), (8, 8, 4), (7, 10, 3)])
def test_spectral_conv_matches_explicit_sums(H, W, K):
    """torch's rfft2/irfft2 with the corner selection equal the truncated
    transform pair written out term by term (odd and even sizes, and a grid
    whose kept rows cover every row)."""
    rng = np.random.default_rng(60)
    v = torch.from_numpy(rng.normal(size=(2, 3, H, W)))
    R = rand_R(rng, K, 3, 4)
    got = fno.spectral_conv(v, R, K).numpy()
    ref = fno.spectral_conv_direct(v.numpy(), R.numpy(), K)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def identity_R(K, C):
    R = torch.zeros(2 * K, K, C, C, 2, dtype=torch.float64)
    R[:, :, range(C), range(C), 0] = 1.0
    return R


@pytest.mark.parametrize("ky,kx,gain", [(0, 0, 1.0), (2, 1, 1.0), (-3, 2, 1.0), (-4, 3, 1.0), (5, 0, 0.0),
                                        (1, 4, 0.0), (-5, 1, 0.0), (-4, 0, 0.5)])
def test_plane_wave_passes_or_is_removed(ky, kx, gain):
    """Identity filters, H = 16, W = 12, K = 4 (kept rows 0..3 and 12..15,
    columns 0..3): a real plane wave cos(2 pi (ky y/H + kx x/W) + phi) in one
    channel comes out unchanged when its mode is kept and as zero when it is
    not.  On the kx = 0 column the two corners are not mirror images (ky = -4
    is kept, ky = +4 is not), so that wave keeps half its amplitude."""
    H, W, K, C = 16, 12, 4, 3
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    wave = np.cos(2 * np.pi * (ky * yy / H + kx * xx / W) + 0.7)
    v = np.zeros((1, C, H, W))
    v[0, 1] = wave
    out = fno.spectral_conv(torch.from_numpy(v), identity_R(K, C), K).numpy()
    assert np.abs(out - gain * v).max() <= 1e-13


def test_adjoint_filters_transpose_the_spectral_convolution():
    """<K_R a, b> = <a, K_R' b> with R'[mode, o, i] = conj(R[mode, i, o]): the
    transpose the GPU backward pass applies to the output gradient."""
    rng = np.random.default_rng(62)
    for H, W, K in [(8, 10, 3), (9, 7, 2)]:
        R = rand_R(rng, K, 3, 5)
        a = torch.from_numpy(rng.normal(size=(2, 3, H, W)))
        b = torch.from_numpy(rng.normal(size=(2, 5, H, W)))
        lhs = float((fno.spectral_conv(a, R, K) * b).sum())
        rhs = float((a * fno.spectral_conv(b, fno.adjoint_filters(R), K)).sum())
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1e-300)


def test_network_is_shift_equivariant():
    """Every layer is per-cell or a Fourier multiplier on the periodic grid, so
    the network commutes with periodic shifts of the field."""
    rng = np.random.default_rng(63)
    K = 3
    params = fno.unflatten(torch.from_numpy(fno.init_params(K, 5)), K)
    # larger filters than the initial scale, so the spectral path matters
    for l in range(fno.LAYERS):
        params[2 + 3 * l] = rand_R(rng, K, 32, 32) * 0.05
    x = torch.from_numpy(rng.normal(size=(1, 3, 8, 12)))
    y = fno.forward(params, x, K)
    ys = fno.forward(params, torch.roll(x, shifts=(3, -5), dims=(2, 3)), K)
    assert torch.allclose(ys, torch.roll(y, shifts=(3, -5), dims=(2, 3)), atol=1e-12)


def test_parameter_layout_and_count():
    K = 12
    n = 32 * 3 + 32 + 4 * (2 * K * K * 32 * 32 * 2 + 32 * 32 + 32) + 128 * 32 + 128 + 3 * 128 + 3
    assert fno.num_params(K) == n == 2_368_259
    flat = torch.arange(fno.num_params(2), dtype=torch.float64)
    ps = fno.unflatten(flat, 2)
    assert fno.flatten(ps).equal(flat)
    assert ps[2].shape == (4, 2, 32, 32, 2) and ps[-4].shape == (128, 32)


def test_network_gradient_matches_central_differences():
    rng = np.random.default_rng(64)
    K = 2
    base = fno.init_params(K, 9)
    base[32 * 3 + 32: 32 * 3 + 32 + 4 * 2 * 32 * 32 * 2] = rng.normal(scale=0.02, size=4 * 2 * 32 * 32 * 2)
    flat = torch.from_numpy(base)
    x = torch.from_numpy(rng.normal(size=(2, 3, 4, 5)))
    tgt = torch.from_numpy(rng.normal(size=(2, 3, 4, 5)))
    L, g = fno.loss_and_grad(flat, x, tgt, K)
    offs = np.cumsum([0] + [int(np.prod(s)) for s in fno.param_shapes(K)])
    picks = [int(rng.integers(offs[i], offs[i + 1])) for i in range(len(offs) - 1)]
    for idx in picks:
        h = 1e-6
        fp, fm = flat.clone(), flat.clone()
        fp[idx] += h
        fm[idx] -= h
        Lp = float(fno.smooth_l1(fno.forward(fno.unflatten(fp, K), x, K), tgt))
        Lm = float(fno.smooth_l1(fno.forward(fno.unflatten(fm, K), x, K), tgt))
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - float(g[idx])) <= 1e-6 * abs(fd) + 2e-10, (idx, fd, float(g[idx]))


def test_kept_modes_need_room():
    with pytest.raises(AssertionError):
        fno.spectral_conv(torch.zeros(1, 1, 5, 8, dtype=torch.float64), torch.zeros(6, 3, 1, 1, 2,
                                                                                     dtype=torch.float64), 3)


@pytest.mark.parametrize("H,W,K", [(8, 10, 3), (9, 7, 2), (6, 6, 3)])
def test_filter_gradient_closed_form(H, W, K):
    """dL/dR for L = <g, K_R v> equals c_kx / (H W) * sum_b conj(X[b, i]) X_g[b, o]
    per kept mode (X, X_g: truncated rfft2 of v and g; c_0 = 1, c_kx = 2):
    the formula the GPU backward evaluates, against autograd of the oracle."""
    rng = np.random.default_rng(65)
    B, Ci, Co = 2, 3, 4
    v = torch.from_numpy(rng.normal(size=(B, Ci, H, W)))
    g = torch.from_numpy(rng.normal(size=(B, Co, H, W)))
    R = rand_R(rng, K, Ci, Co).requires_grad_(True)
    (fno.spectral_conv(v, R, K) * g).sum().backward()
    rows = fno.kept_rows(H, K)
    X = torch.fft.rfft2(v)[:, :, rows, :K]   # (B, Ci, 2K, K)
    Xg = torch.fft.rfft2(g)[:, :, rows, :K]  # (B, Co, 2K, K)
    c = torch.full((K,), 2.0, dtype=torch.float64)
    c[0] = 1.0
    dR = torch.einsum("bimn,bomn->mnio", X.conj(), Xg) * c.view(1, K, 1, 1) / (H * W)
    ref = torch.stack([dR.real, dR.imag], dim=-1)
    assert torch.allclose(R.grad, ref, rtol=1e-10, atol=1e-12 * float(ref.abs().max()))
