"""Fourier-neural-operator surrogate on the GPU vs the FP64 oracle, through the C ABI.

Tolerances (FP32 network vs FP64 oracle on the same float32 inputs and
parameters): outputs relative L2 <= 2e-5 and max error <= 2e-4 of the largest
value; loss relative 1e-5; every parameter block's gradient relative L2
<= 1e-4 (FP32 sums over up to a few thousand cells and 32 channels).
"""
import numpy as np
import pytest
import torch

from oracle import cnn as ocnn
from oracle import fno

pytestmark = pytest.mark.gpu


def params_for(K, seed, filt=0.05):
    """Seeded parameters: pointwise parts uniform in +-1/sqrt(fan_in),
    spectral filters N(0, filt^2) (large enough that the spectral path
    dominates the output)."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in fno.param_shapes(K):
        n = int(np.prod(s))
        if len(s) == 5:
            parts.append(rng.normal(scale=filt, size=n))
        else:
            fan_in = s[1] if len(s) == 2 else 32
            parts.append(rng.uniform(-1, 1, size=n) / np.sqrt(fan_in))
    return np.concatenate(parts).astype(np.float32).astype(np.float64)


def fields(B, ny, nx, seed):
    rng = np.random.default_rng(seed)
    m = rng.normal(size=(B, ny, nx, 3))
    m /= np.linalg.norm(m, axis=-1, keepdims=True)
    return m.astype(np.float32).astype(np.float64)


STATS = np.array([0.1, -0.05, 0.2, 0.6, 0.55, 0.5, 30.0, -12.0, 5.0, 4e4, 3e4, 2e4], dtype=np.float32).astype(
    np.float64)


def dev4(a):
    B, ny, nx, _ = a.shape
    t = torch.zeros((B, 1, ny, nx, 4), dtype=torch.float32)
    t[..., :3] = torch.from_numpy(a.reshape(B, 1, ny, nx, 3))
    return t.cuda()


def oracle_h(flat, m, K, stats=STATS):
    x = fno.to_nchw((m - stats[0:3]) / stats[3:6])
    y = fno.forward(fno.unflatten(torch.from_numpy(flat), K), x, K)
    return fno.from_nchw(y).numpy() * stats[9:12] + stats[6:9]


def make_net(nx, ny, K, B, flat, stats=STATS):
    from paper_2602_12242_gb300.surrogate import FourierSurrogate
    net = FourierSurrogate(nx, ny, K, max_batch=B)
    net.set_params(torch.from_numpy(flat.astype(np.float32)))
    net.set_normalizer(stats)
    return net


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("nx,ny,K,B", [(40, 24, 6, 3), (128, 32, 12, 2), (37, 26, 5, 2), (24, 24, 12, 1),
                                       (1024, 24, 12, 1), (24, 1024, 12, 1), (64, 100, 16, 1)])
def test_forward_matches_oracle(nx, ny, K, B):
    """Small and ragged grids, the paper's K = 12 on the SP4 film grid, the
    kept rows filling the whole column (2K = ny), the largest rows and
    columns (1024) and the largest K."""
    flat = params_for(K, 1)
    m = fields(B, ny, nx, 2)
    net = make_net(nx, ny, K, B, flat)
    h = net.forward(dev4(m)).cpu().numpy()[:, 0, :, :, :3]
    ref = oracle_h(flat, m, K)
    assert rel_l2(h, ref) <= 2e-5
    assert np.abs(h - ref).max() <= 2e-4 * np.abs(ref).max()


def test_batch_members_are_independent():
    """A sample's output does not depend on the rest of the batch (bit for bit)."""
    nx, ny, K = 40, 24, 6
    flat = params_for(K, 3)
    m = fields(3, ny, nx, 4)
    net = make_net(nx, ny, K, 3, flat)
    hb = net.forward(dev4(m)).cpu()
    h1 = net.forward(dev4(m[1:2])).cpu()
    assert torch.equal(hb[1:2], h1)


@pytest.mark.parametrize("nx,ny,K,B", [(24, 16, 4, 2), (37, 26, 5, 3), (128, 32, 12, 1)])
def test_loss_and_gradient_match_oracle(nx, ny, K, B):
    flat = params_for(K, 5)
    m = fields(B, ny, nx, 6)
    rng = np.random.default_rng(7)
    target = (rng.normal(size=(B, ny, nx, 3)) * 1.5 * STATS[9:12] + STATS[6:9]).astype(np.float32).astype(
        np.float64)
    net = make_net(nx, ny, K, B, flat)
    loss, grad = net.loss_grad(dev4(m), dev4(target))
    loss, grad = float(loss.cpu()), grad.cpu().numpy().astype(np.float64)
    x = fno.to_nchw((m - STATS[0:3]) / STATS[3:6])
    t = fno.to_nchw((target - STATS[6:9]) / STATS[9:12])
    L, g = fno.loss_and_grad(torch.from_numpy(flat), x, t, K)
    g = g.numpy()
    assert abs(loss - L) <= 1e-5 * abs(L)
    offs = np.cumsum([0] + [int(np.prod(s)) for s in fno.param_shapes(K)])
    for i in range(len(offs) - 1):
        a, b = grad[offs[i]:offs[i + 1]], g[offs[i]:offs[i + 1]]
        assert rel_l2(a, b) <= 1e-4, (i, fno.param_shapes(K)[i], rel_l2(a, b))


def test_adam_step_matches_oracle():
    nx, ny, K, B = 24, 16, 4, 2
    flat = params_for(K, 8)
    m = fields(B, ny, nx, 9)
    target = fields(B, ny, nx, 10) * STATS[9:12] + STATS[6:9]
    net = make_net(nx, ny, K, B, flat)
    _, grad = net.loss_grad(dev4(m), dev4(target))
    net.adam_step(1e-3, 1e-4)
    got = net.get_params().cpu().numpy().astype(np.float64)
    g = torch.from_numpy(grad.cpu().numpy().astype(np.float64))
    z = torch.zeros_like(g)
    ref, _, _ = ocnn.adam_step(torch.from_numpy(flat), g, z, z, 1, 1e-3, 1e-4)
    assert np.abs(got - ref.numpy()).max() <= 1e-6 * max(1.0, np.abs(flat).max())


def test_film_demag_backend_and_refusals():
    """As the context's demag backend the network gives the demag term of
    mx_heff (bit for bit); the adjoint refuses it; grid mismatches and modes
    without room are refused."""
    from helpers import cfg_of, context
    from paper_2602_12242_gb300 import MxError, _lib
    from paper_2602_12242_gb300.surrogate import FourierSurrogate
    nx, ny, K = 64, 32, 8
    flat = params_for(K, 11)
    net = make_net(nx, ny, K, 1, flat)
    ctx = context(cfg_of(nx=nx, ny=ny, nz=1, dx=3.9e-9, dy=3.9e-9, dz=3e-9))
    m = dev4(fields(1, ny, nx, 12))[0]
    direct = net.forward(m.unsqueeze(0))[0]
    net.attach(ctx.h)
    try:
        h = ctx.heff(m, terms=_lib.MX_TERM_DEMAG)
        assert torch.equal(h[..., :3], direct[..., :3])
        m2 = m.clone()
        ctx.rk_step(m2, 3, 1e-14)
        assert torch.isfinite(m2).all()
        with pytest.raises(MxError) as e:
            ctx.adjoint_reserve(4, 2)
            ctx.rk_forward_record(m, 1e-14)
        assert e.value.status == _lib.MX_ERR_UNSUPPORTED
    finally:
        net.detach(ctx.h)
    ctx3 = context(cfg_of(nx=nx, ny=ny, nz=2))
    with pytest.raises(MxError):
        net.attach(ctx3.h)
    with pytest.raises(MxError):
        FourierSurrogate(30, 20, 12, 1)  # 2K > ny
    with pytest.raises(MxError):
        FourierSurrogate(64, 64, 17, 1)  # K > 16
    assert _lib.mx_fno_num_params(12) == fno.num_params(12)


def test_training_reduces_loss_and_in_loop_fallback():
    """Training through the C ABI lowers the loss; as the demag backend of a
    film run the FFT judge (threshold 1e-2) rejects the briefly trained
    network at its first check, and a loose threshold leaves it in charge."""
    from helpers import cfg_of, context
    from paper_2602_12242_gb300.surrogate import (FourierSurrogate, init_fno_params, make_dataset, normalizer_stats,
                                                  run_in_loop, train)
    c = cfg_of(nx=48, ny=32, nz=1, dx=3.125e-9, dy=3.125e-9, dz=3.125e-9)
    ctx = context(c)
    M, H = make_dataset(ctx, 96, seed0=9100)
    net = FourierSurrogate(48, 32, 6, max_batch=16)
    net.set_params(torch.as_tensor(init_fno_params(6, 3)))
    net.set_normalizer(normalizer_stats(M, H))
    losses = train(net, M, H, epochs=10, batch=16, lr=2e-3)
    assert losses[-1] < 0.7 * losses[0], losses
    m = M[0].clone()
    res = run_in_loop(ctx, net, m, nsteps=6, dt=1e-14, judge_every=3, threshold=1e-2)
    assert res["errors"] and res["fallback_step"] == 3
    nrm = torch.linalg.vector_norm(m[..., :3], dim=-1)
    assert float((nrm - 1).abs().max()) < 1e-5
    m2 = M[1].clone()
    res2 = run_in_loop(ctx, net, m2, nsteps=6, dt=1e-14, judge_every=3, threshold=10.0)
    assert res2["fallback_step"] is None and len(res2["errors"]) == 2
