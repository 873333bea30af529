"""Property-based pins of the oracle over random small shapes (CPU only):
the identities hold for every grid, cell aspect ratio and mode count, not just
the hand-picked cases of the other pin files."""
import numpy as np
import pytest
import torch

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

from oracle import fno  # noqa: E402
from oracle import micromag as mm  # noqa: E402

SETTINGS = dict(max_examples=12, deadline=None, derandomize=True)
cells = st.integers(1, 6)
aspect = st.floats(0.5, 2.0)


@settings(**SETTINGS)
@given(nx=cells, ny=cells, nz=st.integers(1, 3), ay=aspect, az=aspect, seed=st.integers(0, 2 ** 16))
def test_fft_convolution_equals_direct_sum_any_grid(nx, ny, nz, ay, az, seed):
    p = mm.Problem(nx, ny, nz, 2e-9, 2e-9 * ay, 2e-9 * az, Ms=8e5)
    m = mm.normalize(torch.from_numpy(np.random.default_rng(seed).normal(size=(nz, ny, nx, 3))))
    a = mm.demag_field(p, m)
    b = mm.demag_field_direct(p, m)
    assert float((a - b).abs().max()) <= 1e-11 * float(b.abs().max())


@settings(**SETTINGS)
@given(nx=cells, ny=cells, nz=st.integers(1, 3), ay=aspect, dmi=st.booleans(), seed=st.integers(0, 2 ** 16))
def test_linear_operator_is_symmetric_any_grid(nx, ny, nz, ay, dmi, seed):
    """<a, Ms L b> = <b, Ms L a> for exchange + DMI (chiral edges) + demag."""
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx)
    Ms = rng.uniform(6e5, 1e6, size=shape)
    p = mm.Problem(nx, ny, nz, 2e-9, 2e-9 * ay, 2.5e-9, Ms=Ms, A=1.3e-11, D=1.5e-3, dmi=dmi)

    def L(v):
        mp = mm.ghosted(p, v)
        return mm.exchange_field(p, v, mp) + mm.dmi_field(p, v, mp) + mm.demag_field(p, v)

    a = torch.from_numpy(rng.normal(size=shape + (3,)))
    b = torch.from_numpy(rng.normal(size=shape + (3,)))
    w = torch.from_numpy(Ms)[..., None]
    lhs = float((w * a * L(b)).sum())
    rhs = float((w * b * L(a)).sum())
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + abs(rhs) + 1e-300)


@settings(**SETTINGS)
@given(K=st.integers(1, 3), extra_h=st.integers(0, 3), extra_w=st.integers(0, 3), seed=st.integers(0, 2 ** 16))
def test_fno_spectral_conv_equals_explicit_sums_any_grid(K, extra_h, extra_w, seed):
    H, W = 2 * K + extra_h, 2 * K + extra_w
    rng = np.random.default_rng(seed)
    v = torch.from_numpy(rng.normal(size=(1, 2, H, W)))
    R = torch.from_numpy(rng.normal(size=(2 * K, K, 2, 3, 2)))
    got = fno.spectral_conv(v, R, K).numpy()
    ref = fno.spectral_conv_direct(v.numpy(), R.numpy(), K)
    assert np.abs(got - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1e-300)


@settings(**SETTINGS)
@given(K=st.integers(1, 3), extra_h=st.integers(0, 3), extra_w=st.integers(0, 3), seed=st.integers(0, 2 ** 16))
def test_fno_filter_transpose_any_grid(K, extra_h, extra_w, seed):
    H, W = 2 * K + extra_h, 2 * K + extra_w
    rng = np.random.default_rng(seed)
    R = torch.from_numpy(rng.normal(size=(2 * K, K, 3, 2, 2)))
    a = torch.from_numpy(rng.normal(size=(1, 3, H, W)))
    b = torch.from_numpy(rng.normal(size=(1, 2, H, W)))
    lhs = float((fno.spectral_conv(a, R, K) * b).sum())
    rhs = float((a * fno.spectral_conv(b, fno.adjoint_filters(R), K)).sum())
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + abs(rhs) + 1e-300)


@settings(**SETTINGS)
@given(nx=cells, ny=cells, nz=st.integers(1, 3), seed=st.integers(0, 2 ** 16))
def test_llg_right_hand_side_is_tangent_any_grid(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    p = mm.Problem(nx, ny, nz, 2e-9, 2e-9, 2e-9, Ms=8e5, A=1.3e-11, Ku=3e4, alpha=0.2, D=1e-3, dmi=True,
                   h_bias=tuple(rng.normal(size=3) * 1e4))
    m = mm.normalize(torch.from_numpy(rng.normal(size=(nz, ny, nx, 3))))
    dm = mm.rhs(p, m)
    assert float((m * dm).sum(-1).abs().max()) <= 1e-12 * float(dm.abs().max())
