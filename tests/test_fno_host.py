"""Host-side checks of the FNO surrogate's C ABI and parameter layout (CPU only:
no call here reaches the device)."""
import numpy as np
import pytest

from oracle import fno


@pytest.fixture(scope="module")
def lib():
    from paper_2602_12242_gb300 import _lib, build
    build.build()
    return _lib


def test_parameter_count_matches_the_oracle_layout(lib):
    for K in range(1, 17):
        assert lib.mx_fno_num_params(K) == fno.num_params(K)
    assert lib.mx_fno_num_params(0) == -1 and lib.mx_fno_num_params(17) == -1


@pytest.mark.parametrize("nx,ny,K,B", [(30, 20, 12, 1), (20, 30, 12, 1), (64, 64, 0, 1), (64, 64, 17, 1),
                                       (2048, 64, 12, 1), (64, 2048, 12, 1), (64, 64, 12, 0),
                                       (64, 64, 12, 65536)])
def test_create_refuses_grids_without_room_for_the_modes(lib, nx, ny, K, B):
    """2K <= nx, ny <= 1024, 1 <= K <= 16 and 1 <= max_batch <= 65535, checked before any allocation."""
    with pytest.raises(lib.MxError) as e:
        lib.mx_fno_create(nx, ny, K, B)
    assert e.value.status == lib.MX_ERR_INVALID_ARG


def test_initial_parameters_follow_the_layout():
    """The seeded initial vector has the oracle's block sizes: filters in
    [0, 1/32^2), pointwise blocks within +-1/sqrt(fan_in)."""
    from paper_2602_12242_gb300.surrogate import init_fno_params
    K = 5
    flat = init_fno_params(K, 3).astype(np.float64)
    assert flat.size == fno.num_params(K)
    o = 0
    for s in fno.param_shapes(K):
        n = int(np.prod(s))
        blk = flat[o:o + n]
        if len(s) == 5:
            assert blk.min() >= 0.0 and blk.max() < 1.0 / 1024
        else:
            fan_in = {(32, 3): 3, (32,): None, (32, 32): 32, (128, 32): 32, (128,): 32, (3, 128): 128,
                      (3,): 128}[s]
            if fan_in is not None:
                assert np.abs(blk).max() <= 1.0 / np.sqrt(fan_in)
        o += n
    assert o == flat.size
