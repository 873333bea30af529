"""Host-side logic of the Python layer (CPU only): the surrogate training
loop's control flow with a stand-in network that records its calls (the step
schedule of Sec. II-D, halving the rate at epochs 20, 40 and 60; one pass
over a fresh permutation of the pairs per epoch; the mean loss per epoch),
and the size checks the wrappers make before handing pointers to the
library."""
import numpy as np
import torch

from paper_2602_12242_gb300.surrogate import normalizer_stats, train


class Recorder:
    def __init__(self):
        self.lrs, self.seen, self.wd = [], [], set()

    def loss_grad(self, m, h, want_grad=True):
        self.seen.append(m[:, 0, 0, 0, 0].clone())
        return torch.tensor([float(m[:, 0, 0, 0, 0].mean())]), None

    def adam_step(self, lr, weight_decay):
        self.lrs.append(lr)
        self.wd.add(weight_decay)


def test_schedule_batches_and_epoch_losses():
    n, batch, epochs = 12, 4, 70
    M = torch.zeros((n, 1, 2, 2, 4))
    M[:, 0, 0, 0, 0] = torch.arange(n, dtype=torch.float32)
    net = Recorder()
    losses = train(net, M, M.clone(), epochs=epochs, batch=batch, lr=1e-3, weight_decay=1e-4, seed=3)
    steps = n // batch
    assert len(net.lrs) == epochs * steps and net.wd == {1e-4}
    lr_at = [net.lrs[e * steps] for e in range(epochs)]
    assert lr_at[0] == lr_at[19] == 1e-3
    assert lr_at[20] == lr_at[39] == 5e-4
    assert lr_at[40] == 2.5e-4 and lr_at[60] == lr_at[69] == 1.25e-4
    for e in range(epochs):
        seen = torch.cat(net.seen[e * steps:(e + 1) * steps])
        assert sorted(seen.tolist()) == list(range(n))  # every pair once per epoch
        assert abs(losses[e] - float(seen.mean())) < 1e-6
    assert not torch.equal(torch.cat(net.seen[:steps]), torch.cat(net.seen[steps:2 * steps]))


def test_normalizer_statistics_per_component():
    rng = np.random.default_rng(4)
    M = torch.from_numpy(rng.normal(size=(5, 1, 3, 4, 4)).astype(np.float32))
    H = torch.from_numpy(rng.normal(size=(5, 1, 3, 4, 4)).astype(np.float32) * 7 + 2)
    st = normalizer_stats(M, H)
    m = M[..., :3].reshape(-1, 3).double()
    h = H[..., :3].reshape(-1, 3).double()
    ref = m.mean(0).tolist() + m.std(0, unbiased=False).tolist() + h.mean(0).tolist() + \
        h.std(0, unbiased=False).tolist()
    assert np.allclose(st, ref, rtol=1e-12)


class FakeField:
    """Stands in for a CUDA tensor in the wrappers' size checks."""

    def __init__(self, shape, dtype=torch.float32, cuda=True, contiguous=True):
        self.shape, self.dtype, self.is_cuda, self._c = torch.Size(shape), dtype, cuda, contiguous

    def dim(self):
        return len(self.shape)

    def is_contiguous(self):
        return self._c


def test_wrappers_check_field_sizes_before_the_library():
    import pytest
    from paper_2602_12242_gb300.surrogate import _fields
    g = (1, 32, 48)
    assert _fields(g, 4, FakeField((1, 32, 48, 4))) == 1
    assert _fields(g, 4, FakeField((3, 1, 32, 48, 4)), FakeField((3, 1, 32, 48, 4))) == 3
    assert _fields(g, 4, FakeField((1, 32, 48, 4)), FakeField((1, 1, 32, 48, 4))) == 1
    bad = [
        [FakeField((5, 1, 32, 48, 4))],                                   # above max_batch
        [FakeField((0, 1, 32, 48, 4))],                                   # empty batch
        [FakeField((1, 32, 47, 4))],                                      # another grid
        [FakeField((2, 1, 32, 48, 3))],                                   # float3 records
        [FakeField((2, 1, 32, 48, 4)), FakeField((3, 1, 32, 48, 4))],     # batches differ
        [FakeField((1, 32, 48, 4), dtype=torch.float64)],
        [FakeField((1, 32, 48, 4), cuda=False)],
        [FakeField((1, 32, 48, 4), contiguous=False)],
    ]
    for ts in bad:
        with pytest.raises(ValueError):
            _fields(g, 4, *ts)


def test_material_maps_are_checked_against_the_grid():
    import types

    import pytest
    from paper_2602_12242_gb300.solver import Context
    me = types.SimpleNamespace(shape=(2, 3, 4))
    Context._check_map(me, FakeField((2, 3, 4)), ())
    Context._check_map(me, FakeField((2, 3, 4, 4)), (4,))
    for t, rec in [(FakeField((2, 3, 5)), ()), (FakeField((24,)), ()), (FakeField((2, 3, 4, 3)), (4,)),
                   (FakeField((2, 3, 4), dtype=torch.float64), ()), (FakeField((2, 3, 4), cuda=False), ())]:
        with pytest.raises(ValueError):
            Context._check_map(me, t, rec)


def test_checkpoint_round_trip(tmp_path):
    """save_state / load_state keep the field bit for bit (FP32), the time,
    the step count and the metadata."""
    from paper_2602_12242_gb300.solver import load_state, save_state, to_dev4
    rng = np.random.default_rng(8)
    a = rng.normal(size=(2, 3, 5, 3))
    m = to_dev4(a / np.linalg.norm(a, axis=-1, keepdims=True), device="cpu")
    path = tmp_path / "run.npz"
    save_state(path, m, t=1.25e-10, step=2500, meta={"workload": "film", "dt": 5e-14})
    m2, t, step, meta = load_state(path, device="cpu")
    assert torch.equal(m2, m) and m2.shape == (2, 3, 5, 4)
    assert t == 1.25e-10 and step == 2500 and meta == {"workload": "film", "dt": 5e-14}
