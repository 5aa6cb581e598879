"""Host logic of the denoiser's training loop (CPU): slab choice, the learning-rate schedule
and the averaging of the last steps' parameters, against a stand-in for the denoiser that
records what the loop asks of it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2509_16793_gb300 import denoise_train


class FakeDenoiser:
    """Parameters move by a known amount per training step: after step i they hold i + 1."""

    def __init__(self, n=5):
        self.p = np.zeros(n, np.float32)
        self.rates = []
        self.slabs = []
        self.installed = []

    def train_step(self, x, t, lr, z_margin=0):
        assert x.shape == t.shape and x.is_contiguous()
        self.slabs.append(x.shape[0])
        self.rates.append(lr)
        self.p = self.p + 1.0
        return float(len(self.rates))

    def params(self):
        return self.p.copy()

    def set_params(self, p):
        self.installed.append(np.array(p))
        self.p = np.array(p, np.float32)


def pairs(n=3, nz=40):
    xs = [torch.full((nz, 3, 2, 2), float(k)) for k in range(n)]
    ts = [torch.full((nz, 3, 2, 2), float(k)) for k in range(n)]
    return xs, ts


def test_schedule_and_slabs():
    den = FakeDenoiser()
    xs, ts = pairs()
    losses = denoise_train.train(den, xs, ts, iters=50, slab=8, lr=1e-3, average_tail=0.0)
    assert len(losses) == 50 and den.slabs == [8] * 50
    # the rate drops tenfold after 80 % of the steps
    assert den.rates[:41] == [1e-3] * 41 and all(r == pytest.approx(1e-4) for r in den.rates[41:])
    # no averaging: the parameters are the last step's
    assert den.installed == [] and np.all(den.p == 50)


def test_average_of_the_tail():
    den = FakeDenoiser()
    xs, ts = pairs()
    denoise_train.train(den, xs, ts, iters=100, slab=8, average_tail=0.2, average_every=10)
    # sampled after steps 89 and 99 (the last step, then every 10th back to step 80):
    # the parameters then held 90 and 100
    assert len(den.installed) == 1
    assert np.allclose(den.installed[0], 95.0)


def test_average_every_step_of_the_tail():
    den = FakeDenoiser()
    xs, ts = pairs()
    denoise_train.train(den, xs, ts, iters=20, slab=8, average_tail=0.25, average_every=1)
    # steps 15..19 sampled: values 16..20
    assert np.allclose(den.installed[0], np.mean(np.arange(16, 21)))
