"""Pins of the FP64 NumPy reference of the corrector network (oracle/conv_ref.py):
its gradients against central finite differences of its own loss, and its
BF16 rounding against PyTorch's float32 -> bfloat16 conversion."""
import numpy as np

from oracle import conv_ref as R


def test_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    layers = R.layers_of(3, 4, 3, 2 * 2 * 2)
    n = sum(ci * co * 9 + co for ci, co in layers)
    p = rng.standard_normal(n) * 0.3
    x = rng.standard_normal((3, 5, 6))
    t = rng.standard_normal((2, 10, 12))
    fw = (1.0, 0.5)
    loss, g = R.loss_and_grad(p, layers, x, t, 2, 2, fw)
    idx = rng.choice(n, size=40, replace=False)
    for i in idx:
        e = np.zeros(n)
        e[i] = 1e-6
        lp, _ = R.loss_and_grad(p + e, layers, x, t, 2, 2, fw)
        lm, _ = R.loss_and_grad(p - e, layers, x, t, 2, 2, fw)
        fd = (lp - lm) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * (1 + abs(g[i])), (i, fd, g[i])


def test_shuffle_roundtrip_and_bf16():
    import torch
    rng = np.random.default_rng(1)
    y = rng.standard_normal((3 * 16, 4, 5))
    assert np.array_equal(R.unshuffle(R.shuffle(y, 4, 3), 4, 3), y)
    a = rng.standard_normal(10000).astype(np.float32) * 10.0 ** rng.integers(-5, 5, 10000)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(R.bf16_round(a), ref)


class _FakeSolver:
    """Host stand-in for a solver: CFL steps of about 3.4 s that drop now and
    then to a small fraction (a thin layer running up a shore)."""

    def __init__(self, seed):
        self.t, self.last = 0.0, 0.0
        self.rng = np.random.default_rng(seed)
        self.nd, self.courant = 3.4, 0.0

    def _roll(self):
        self.nd = 3.4 if self.rng.random() > 0.1 else 3.4 * self.rng.uniform(0.05, 1.0)

    def next_dt(self):
        return self.nd

    def step(self, k):
        for _ in range(k):
            self.t += self.nd
            self.last = self.nd
            self._roll()
        return self.t

    def step_dt(self, h):
        self.courant = max(self.courant, h / self.nd)
        self.t += h
        self.last = h
        self._roll()

    def status(self):
        return 0, self.last, 0.0


def test_advance_to_hits_output_times_within_the_cfl_step():
    from paper_2606_12162_gb300 import corrector
    for seed in range(100):
        sv = _FakeSolver(seed)
        t = 0.0
        for T in (60.0, 120.0, 180.0, 240.0, 300.0):
            t, n = corrector.advance_to(sv, t, T)
            assert t == T and abs(sv.t - T) < 1e-6 and n > 0
        assert sv.courant <= 1.0 + 1e-12
