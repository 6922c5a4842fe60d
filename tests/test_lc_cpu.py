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
