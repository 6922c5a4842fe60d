"""State in and out of the solver through the three kinds of buffer the C ABI
accepts: pageable host memory (staged through a device buffer), pinned mapped
host memory (read and written by the conversion kernels in place) and device
memory.  All three must give the same state bit for bit, with field masks."""
import ctypes

import numpy as np
import pytest

from paper_2606_12162_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_12162_gb300 import build, sgn
    build.build()
    sgn.load()
    return sgn


@pytest.mark.parametrize("precision", [0, 1])
def test_pageable_pinned_and_device_buffers_agree(S, precision):
    import torch
    model = 2
    b, q = W.random_small_case(model, 130, 67, seed=17, dx=0.05, wetdry=True, amp=0.2)
    cfg = dict(model=model, dx=0.05, h_star=0.6, precision=precision)
    ref = S.Solver(b, **cfg)
    ref.set_state(q)
    ref.step(6)
    q_ref, t_ref = ref.get_state()

    pin = S.Solver(b, **cfg)
    hq = torch.from_numpy(q.copy()).pin_memory()
    pin.set_state_ptr(hq.data_ptr())
    pin.step(6)
    out = torch.zeros(q.shape, dtype=torch.float64).pin_memory()
    pin.get_state_ptr(out.data_ptr(), out.numel())
    assert np.array_equal(out.numpy(), q_ref)
    # a field mask into pinned memory: eta and hv, packed
    sel = torch.zeros((2,) + q.shape[1:], dtype=torch.float64).pin_memory()
    rc = S.load().sgn_get_state(pin.h, 0b101, ctypes.cast(sel.data_ptr(), S.DP), sel.numel(), None)
    assert rc == 0
    assert np.array_equal(sel.numpy()[0], q_ref[0]) and np.array_equal(sel.numpy()[1], q_ref[2])
    # too small a pinned buffer is rejected before anything is written
    rc = S.load().sgn_get_state(pin.h, 0b101, ctypes.cast(sel.data_ptr(), S.DP), sel.numel() - 1, None)
    assert rc == -9

    dev = S.Solver(b, **cfg)
    dq = torch.from_numpy(q.copy()).cuda()
    dev.set_state_device(dq)
    dev.step(6)
    dout = torch.zeros_like(dq)
    dev.get_state_device(dout)
    torch.cuda.synchronize()
    assert np.array_equal(dout.cpu().numpy(), q_ref)
    assert pin.next_dt() == ref.next_dt() == dev.next_dt()
