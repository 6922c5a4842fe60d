"""The one-pass step (schedule 2 of sgn_set_tuning: k_step_fused, the whole
mixed-precision step in one launch) on the GPU.

It computes the same quantities over the same index ranges as the kernel
sequence of the default schedule, with the same device functions; the compiler
may contract a different set of multiply-adds, so the two agree to FP32
rounding, not bit for bit.  Checked on grids that span several strips and row
chunks with ragged tails, for every boundary kind, wet/dry bathymetry, SWE,
mbHSGN and HSGN, and each of its row counts: same time, same next time step to
1e-6, every field within 1e-5 of its largest magnitude after a few steps (a
wrong index or a missed face shows at 1e-2 or more).  The one-pass path is also
compared with the FP64 oracle directly, within the mixed-precision tolerances."""
import numpy as np
import pytest

from paper_2606_12162_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FUSED = 2


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_12162_gb300 import build, sgn
    build.build()
    sgn.load()
    return sgn


def run(S, b, q, steps, choice=None, gauges=None, **cfg):
    s = S.Solver(b, precision=1, **cfg)
    if choice is not None:
        s.set_tuning(choice)
    s.set_state(q)
    if gauges is not None:
        s.add_gauges(gauges, steps + 2)
    s.step(steps)
    qg, t = s.get_state()
    return s, qg, t


def close(a, b, rel=1e-5):
    scale = np.abs(b).max(axis=(1, 2)) + 1e-30
    return bool((np.abs(a - b).max(axis=(1, 2)) <= rel * scale).all())


def fused_choice(rows_opt=0):
    ch = [0] * 8
    ch[6] = rows_opt
    ch[7] = FUSED
    return ch


CASES = [
    # model, nx, ny, bc, wetdry, steps
    (2, 300, 270, (0, 1, 2, 2), True, 12),    # 3 strips, 3 chunks, ragged tails, periodic in y
    (1, 130, 140, (1, 1, 0, 0), True, 10),
    (0, 250, 70, (2, 2, 0, 1), True, 10),
    (2, 122, 128, (0, 0, 0, 0), False, 15),   # exactly one strip and one chunk
    (2, 123, 129, (1, 0, 1, 0), True, 9),     # one column / row past them
    (1, 61, 300, (2, 2, 1, 0), True, 8),
    (2, 5, 3, (1, 0, 1, 0), False, 8),
    (2, 2, 2, (0, 0, 0, 0), False, 5),
]


@pytest.mark.parametrize("model,nx,ny,bc,wetdry,steps", CASES)
def test_fused_equals_kernel_sequence(S, model, nx, ny, bc, wetdry, steps):
    b, q = W.random_small_case(model, nx, ny, seed=3 * nx + ny + model, dx=0.05, wetdry=wetdry, amp=0.15)
    cfg = dict(model=model, dx=0.05, dy=0.04, bc=bc, h_star=0.6)
    g = np.array([[0.05 * nx * 0.3, 0.04 * ny * 0.6], [0.05 * nx * 0.9, 0.04 * ny * 0.1]])
    ref = run(S, b, q, steps, choice=[0] * 8, gauges=g, **cfg)   # the kernel sequence
    assert ref[0].status()[0] == 0
    for opt in range(3):
        got = run(S, b, q, steps, choice=fused_choice(opt), gauges=g, **cfg)
        assert got[0].tuning()["schedule"][0] == FUSED
        (sa, qa, ta), (sb, qb, tb) = got, ref
        assert close(qa, qb), (opt, np.abs(qa - qb).max(axis=(1, 2)))
        assert abs(ta - tb) <= 1e-6 * tb
        assert abs(sa.next_dt() - sb.next_dt()) <= 1e-6 * sb.next_dt()
        assert sa.status()[0] == sb.status()[0] == 0
        assert abs(sa.mass() - sb.mass()) <= 1e-6 * sb.mass()
        ga, gb = sa.gauges(), sb.gauges()
        assert ga.shape == gb.shape and np.abs(ga - gb).max() <= 1e-5 * (1 + np.abs(gb).max())


def test_fused_limiters_and_lie(S):
    b, q = W.random_small_case(2, 140, 150, seed=5, dx=0.05, wetdry=True, amp=0.2)
    for limiter, strang in ((0, 1), (2, 1), (1, 0)):
        cfg = dict(model=2, dx=0.05, bc=(0, 1, 0, 1), h_star=0.6, limiter=limiter, strang=strang)
        ref = run(S, b, q, 10, choice=[0] * 8, **cfg)
        got = run(S, b, q, 10, choice=fused_choice(1), **cfg)
        assert close(got[1], ref[1]) and abs(got[2] - ref[2]) <= 1e-6 * ref[2]


def test_fused_against_oracle(S, oracle_mod):
    """The one-pass path against the FP64 oracle: the mixed tolerances of the
    default path (relative L2 over wet cells: eta 1e-5, hu, hv 1e-3)."""
    b, q = W.random_small_case(2, 250, 190, seed=12, dx=0.05, wetdry=True, amp=0.15)
    cfg = dict(dx=0.05, model=2, bc=(0, 0, 0, 0), h_star=0.6)
    s, qg, tg = run(S, b, q, 40, choice=fused_choice(0), **cfg)
    o = oracle_mod.Oracle(b, **cfg)
    o.set_state(q)
    assert o.step(40) == 0
    qo, to = o.get_state()
    wet = (qo[0] - b) > 1e-3
    err = []
    for k in range(3):
        x, y = qg[k][wet], qo[k][wet]
        err.append(np.linalg.norm(x - y) / np.linalg.norm(y))
    assert err[0] <= 1e-5 and err[1] <= 1e-3 and err[2] <= 1e-3, err
    assert abs(tg - to) <= 1e-5 * to


def test_fused_is_the_mixed_default_on_large_grids(S):
    """A new mixed solver runs the one-pass step when the grid gives the device
    enough tiles (1024 x 1024 does on a GB300, with 32-row chunks), the kernel
    sequence on small grids (140 x 90)."""
    b, q = W.random_small_case(2, 140, 90, seed=2, dx=0.05, wetdry=True, amp=0.15)
    s = S.Solver(b, model=2, dx=0.05, precision=1, h_star=0.6)
    assert s.tuning()["schedule"][0] == 0
    b = np.full((1024, 1024), -50.0)
    s = S.Solver(b, model=2, dx=10.0, precision=1, h_star=20.0)
    t = s.tuning()
    assert t["schedule"][0] == FUSED and t["update"][1] == (128, 32)
    assert s.launches_per_step() == 2


def test_fused_rejected_where_not_built(S):
    b, q = W.random_small_case(2, 40, 30, seed=1, dx=0.05, wetdry=False)
    s = S.Solver(b, model=2, dx=0.05, precision=0)   # FP64: the one-pass kernel is FP32 only
    with pytest.raises(S.SGNError):
        s.set_tuning(fused_choice(0))


def test_fused_autotune_keeps_run(S):
    """Autotuning with the one-pass schedule among the candidates leaves the
    state, time and status as they were; the run continues on the kept schedule
    (the one-pass schedule agrees with the others to FP32 rounding)."""
    b, q = W.random_small_case(2, 260, 200, seed=44, dx=0.05, wetdry=True, amp=0.15)
    cfg = dict(model=2, dx=0.05, bc=(1, 1, 1, 1), h_star=0.6)
    ref = run(S, b, q, 12, choice=[0] * 8, **cfg)
    s = S.Solver(b, precision=1, **cfg)
    s.set_state(q)
    s.step(4)
    ch, ms = s.autotune(reps=2)
    assert ms[7, 2] > 0          # the one-pass schedule was timed
    s.step(8)
    qg, t = s.get_state()
    assert close(qg, ref[1]) and abs(t - ref[2]) <= 1e-6 * ref[2]
