"""Autotuner of the step's launch shapes and schedule (sgn_autotune and
sgn_amr_autotune of include/sgn.h / sgn_amr.h) on the GPU.

Every launch-shape option of every tuned kernel and both schedules must give
the default path's results bit for bit (a block shape changes only which
thread computes a value, never how), on grids with ragged tails in both
directions, in FP64 and mixed precision, for SWE, mbHSGN and HSGN.  The default
path is the one checked against the oracle elsewhere, so bit-identity carries
that parity over to every tuning.  Tuning itself must leave the state, time,
next step and status as they were."""
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


def run(S, b, q, steps, choice=None, autotune_after=None, **cfg):
    s = S.Solver(b, **cfg)
    s.set_state(q)
    if choice is not None:
        s.set_tuning(choice)
    if autotune_after is not None:
        s.step(autotune_after)
        ch, ms = s.autotune(reps=3)
        s.step(steps - autotune_after)
    else:
        s.step(steps)
    qg, t = s.get_state()
    return s, qg, t


def same_run(a, b):
    (sa, qa, ta), (sb, qb, tb) = a, b
    assert ta == tb
    assert np.array_equal(qa, qb)
    assert sa.next_dt() == sb.next_dt()
    assert sa.status() == sb.status()
    assert sa.mass() == sb.mass()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("model", [0, 1, 2])
def test_every_option_matches_default(S, model, precision):
    nx, ny = 131, 67
    b, q = W.random_small_case(model, nx, ny, seed=900 + model, dx=0.05, wetdry=True, amp=0.15)
    cfg = dict(model=model, dx=0.05, dy=0.04, bc=(1, 0, 0, 1), h_star=0.6, precision=precision)
    # the kernel sequence with default shapes (a mixed solver starts on the one-pass
    # schedule, which agrees with these to FP32 rounding: tests/test_gpu_fused.py)
    ref = run(S, b, q, 8, choice=[0] * S.TUNE_N, **cfg)
    assert ref[0].status()[0] == 0
    for o in range(S.TUNE_OPTS):
        for sched in (0, 1):
            choice = [o] * (S.TUNE_N - 1) + [sched]
            got = run(S, b, q, 8, choice=choice, **cfg)
            assert got[0].tuning()["schedule"][0] == sched
            same_run(got, ref)


def test_mixed_options_per_slot(S):
    # options differing between slots (each slot's table is read separately)
    model = 2
    b, q = W.random_small_case(model, 97, 113, seed=77, dx=0.05, wetdry=True, amp=0.2)
    cfg = dict(model=model, dx=0.05, bc=(0, 0, 0, 0), h_star=0.6, precision=1)
    ref = run(S, b, q, 10, choice=[0] * S.TUNE_N, **cfg)
    for choice in ([1, 2, 0, 2, 1, 0, 2, 1], [2, 0, 1, 1, 2, 2, 0, 0], [0, 1, 2, 0, 0, 1, 1, 1]):
        same_run(run(S, b, q, 10, choice=choice, **cfg), ref)


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_leaves_the_run_unchanged(S, precision):
    model = 2
    b, q = W.random_small_case(model, 160, 90, seed=31, dx=0.05, wetdry=True, amp=0.2)
    cfg = dict(model=model, dx=0.05, bc=(1, 1, 0, 0), h_star=0.6, precision=precision)
    for k in (4, 0):      # after some steps, and before the first
        got = run(S, b, q, 9, autotune_after=k, **cfg)
        kept = [v[0] for v in got[0].tuning().values()]
        # the same run without tuning: k steps on the default schedule, then the kept one
        s = S.Solver(b, **cfg)
        s.set_state(q)
        s.step(k)
        s.set_tuning(kept)
        s.step(9 - k)
        qr, tr = s.get_state()
        same_run(got, (s, qr, tr))


def test_autotune_report(S):
    b, q = W.random_small_case(2, 300, 200, seed=5, dx=0.05, wetdry=True, amp=0.2)
    s = S.Solver(b, model=2, dx=0.05, h_star=0.6, precision=1)
    s.set_state(q)
    ch, ms = s.autotune(reps=5)
    assert len(ch) == S.TUNE_N
    assert all(0 <= c < S.TUNE_OPTS for c in ch[:-1]) and ch[-1] in (0, 1, 2)
    # every kernel option timed; the schedule slot has three options (the
    # one-pass kernel is built for the mixed path of uniform grids)
    assert (ms[:-1] > 0).all()
    assert (ms[-1] > 0).all()
    # the kept schedule is the fastest whole step measured
    assert ms[-1, ch[-1]] == ms[-1].min()
    # the kept option is the fastest measured (with the one-pass schedule the
    # update slot selects that kernel's rows per block instead)
    for k in range(S.TUNE_N - 1):
        if ch[-1] == 2 and k == 6:
            continue
        assert ms[k, ch[k]] == ms[k].min()
    tun = s.tuning()
    assert [tun[n][0] for n in S.TUNE_SLOTS] == ch
    assert tun["face_x"][1][0] * tun["face_x"][1][1] in (128, 256, 512)
    if ch[-1] == 2:
        assert tun["update"][1][0] == 128 and tun["update"][1][1] in (32, 64, 128, 256)
    assert tun["schedule"][1] == (0, 0)
    s.step(3)
    assert s.status()[0] == 0


def test_tuning_arguments(S):
    b, q = W.random_small_case(1, 40, 30, seed=3, dx=0.05, wetdry=False)
    s = S.Solver(b, model=1, dx=0.05)
    s.set_state(q)
    with pytest.raises(S.SGNError) as e:
        s.set_tuning([0] * 7 + [2])
    assert e.value.code == -1
    with pytest.raises(S.SGNError) as e:
        s.set_tuning([3] + [0] * 7)
    assert e.value.code == -1
    with pytest.raises(S.SGNError) as e:
        s.autotune(reps=0)
    assert e.value.code == -1
    # a rejected tuning leaves the previous one (FP64 solver: schedule 0 by default)
    assert all(v[0] == 0 for v in s.tuning().values())
    # a mixed solver on a grid this small starts on the kernel sequence (the
    # one-pass default on large grids: test_gpu_fused.py); the one-pass schedule
    # is accepted
    s2 = S.Solver(b, model=1, dx=0.05, precision=1)
    assert s2.tuning()["schedule"][0] == 0
    s2.set_tuning([0] * 7 + [2])
    assert s2.tuning()["schedule"][0] == 2


def test_hierarchy_autotune_and_options(S):
    from paper_2606_12162_gb300 import amr
    amr.lib()
    model, nx0, ny0, r = 2, 24, 20, 2
    boxes = W.amr_boxes_small()
    L = len(boxes) + 1
    b, qs = W.amr_small_case(model, nx0, ny0, r, L, seed=10, wetdry=True, amp=0.2)

    def hier(precision):
        g = amr.Hierarchy(b, nx0, ny0, 0.2, r, boxes, model=model, precision=precision, h_star=0.0,
                          dry_tol=1e-3, alpha=3.0)
        g.set_state(qs)
        return g

    def patches(g):
        return [g.get_patch(l, k) for l in range(L) for k in range(g.npatches(l))]

    for precision in (0, 1):
        ref = hier(precision)
        ref.step(6)
        want = patches(ref)
        tuned = hier(precision)
        tuned.step(2)
        ch, ms = tuned.autotune(reps=3)
        assert ch.shape == (L, S.TUNE_N)
        tuned.step(4)
        forced = hier(precision)
        # FP64: the forked kernel sequence with the third shape of every kernel;
        # mixed: the one-pass kernel on every level with 256-row chunks
        forced.set_tuning([[2] * (S.TUNE_N - 1) + [1 if precision == 0 else 2]] * L)
        forced.step(6)
        for g in (tuned, forced):
            got = patches(g)
            assert g.status() == ref.status()
            if precision == 0:
                assert all(np.array_equal(x, y) for x, y in zip(got, want))
                assert g.next_dt() == ref.next_dt()
                assert g.mass() == ref.mass()
            else:
                # the one-pass kernel may replace the sequence on a level: FP32 rounding
                for x, y in zip(got, want):
                    scale = np.abs(y).max(axis=(1, 2)) + 1e-30
                    assert (np.abs(x - y).max(axis=(1, 2)) <= 1e-5 * scale).all()
                assert abs(g.next_dt() - ref.next_dt()) <= 1e-6 * ref.next_dt()
