"""Refined hierarchy on the GPU (include/sgn_amr.h, batched atlas kernels)
against the plain refinement oracle (oracle/amr_oracle.py), patch by patch.

FP64: per-field relative L2 <= 1e-12 on every patch, and the next level-0
step, the mass and the clipped water to 1e-12.  Mixed precision: per-field
tolerances as for the uniform grid.  Also: one level equals the uniform GPU
solver bit for bit, lake at rest, and mass up to the reported clipping."""
import numpy as np
import pytest

from paper_2606_12162_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
CFG = dict(h_star=0.0, dry_tol=1e-3, alpha=3.0)
BOXES_R4 = [[(8, 8, 24, 16), (32, 8, 16, 16), (0, 32, 16, 16)], [(48, 48, 32, 32)]]


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_12162_gb300 import amr, build
    build.build()
    amr.lib()
    return amr


@pytest.fixture(scope="module")
def A(oracle_mod):
    from oracle import amr_oracle
    return amr_oracle


def rel_l2(a, b):
    out = []
    for k in range(a.shape[0]):
        den = np.linalg.norm(b[k])
        num = np.linalg.norm(a[k] - b[k])
        out.append(num / den if den > 0 else num)
    return np.array(out)


def run_pair(M, A, model, nx0, ny0, r, boxes, seed, steps, precision=0, wetdry=True, bc=(0, 0, 0, 0), amp=0.2,
             dx0=0.2):
    L = len(boxes) + 1
    b, qs = W.amr_small_case(model, nx0, ny0, r, L, seed=seed, wetdry=wetdry, amp=amp, dx0=dx0)
    g = M.Hierarchy(b, nx0, ny0, dx0, r, boxes, model=model, bc=bc, precision=precision, **CFG)
    g.set_state(qs)
    o = A.AmrOracle(b, nx0, ny0, dx0, r, boxes, model=model, bc=bc, **CFG)
    o.set_state(qs)
    assert abs(g.next_dt() - o.dt_next) <= 1e-6 * o.dt_next
    g.step(steps)
    assert o.step(steps) == 0
    return g, o, b


@pytest.mark.parametrize("model,nx0,ny0,r,boxes,seed,steps,wetdry", [
    (2, 24, 20, 2, W.amr_boxes_small(), 4, 10, True),
    (1, 24, 20, 2, W.amr_boxes_small(), 5, 10, False),
    (2, 16, 12, 4, BOXES_R4, 6, 6, True),
    (0, 24, 20, 2, W.amr_boxes_small(), 7, 10, True),
])
def test_fp64_hierarchy_against_oracle(M, A, model, nx0, ny0, r, boxes, seed, steps, wetdry):
    g, o, _ = run_pair(M, A, model, nx0, ny0, r, boxes, seed, steps, wetdry=wetdry)
    for l in range(g.L):
        for k in range(len(g.boxes[l])):
            err = rel_l2(g.get_patch(l, k), o.patch_state(l, k))
            assert (err <= FP64_TOL).all(), (l, k, err)
    assert abs(g.next_dt() - o.dt_next) <= FP64_TOL * o.dt_next
    m, c = g.mass()
    mo = o.mass()
    assert abs(m - mo) <= FP64_TOL * mo
    assert abs(c - o.clipped) <= FP64_TOL * mo
    assert g.status() == 0
    assert g.launches_per_step() > 0


def test_fixed_step_and_fine_level_covering_the_domain(M, A):
    nx0, ny0, r = 12, 10, 2
    boxes = [[(0, 0, nx0 * r, ny0 * r)]]
    b, qs = W.amr_small_case(2, nx0, ny0, r, 2, seed=8)
    g = M.Hierarchy(b, nx0, ny0, 0.2, r, boxes, model=2, **CFG)
    g.set_state(qs)
    o = A.AmrOracle(b, nx0, ny0, 0.2, r, boxes, model=2, **CFG)
    o.set_state(qs)
    dt = 0.5 * o.dt_next
    for _ in range(3):
        g.step_dt(dt)
        assert o.step_dt(dt) == 0
    for l in range(2):
        assert (rel_l2(g.get_patch(l, 0), o.patch_state(l, 0)) <= FP64_TOL).all()


def test_one_level_equals_the_uniform_solver(M):
    from paper_2606_12162_gb300 import sgn
    b, qs = W.amr_small_case(2, 40, 30, 2, 1, seed=9)
    g = M.Hierarchy(b, 40, 30, 0.1, 2, [], model=2, bc=(0, 1, 1, 0), **CFG)
    g.set_state(qs)
    s = sgn.Solver(b, model=2, dx=0.1, bc=(0, 1, 1, 0), **CFG)
    s.set_state(qs[0])
    assert g.next_dt() == s.next_dt()
    g.step(7)
    s.step(7)
    assert np.array_equal(g.get_patch(0, 0), s.get_state()[0])


def test_mixed_hierarchy_against_fp64_oracle(M, A):
    g, o, b = run_pair(M, A, 2, 24, 20, 2, W.amr_boxes_small(), 10, 10, precision=1, wetdry=False, amp=0.15)
    for l in range(g.L):
        for k in range(len(g.boxes[l])):
            err = rel_l2(g.get_patch(l, k)[:3], o.patch_state(l, k)[:3])
            assert err[0] <= 1e-5 and err[1] <= 1e-3 and err[2] <= 1e-3, (l, k, err)


def seq_choice(L, sched=0):
    """The same schedule on every level (default shapes): 0 the kernel
    sequence, 2 the one-pass kernel."""
    ch = [0] * 8
    ch[7] = sched
    return [ch] * L


@pytest.mark.parametrize("model,nx0,ny0,r,boxes,seed,steps", [
    (2, 24, 20, 2, W.amr_boxes_small(), 11, 10),
    (1, 16, 12, 4, BOXES_R4, 12, 6),
    (0, 24, 20, 2, W.amr_boxes_small(), 13, 10),
])
def test_mixed_one_pass_hierarchy_equals_kernel_sequence(M, A, model, nx0, ny0, r, boxes, seed, steps):
    """Mixed precision steps a level with ONE launch of the one-pass kernel
    (the default where the level's atlas is large enough; forced on every level
    here): three-cell frames, the positivity factors of sibling ghosts computed
    in the frame, the coarse/fine face fluxes exported by the kernel.
    Against the same hierarchy stepped by the kernel sequence (sibling factors
    copied, fluxes read from the face planes): every patch within 1e-5 of its
    field's largest magnitude, the next step to 1e-6, mass up to the clipped
    water to FP32 rounding in both (a positivity factor that differed between
    the two sides of a sibling face would move mass), against the FP64 oracle
    within the mixed tolerances, and fewer launches per level-0 step."""
    L = len(boxes) + 1
    b, qs = W.amr_small_case(model, nx0, ny0, r, L, seed=seed, wetdry=True, amp=0.2)

    def run(choice):
        g = M.Hierarchy(b, nx0, ny0, 0.2, r, boxes, model=model, precision=1, **CFG)
        if choice is not None:
            g.set_tuning(choice)
        g.set_state(qs)
        m0, _ = g.mass()
        g.step(steps)
        return g, m0

    f, m0 = run(seq_choice(L, 2))
    q, _ = run(seq_choice(L))
    for l in range(L):
        for k in range(len(f.boxes[l])):
            pf, pq = f.get_patch(l, k), q.get_patch(l, k)
            scale = np.abs(pq).max(axis=(1, 2)) + 1e-30
            assert (np.abs(pf - pq).max(axis=(1, 2)) <= 1e-5 * scale).all(), (l, k)
    assert abs(f.next_dt() - q.next_dt()) <= 1e-6 * q.next_dt()
    for g in (f, q):
        m, c = g.mass()
        assert abs(m - m0 - c) <= 2e-6 * m0, (m, m0, c)
        assert g.status() == 0
    assert f.launches_per_step() < q.launches_per_step()
    o = A.AmrOracle(b, nx0, ny0, 0.2, r, boxes, model=model, bc=(0, 0, 0, 0), **CFG)
    o.set_state(qs)
    assert o.step(steps) == 0
    for l in range(L):
        for k in range(len(f.boxes[l])):
            err = rel_l2(f.get_patch(l, k)[:3], o.patch_state(l, k)[:3])
            assert err[0] <= 1e-5 and err[1] <= 1e-3 and err[2] <= 1e-3, (l, k, err)


def test_hierarchy_levels_mix_schedules(M):
    """Each level runs its own schedule: the one-pass kernel on some levels and
    the kernel sequence on others (both export the same coarse/fine fluxes and
    give sibling ghosts the same positivity factors) agrees with either alone
    to FP32 rounding; FP64 rejects the one-pass kernel on any level."""
    b, qs = W.amr_small_case(2, 24, 20, 2, 3, seed=14)
    fused = [0] * 7 + [2]

    def run(choice):
        g = M.Hierarchy(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, precision=1, **CFG)
        g.set_tuning(choice)
        g.set_state(qs)
        g.step(8)
        return [g.get_patch(l, k) for l in range(3) for k in range(len(g.boxes[l]))]

    ref = run(seq_choice(3))
    for choice in ([fused, [0] * 8, fused], [[0] * 8, fused, [0] * 8]):
        got = run(choice)
        for x, y in zip(got, ref):
            scale = np.abs(y).max(axis=(1, 2)) + 1e-30
            assert (np.abs(x - y).max(axis=(1, 2)) <= 1e-5 * scale).all()
    d = M.Hierarchy(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, precision=0, **CFG)
    with pytest.raises(Exception):
        d.set_tuning([[0] * 8, [0] * 8, fused])


@pytest.mark.parametrize("precision", [0, 1])
def test_retake_of_a_level0_step_over_the_cfl_limit(M, precision):
    """A level-0 step of 2.5 times the CFL step breaks the limit (SGN_ECFL
    without retaking).  With retaking the step is undone -- the states of all
    levels, time, clipped water and status as before it -- and taken again with
    dt0 * CFL / Courant: the result equals a direct step of that size bit for
    bit (FP64, and mixed precision with the one-pass kernel on every level),
    the time advances by that step, and the run goes on; the setting and the
    count carry over a regrid."""
    from paper_2606_12162_gb300 import sgn
    b, qs = W.amr_small_case(2, 24, 20, 2, 3, seed=15)

    def mk():
        g = M.Hierarchy(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, precision=precision, **CFG)
        if precision == 1:
            g.set_tuning(seq_choice(3, 2))
        g.set_state(qs)
        return g

    g0 = mk()
    dt = g0.next_dt()
    with pytest.raises(sgn.SGNError):
        g0.step_dt(2.5 * dt)
    g1 = mk()
    with pytest.raises(sgn.SGNError):
        g1.set_retake(17)
    g1.set_retake(4)
    g1.step_dt(2.5 * dt)
    t1 = g1.step(0)
    assert 0.0 < t1 < 1.2 * dt and g1.retakes() >= 1 and g1.status() == 0
    g2 = mk()
    g2.step_dt(t1)
    assert g2.step(0) == t1
    for l in range(3):
        for k in range(len(g1.boxes[l])):
            assert np.array_equal(g1.get_patch(l, k), g2.get_patch(l, k)), (l, k)
    assert g1.mass() == g2.mass() and g1.next_dt() == g2.next_dt()
    n = g1.retakes()
    g1.regrid(b, W.amr_boxes_small())
    assert g1.retakes() == n
    g1.step(3)
    assert g1.status() == 0


def test_config4_kind_hierarchy_mixed_against_fp64(M):
    """Config 4 at a quarter of its level-0 size (256^2 at 2 km, ratio 4, three
    levels over the fractal bathymetry and coast strip) with the patches on the
    source (a disk of 60 km around the 2 m uplift: 14 + 197 patches of
    16..128 cells in regions): the mixed hierarchy, every level on the one-pass
    kernel, against the FP64 hierarchy (oracle-equal on the small cases) over
    six level-0 steps of the same dt.  Per level over all patches: relative L2
    of eta <= 1e-5 and of hu, hv <= 1e-3, largest eta difference <= 1e-3 of
    the uplift; masses within 1e-6; no status flag."""
    boxes = W.config4_boxes(256, 4, 3, centre=(0.45, 0.5), radius=30e3, width=60e3, dx0=2000.0)
    c = W.config4(n0=256, boxes=boxes)

    def hier(precision):
        g = M.Hierarchy(c["b"], 256, 256, c["dx0"], 4, c["boxes"], model=2, bc=c["bc"], precision=precision,
                        alpha=c["alpha"], h_star=c["h_star"], cfl=c["cfl"], dry_tol=c["dry_tol"])
        for l, lv in enumerate(c["states"]):
            for k, q in enumerate(lv):
                g.set_patch(l, k, q)
        return g
    g64, gm = hier(0), hier(1)
    gm.set_tuning([[0] * 7 + [2]] * 3)
    for _ in range(6):
        dt = g64.next_dt()
        g64.step_dt(dt)
        gm.step_dt(dt)
    assert g64.status() == 0 and gm.status() == 0
    assert gm.launches_per_step() < g64.launches_per_step()
    for l in range(3):
        a = np.concatenate([g64.get_patch(l, k).reshape(7, -1) for k in range(g64.npatches(l))], axis=1)
        m = np.concatenate([gm.get_patch(l, k).reshape(7, -1) for k in range(gm.npatches(l))], axis=1)
        err = [np.linalg.norm(m[f] - a[f]) / np.linalg.norm(a[f]) for f in range(3)]
        assert err[0] <= 1e-5 and err[1] <= 1e-3 and err[2] <= 1e-3, (l, err)
        assert np.abs(m[0] - a[0]).max() <= 1e-3 * 2.0, l
    m64, mm = g64.mass()[0], gm.mass()[0]
    assert abs(mm - m64) <= 1e-6 * m64


def test_lake_at_rest_and_mass(M, A):
    b, qs = W.amr_small_case(2, 24, 20, 2, 3, seed=3, wetdry=False)
    rest = []
    for l in range(3):
        bl = b
        for _ in range(2 - l):
            bl = A.block_mean(bl, 2)
        z = np.zeros_like(qs[l])
        z[0] = np.maximum(bl, 0.0)
        rest.append(z)
    g = M.Hierarchy(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, bc=(0, 0, 1, 1), **CFG)
    g.set_state(rest)
    g.step(5)
    for l in range(3):
        for k in range(len(g.boxes[l])):
            assert np.abs(g.get_patch(l, k)[1:]).max() <= 1e-14
    # mass with walls over wet/dry bathymetry, up to the reported clipping
    b, qs = W.amr_small_case(2, 24, 20, 2, 3, seed=4, amp=0.3)
    g = M.Hierarchy(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, **CFG)
    g.set_state(qs)
    m0, _ = g.mass()
    g.step(12)
    m, c = g.mass()
    assert abs(m - m0 - c) <= 1e-12 * m0


def test_invalid_hierarchies_are_rejected(M):
    from paper_2606_12162_gb300 import sgn
    b, _ = W.amr_small_case(2, 24, 20, 2, 2, seed=1)
    for boxes in ([[(1, 8, 16, 12)]],                        # not aligned to parent cells
                  [[(8, 8, 16, 12), (16, 12, 8, 8)]],        # overlapping
                  [[(40, 8, 16, 8)]],                        # beyond the domain
                  [[(2, 2, 8, 8)]]):                         # one parent cell from the edge
        with pytest.raises(sgn.SGNError):
            M.Hierarchy(b, 24, 20, 0.2, 2, boxes, model=2, **CFG)


@pytest.mark.parametrize("model,seed,wetdry", [(2, 21, True), (0, 22, True), (1, 23, False)])
def test_regrid_against_oracle(M, A, model, seed, wetdry):
    """sgn_amr_regrid (reading A11) against the oracle's regrid: step, move
    the patches, step on; every patch, next dt, time, mass and clipped water."""
    nx0, ny0, r = 24, 20, 2
    b, qs = W.amr_small_case(model, nx0, ny0, r, 3, seed=seed, wetdry=wetdry, amp=0.25)
    g = M.Hierarchy(b, nx0, ny0, 0.2, r, W.amr_boxes_small(), model=model, **CFG)
    g.set_state(qs)
    o = A.AmrOracle(b, nx0, ny0, 0.2, r, W.amr_boxes_small(), model=model, **CFG)
    o.set_state(qs)
    g.step(4)
    assert o.step(4) == 0
    g.regrid(b, W.amr_boxes_small_moved())
    o.regrid(W.amr_boxes_small_moved())
    assert abs(g.next_dt() - o.dt_next) <= FP64_TOL * o.dt_next
    for l in range(g.L):
        for k in range(len(g.boxes[l])):
            err = rel_l2(g.get_patch(l, k), o.patch_state(l, k))
            assert (err <= FP64_TOL).all(), ("after regrid", l, k, err)
    t = g.step(5)
    assert o.step(5) == 0
    assert abs(t - o.t) <= FP64_TOL * o.t
    for l in range(g.L):
        for k in range(len(g.boxes[l])):
            err = rel_l2(g.get_patch(l, k), o.patch_state(l, k))
            assert (err <= FP64_TOL).all(), (l, k, err)
    assert abs(g.next_dt() - o.dt_next) <= FP64_TOL * o.dt_next
    m, c = g.mass()
    assert abs(m - o.mass()) <= FP64_TOL * o.mass()
    assert abs(c - o.clipped) <= FP64_TOL * o.mass()
    assert g.status() == 0


def test_regrid_out_of_device_memory_keeps_the_hierarchy(M):
    """A regrid's new hierarchy takes over the old one's level-0 solver (level
    0 does not change).  If it then runs out of device memory -- the allocator
    refuses after the first n allocations of the regrid, for several n, so the
    failure comes at different points of its set-up and state transfer -- the
    call returns SGN_ENOMEM and gives level 0 back with its own kind and
    export planes: the old hierarchy steps on exactly as one that never tried
    the regrid."""
    from paper_2606_12162_gb300 import sgn
    nx0, ny0, r = 24, 20, 2
    b, qs = W.amr_small_case(2, nx0, ny0, r, 3, seed=24, amp=0.25)
    moved = W.amr_boxes_small_moved()

    def make():
        g = M.Hierarchy(b, nx0, ny0, 0.2, r, W.amr_boxes_small(), model=2, precision=1, **CFG)
        g.set_state(qs)
        return g
    ref = make()
    ref.step(6)
    failed = 0
    for n in (0, 3, 12, 30, 60, 120):
        g = make()
        g.step(3)
        g._alloc.allow = n
        try:
            g.regrid(b, moved)
            g._alloc.allow = None
            continue                      # enough memory: the regrid went through
        except sgn.SGNError as e:
            assert e.code == -2           # SGN_ENOMEM
        g._alloc.allow = None
        failed += 1
        g.step(3)
        for l in range(3):
            for k in range(len(g.boxes[l])):
                assert np.array_equal(g.get_patch(l, k), ref.get_patch(l, k)), (n, l, k)
        assert g.next_dt() == ref.next_dt() and g.mass() == ref.mass() and g.status() == 0
    assert failed >= 3


def test_regrid_same_boxes_bitwise_and_invalid_rejected(M):
    from paper_2606_12162_gb300 import sgn
    nx0, ny0, r = 24, 20, 2
    b, qs = W.amr_small_case(2, nx0, ny0, r, 3, seed=24, amp=0.25)

    def make():
        g = M.Hierarchy(b, nx0, ny0, 0.2, r, W.amr_boxes_small(), model=2, precision=1, **CFG)
        g.set_state(qs)
        return g
    ref = make()
    ref.step(8)
    g = make()
    g.step(3)
    with pytest.raises(sgn.SGNError) as e:
        g.regrid(b, [[(1, 8, 16, 12)], []])                  # not aligned: rejected, old hierarchy kept
    assert e.value.code == -1
    g.step(2)
    g.regrid(b, W.amr_boxes_small())
    g.step(3)
    for l in range(3):
        for k in range(len(g.boxes[l])):
            assert np.array_equal(g.get_patch(l, k), ref.get_patch(l, k))
    assert g.next_dt() == ref.next_dt()
    assert g.mass() == ref.mass()


def test_mixed_regrid_against_fp64_oracle(M, A):
    nx0, ny0, r = 24, 20, 2
    b, qs = W.amr_small_case(2, nx0, ny0, r, 3, seed=25, wetdry=False, amp=0.15)
    g = M.Hierarchy(b, nx0, ny0, 0.2, r, W.amr_boxes_small(), model=2, precision=1, **CFG)
    g.set_state(qs)
    o = A.AmrOracle(b, nx0, ny0, 0.2, r, W.amr_boxes_small(), model=2, **CFG)
    o.set_state(qs)
    g.step(5)
    assert o.step(5) == 0
    g.regrid(b, W.amr_boxes_small_moved())
    o.regrid(W.amr_boxes_small_moved())
    g.step(5)
    assert o.step(5) == 0
    for l in range(g.L):
        for k in range(len(g.boxes[l])):
            err = rel_l2(g.get_patch(l, k)[:3], o.patch_state(l, k)[:3])
            assert err[0] <= 1e-5 and err[1] <= 1e-3 and err[2] <= 1e-3, (l, k, err)


@pytest.mark.parametrize("precision", [0, 1])
def test_flagged_regrid_tracks_like_the_oracle(M, A, precision):
    """sgn_amr_regrid_flagged (reading A12) every four level-0 steps on a
    travelling solitary wave: the same boxes as the oracle's flag rule at every
    regrid (FP64: bit for bit; mixed: where no jump is within 1e-4 of the
    threshold), and the same states (FP64 1e-12; mixed within the hierarchy
    tolerances)."""
    nx0, ny0, r, dx0, H = 96, 8, 2, 0.4, 1.0
    xf, yf = W.cell_centres(nx0 * r, ny0 * r, dx0 / r, dx0 / r)
    bf = np.full(xf.shape, -H)
    qf = W.soliton_state(2, xf, yf, bf, 0.3, H, 10.0)
    qs = [qf.reshape(qf.shape[0], ny0, r, nx0, r).mean(axis=(2, 4)), qf]
    boxes0 = [[(36, 0, 28, 16)]]
    g = M.Hierarchy(bf, nx0, ny0, dx0, r, boxes0, model=2, precision=precision, **CFG)
    g.set_state(qs)
    o = A.AmrOracle(bf, nx0, ny0, dx0, r, boxes0, model=2, **CFG)
    o.set_state(qs)
    tol, moved = 0.01, 0
    for it in range(6):
        g.step(4)
        assert o.step(4) == 0
        ob = o.flag_boxes(tol, 4, 2)
        e = o.patch_state(0, 0)[0]
        near = np.abs(np.abs(np.diff(e, axis=1)) - tol).min()
        nb = g.regrid_flagged(bf, tol, 4, 2)
        if precision == 0 or near > 1e-4:
            assert g.boxes[1] == ob[0], it
        o.regrid(g.boxes[1:])
        assert nb == [len(g.boxes[1])]
        moved += g.boxes[1] != boxes0[0]
        for k in range(len(g.boxes[1])):
            err = rel_l2(g.get_patch(1, k), o.patch_state(1, k))
            if precision == 0:
                assert (err <= FP64_TOL).all(), (it, k, err)
            else:
                assert err[0] <= 1e-5 and err[1] <= 1e-3, (it, k, err)
    assert moved > 0
    assert g.status() == 0


def test_regrid_arguments_and_boxes_query(M):
    """sgn_amr_get_boxes reports the boxes of every level (EINVAL for a bad
    level, ERANGE for a short buffer); sgn_amr_regrid_flagged rejects a
    non-positive threshold, a zero tile and a negative buffer, and a one-level
    hierarchy, leaving the hierarchy as it was."""
    import ctypes
    from paper_2606_12162_gb300 import amr, sgn
    nx0, ny0, r = 24, 20, 2
    b, qs = W.amr_small_case(2, nx0, ny0, r, 3, seed=31, amp=0.2)
    g = M.Hierarchy(b, nx0, ny0, 0.2, r, W.amr_boxes_small(), model=2, **CFG)
    g.set_state(qs)
    assert g.get_boxes(0) == [(0, 0, nx0, ny0)]
    assert g.get_boxes(1) == list(W.amr_boxes_small()[0])
    assert g.get_boxes(2) == list(W.amr_boxes_small()[1])
    L = amr.lib()
    assert L.sgn_amr_get_boxes(g.h, 3, None, 0) == -1
    buf = (ctypes.c_int * 8)()
    assert L.sgn_amr_get_boxes(g.h, 1, buf, 2) == -9
    before = [g.get_patch(l, k) for l in range(3) for k in range(g.npatches(l))]
    for tol, tile, buffer in ((0.0, 4, 2), (0.01, 0, 2), (0.01, 4, -1)):
        with pytest.raises(sgn.SGNError) as e:
            g.regrid_flagged(b, tol, tile, buffer)
        assert e.value.code == -1
    after = [g.get_patch(l, k) for l in range(3) for k in range(g.npatches(l))]
    assert all(np.array_equal(x, y) for x, y in zip(before, after))
    g.step(2)
    assert g.status() == 0
    with pytest.raises(sgn.SGNError):
        M.Hierarchy(b[::4, ::4], nx0, ny0, 0.2, r, [], model=2, **CFG).regrid_flagged(b[::4, ::4], 0.01, 4, 2)


@pytest.mark.parametrize("seed,tol,tile,buffer", [(43, 0.001, 3, 0), (41, 0.005, 5, 1)])
def test_flagged_boxes_with_remainders_match_the_oracle(M, A, seed, tol, tile, buffer):
    """Tiles that do not divide the refinable regions (one-cell remainders at
    the domain boundary are joined to the tile before them): the library's
    boxes equal the oracle's A12 boxes on both refined levels, the hierarchy
    accepts them, and the regridded states match the oracle's regrid."""
    nx0, ny0, r = 24, 20, 2
    b, qs = W.amr_small_case(2, nx0, ny0, r, 3, seed=seed, amp=0.3)
    g = M.Hierarchy(b, nx0, ny0, 0.2, r, W.amr_boxes_small(), model=2, **CFG)
    g.set_state(qs)
    o = A.AmrOracle(b, nx0, ny0, 0.2, r, W.amr_boxes_small(), model=2, **CFG)
    o.set_state(qs)
    g.step(2)
    assert o.step(2) == 0
    want = o.flag_boxes(tol, tile, buffer)
    g.regrid_flagged(b, tol, tile, buffer)
    assert g.boxes[1] == want[0] and g.boxes[2] == want[1]
    o.regrid(want)
    g.step(2)
    assert o.step(2) == 0
    for l in range(3):
        for k in range(len(g.boxes[l])):
            assert (rel_l2(g.get_patch(l, k), o.patch_state(l, k)) <= FP64_TOL).all(), (l, k)
    # again from the tiled boxes, which abut in rows (one atlas region, one
    # frame): the flags still compare neighbours within a patch only
    want = o.flag_boxes(tol, tile, buffer)
    g.regrid_flagged(b, tol, tile, buffer)
    assert g.boxes[1] == want[0] and g.boxes[2] == want[1]


def test_regrid_to_empty_levels_and_back(M, A):
    """A state at rest raises no flag: the flagged layout has no patches on the
    refined levels (the atlases hold no patch); the hierarchy steps on, then
    regrids back to the original boxes, all as the oracle does."""
    b, qs = W.amr_small_case(2, 24, 20, 2, 3, seed=3, wetdry=False)
    rest = []
    for l in range(3):
        bl = b
        for _ in range(2 - l):
            bl = A.block_mean(bl, 2)
        z = np.zeros_like(qs[l])
        z[0] = np.maximum(bl, 0.0)
        rest.append(z)
    g = M.Hierarchy(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, bc=(0, 0, 1, 1), **CFG)
    g.set_state(rest)
    o = A.AmrOracle(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, bc=(0, 0, 1, 1), **CFG)
    o.set_state(rest)
    g.step(1)
    assert o.step(1) == 0
    assert g.regrid_flagged(b, 0.01, 4, 2) == [0, 0]
    o.regrid(o.flag_boxes(0.01, 4, 2))
    g.step(2)
    assert o.step(2) == 0
    assert g.status() == 0
    assert (rel_l2(g.get_patch(0, 0), o.patch_state(0, 0)) <= FP64_TOL).all()
    g.regrid(b, W.amr_boxes_small())
    o.regrid(W.amr_boxes_small())
    g.step(2)
    assert o.step(2) == 0
    for l in range(3):
        for k in range(len(g.boxes[l])):
            q = g.get_patch(l, k)
            assert np.abs(q[1:]).max() <= 1e-14
            assert (rel_l2(q, o.patch_state(l, k)) <= FP64_TOL).all()


@pytest.mark.parametrize("precision", [0, 1])
def test_level_gather_on_the_device_equals_the_patches(M, precision):
    """sgn_amr_get_level_device writes every patch's interior at its place in
    the level's full grid, exactly the values sgn_amr_get_patch returns, and
    leaves the cells no patch covers untouched; field subsets and bad
    arguments."""
    import torch
    b, qs = W.amr_small_case(2, 24, 20, 2, 3, seed=8, amp=0.2)
    g = M.Hierarchy(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, precision=precision, **CFG)
    g.set_state(qs)
    g.step(3)
    for l in range(3):
        R = 2 ** l
        out = torch.full((g.nvar, 20 * R, 24 * R), -7.0, dtype=torch.float64, device="cuda")
        g.get_level_device(l, out)
        o = out.cpu().numpy()
        covered = np.zeros((20 * R, 24 * R), dtype=bool)
        for k, (i0, j0, nx, ny) in enumerate(g.boxes[l]):
            assert np.array_equal(o[:, j0:j0 + ny, i0:i0 + nx], g.get_patch(l, k))
            covered[j0:j0 + ny, i0:i0 + nx] = True
        assert (o[:, ~covered] == -7.0).all()
        two = torch.full((2, 20 * R, 24 * R), -7.0, dtype=torch.float64, device="cuda")
        g.get_level_device(l, two)
        assert np.array_equal(two.cpu().numpy(), o[:2])
    with pytest.raises(ValueError):
        g.get_level_device(1, torch.zeros((3, 20, 24), dtype=torch.float64, device="cuda"))
    with pytest.raises(M.sgn.SGNError):       # more fields than the model has
        g.get_level_device(0, torch.zeros((g.nvar + 1, 20, 24), dtype=torch.float64, device="cuda"))
