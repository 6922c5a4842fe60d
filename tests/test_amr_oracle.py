"""Pins of the refined-hierarchy oracle (oracle/amr_oracle.py) against facts that
do not depend on it: a one-level hierarchy is the uniform oracle; a finer level
covering the whole domain is the uniform fine oracle stepped r times as often;
lake at rest over wet/dry bathymetry; exact mass with walls (and that dropping
the reflux breaks it); mirror symmetry; a refined patch brings the solution
closer to the uniform fine grid."""
import numpy as np
import pytest

from paper_2606_12162_gb300 import workloads as W


@pytest.fixture(scope="module")
def A(oracle_mod):
    from oracle import amr_oracle
    return amr_oracle


CFG = dict(h_star=0.0, dry_tol=1e-3, alpha=3.0)


def _interior(am, l, k):
    return am.patch_state(l, k)


def test_one_level_is_the_uniform_oracle(A, oracle_mod):
    b, qs = W.amr_small_case(2, 20, 16, 2, 1, seed=1)
    am = A.AmrOracle(b, 20, 16, 0.1, 2, [], model=2, bc=(0, 1, 0, 1), **CFG)
    am.set_state(qs)
    o = oracle_mod.Oracle(b, dx=0.1, model=2, bc=(0, 1, 0, 1), **CFG)
    o.set_state(qs[0])
    for _ in range(6):
        assert am.dt_next == o.dt_cfl()
        am.step(1)
        assert o.step(1) == 0
    assert np.array_equal(_interior(am, 0, 0), o.get_state()[0])


@pytest.mark.parametrize("r", [2, 4])
def test_fine_level_covering_the_domain_is_the_uniform_fine_grid(A, oracle_mod, r):
    """Level 1 = the whole domain: its ghost cells are all boundary cells, so with
    a fixed level-0 step dt it must equal the uniform fine oracle taking r steps
    of dt / r, and level 0 must hold the block means of level 1."""
    nx0, ny0 = 12, 10
    b, qs = W.amr_small_case(2, nx0, ny0, r, 2, seed=2)
    am = A.AmrOracle(b, nx0, ny0, 0.2, r, [[(0, 0, nx0 * r, ny0 * r)]], model=2, bc=(0, 0, 0, 0), **CFG)
    am.set_state(qs)
    o = oracle_mod.Oracle(b, dx=0.2 / r, model=2, bc=(0, 0, 0, 0), **CFG)
    o.set_state(qs[1])
    dt = 0.5 * am.dt_next
    for _ in range(4):
        assert am.step_dt(dt) == 0
        for _ in range(r):
            assert o.step_dt(dt / r) == 0
    fine = _interior(am, 1, 0)
    assert np.array_equal(fine, o.get_state()[0])
    coarse = _interior(am, 0, 0)
    mean = A.block_mean(fine[1], r)
    assert np.array_equal(coarse[1], mean)


def test_lake_at_rest_across_levels(A):
    """Wet bathymetry under every patch edge (reading A10): eta = 0 and zero
    momenta stay exact through interpolation, subcycling, reflux and
    average-down."""
    b, qs = W.amr_small_case(2, 24, 20, 2, 3, seed=3, wetdry=False)
    rest = []
    for l, q in enumerate(qs):
        z = np.zeros_like(q)
        bl = b
        for _ in range(2 - l):
            bl = A.block_mean(bl, 2)
        z[0] = np.maximum(bl, 0.0)
        rest.append(z)
    am = A.AmrOracle(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, bc=(0, 0, 1, 1), **CFG)
    am.set_state(rest)
    for _ in range(5):
        assert am.step(1) == 0
    for l, pats in enumerate(am.levels):
        for k in range(len(pats)):
            q = _interior(am, l, k)
            i0, j0, nx, ny = pats[k]["box"]
            bl = am.b[l][j0:j0 + ny, i0:i0 + nx]
            assert np.abs(q[0] - np.maximum(bl, 0.0)).max() <= 1e-14
            assert np.abs(q[1:]).max() <= 1e-14


@pytest.mark.parametrize("model,wetdry", [(1, False), (2, True), (2, False)])
def test_mass_is_exact_with_walls(A, model, wetdry):
    b, qs = W.amr_small_case(model, 24, 20, 2, 3, seed=4, amp=0.3, wetdry=wetdry)
    am = A.AmrOracle(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=model, bc=(0, 0, 0, 0), **CFG)
    am.set_state(qs)
    m0 = am.mass()
    for _ in range(12):
        assert am.step(1) == 0
    # exact up to the water added where a refluxed cell would go dry (reading A7)
    assert abs(am.mass() - m0 - am.clipped) <= 1e-13 * m0
    if not wetdry:
        assert am.clipped == 0.0
    assert am.clipped <= 1e-4 * m0


def test_mass_pin_detects_a_missing_reflux(A):
    """Plant a mistake in the oracle (no reflux): the mass pin must fail."""
    class NoReflux(A.AmrOracle):
        def _build_registers(self):
            super()._build_registers()
            self.regs = [[] for _ in range(self.L)]
    b, qs = W.amr_small_case(2, 24, 20, 2, 3, seed=4, amp=0.3)
    am = NoReflux(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, bc=(0, 0, 0, 0), **CFG)
    am.set_state(qs)
    m0 = am.mass()
    for _ in range(12):
        am.step(1)
    assert abs(am.mass() - m0) > 1e-9 * m0


def test_mirror_symmetry(A):
    """x-mirror of bathymetry, state and boxes: the solution mirrors (hu flips)."""
    nx0, ny0, r = 24, 16, 2
    b, qs = W.amr_small_case(1, nx0, ny0, r, 3, seed=6)
    bs = 0.5 * (b + b[:, ::-1])
    qsym = []
    for q in qs:
        s = 0.5 * (q + q[:, :, ::-1])
        s[1] = 0.5 * (q[1] - q[1, :, ::-1])
        qsym.append(s)
    # eta must stay above b after symmetrisation: use a rest state plus the symmetric hump
    hb = []
    for l in range(3):
        bl = bs
        for _ in range(2 - l):
            bl = A.block_mean(bl, r)
        hb.append(bl)
    for l in range(3):
        qsym[l][0] = np.maximum(qsym[l][0], hb[l])
    lvl1 = [(8, 8, 12, 12), (28, 8, 12, 12)]
    lvl2 = [(20, 20, 12, 8), (64, 20, 12, 8)]
    am = A.AmrOracle(bs, nx0, ny0, 0.2, r, [lvl1, lvl2], model=1, bc=(0, 0, 0, 0), **CFG)
    am.set_state(qsym)
    for _ in range(6):
        assert am.step(1) == 0
    q0 = _interior(am, 0, 0)
    assert np.abs(q0[0] - q0[0, :, ::-1]).max() <= 1e-13
    assert np.abs(q0[1] + q0[1, :, ::-1]).max() <= 1e-13
    a, c = _interior(am, 1, 0), _interior(am, 1, 1)
    assert np.abs(a[0] - c[0, :, ::-1]).max() <= 1e-13
    a, c = _interior(am, 2, 0), _interior(am, 2, 1)
    assert np.abs(a[0] - c[0, :, ::-1]).max() <= 1e-13


def test_refined_patch_approaches_the_fine_grid(A, oracle_mod):
    """A level-1 patch (ratio 2) over the hump: the surface in the patch is closer
    to the uniform fine solution than the uniform coarse solution is."""
    nx0, ny0, r = 24, 24, 2
    b, qs = W.amr_small_case(1, nx0, ny0, r, 2, seed=7, wetdry=False)
    hump = np.unravel_index(np.argmax(qs[1][0] - b), b.shape)
    jc, ic = int(hump[0]) // (2 * r) * r, int(hump[1]) // (2 * r) * r
    i0 = min(max(ic - 8, 4), nx0 * r - 20)
    j0 = min(max(jc - 8, 4), ny0 * r - 20)
    box = (i0 - i0 % r, j0 - j0 % r, 16, 16)
    am = A.AmrOracle(b, nx0, ny0, 0.2, r, [[box]], model=1, bc=(0, 0, 0, 0), **CFG)
    am.set_state(qs)
    fine = oracle_mod.Oracle(b, dx=0.2 / r, model=1, bc=(0, 0, 0, 0), **CFG)
    fine.set_state(qs[1])
    coarse = oracle_mod.Oracle(A.block_mean(b, r), dx=0.2, model=1, bc=(0, 0, 0, 0), **CFG)
    coarse.set_state(qs[0])
    dt = 0.8 * am.dt_next
    for _ in range(8):
        assert am.step_dt(dt) == 0
        assert coarse.step_dt(dt) == 0
        for _ in range(r):
            assert fine.step_dt(dt / r) == 0
    i0, j0, nx, ny = box
    ref = fine.get_state()[0][0, j0:j0 + ny, i0:i0 + nx]
    e_amr = np.linalg.norm(_interior(am, 1, 0)[0] - ref)
    cprol = np.repeat(np.repeat(coarse.get_state()[0][0], r, 0), r, 1)[j0:j0 + ny, i0:i0 + nx]
    e_coarse = np.linalg.norm(cprol - ref)
    assert e_amr < 0.5 * e_coarse


def _pair_states(a, b):
    return all(np.array_equal(a.patch_state(l, k), b.patch_state(l, k))
               for l in range(a.L) for k in range(len(a.levels[l])))


def test_regrid_to_the_same_boxes_changes_nothing(A):
    """A11: every new cell lies in an old patch of its level (copies only) and
    average-down reproduces the covered coarse cells, so the run continues
    bit for bit."""
    b, qs = W.amr_small_case(2, 24, 20, 2, 3, seed=12, amp=0.25)
    ref = A.AmrOracle(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, **CFG)
    ref.set_state(qs)
    assert ref.step(7) == 0
    am = A.AmrOracle(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, **CFG)
    am.set_state(qs)
    assert am.step(3) == 0
    am.regrid(W.amr_boxes_small())
    assert am.step(4) == 0
    assert _pair_states(am, ref) and am.t == ref.t and am.dt_next == ref.dt_next


def test_regrid_keeps_rest_and_mass(A):
    """Moving the patches keeps the lake at rest exactly, and mass up to
    rounding over wet bathymetry (the interpolated surface has the parent's
    mean: the limited slopes cancel over the r x r children)."""
    b, qs = W.amr_small_case(2, 24, 20, 2, 3, seed=3, wetdry=False)
    rest = []
    for l, q in enumerate(qs):
        z = np.zeros_like(q)
        bl = b
        for _ in range(2 - l):
            bl = A.block_mean(bl, 2)
        z[0] = np.maximum(bl, 0.0)
        rest.append(z)
    am = A.AmrOracle(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, bc=(0, 0, 1, 1), **CFG)
    am.set_state(rest)
    assert am.step(2) == 0
    am.regrid(W.amr_boxes_small_moved())
    assert am.step(3) == 0
    for l, pats in enumerate(am.levels):
        for k in range(len(pats)):
            i0, j0, nx, ny = pats[k]["box"]
            q = am.patch_state(l, k)
            assert np.abs(q[0] - np.maximum(am.b[l][j0:j0 + ny, i0:i0 + nx], 0.0)).max() <= 1e-14
            assert np.abs(q[1:]).max() <= 1e-14
    b, qs = W.amr_small_case(2, 24, 20, 2, 3, seed=5, amp=0.3, wetdry=False)
    am = A.AmrOracle(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, bc=(0, 0, 0, 0), **CFG)
    am.set_state(qs)
    assert am.step(4) == 0
    m0, t0 = am.mass(), am.t
    am.regrid(W.amr_boxes_small_moved())
    assert abs(am.mass() - m0) <= 1e-13 * m0 and am.t == t0
    assert am.step(4) == 0
    assert abs(am.mass() - m0 - am.clipped) <= 1e-13 * m0


def test_regrid_copies_and_interpolates(A):
    """New cells inside an old patch of their level keep its values; new cells
    outside take the parent's interpolation, whose r x r mean is the parent
    value where the parent is wet (smooth wet data, no clipping)."""
    b, qs = W.amr_small_case(2, 24, 20, 2, 3, seed=6, amp=0.2, wetdry=False)
    am = A.AmrOracle(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, **CFG)
    am.set_state(qs)
    assert am.step(3) == 0
    before = [[p["q"].copy() for p in am.levels[l]] for l in range(3)]
    boxes_before = [list(am.boxes[l]) for l in range(3)]
    am.regrid(W.amr_boxes_small_moved())
    # level-1 patch (8, 8, 16, 12) is in both layouts: every interior cell kept
    # except the covered ones (average-down of the new level 2)
    k_old = boxes_before[1].index((8, 8, 16, 12))
    k_new = am.boxes[1].index((8, 8, 16, 12))
    q_old = before[1][k_old][:, 2:-2, 2:-2]
    q_new = am.patch_state(1, k_new)
    cov = am.cover[1][k_new]
    assert np.array_equal(q_new[:, ~cov][0], q_old[:, ~cov][0])
    # new level-2 cells of (24, 20, 16, 12) outside the old (20, 20, 16, 12)
    # (level-2 x 36..39, parent cells ic = 18, 19, uncovered before): the 2 x 2
    # mean of eta over each parent cell is that cell's value before regridding
    k2 = am.boxes[2].index((24, 20, 16, 12))
    q2 = am.patch_state(2, k2)[0]
    for jc in range(10, 16):
        for ic in range(18, 20):
            m = q2[2 * jc - 20:2 * jc - 18, 2 * ic - 24:2 * ic - 22].mean()
            assert abs(m - q_old[0, jc - 8, ic - 8]) <= 1e-14 * max(1.0, abs(m))
            assert np.ptp(q2[2 * jc - 20:2 * jc - 18, 2 * ic - 24:2 * ic - 22]) > 0.0   # not a plain copy


def _channel_soliton(A, a=0.3, nx0=96, ny0=8, r=2, dx0=0.4, H=1.0, x0=10.0):
    xf, yf = W.cell_centres(nx0 * r, ny0 * r, dx0 / r, dx0 / r)
    bf = np.full(xf.shape, -H)
    qf = W.soliton_state(2, xf, yf, bf, a, H, x0)
    qc = qf.reshape(qf.shape[0], ny0, r, nx0, r).mean(axis=(2, 4))
    return bf, [qc, qf], nx0, ny0, r, dx0


def test_flagged_boxes_follow_the_wave(A, oracle_mod):
    """A12 (Sec. 6.3 flag): regridding from the surface-jump flags every four
    level-0 steps keeps the fine level on a travelling solitary wave, so the
    composite solution stays closer to the uniform fine grid than with the
    patch left where the wave started; the flagged boxes obey the nesting
    rules (the constructor validates them) and cover every flagged cell."""
    bf, qs, nx0, ny0, r, dx0 = _channel_soliton(A)
    T, tol = 3.0, 0.01

    def run(regrid_every):
        am = A.AmrOracle(bf, nx0, ny0, dx0, r, [[(36, 0, 28, 16)]], model=2, **CFG)
        am.set_state(qs)
        n = 0
        while am.t < T - 1e-12:
            assert am.step_dt(min(am.dt_next, T - am.t)) == 0
            n += 1
            if regrid_every and n % regrid_every == 0:
                boxes = am.flag_boxes(tol, 4, 2)
                e = am.patch_state(0, 0)[0]
                jump = np.zeros(e.shape, dtype=bool)
                jump[:, 1:] |= np.abs(np.diff(e, axis=1)) > tol
                jump[:, :-1] |= np.abs(np.diff(e, axis=1)) > tol
                cov = np.zeros(e.shape, dtype=bool)
                for (i0, j0, nx, ny) in boxes[0]:
                    cov[j0 // r:(j0 + ny) // r, i0 // r:(i0 + nx) // r] = True
                assert cov[jump].all()
                am.regrid(boxes)
        return am
    u = oracle_mod.Oracle(bf, dx=dx0 / r, model=2, **CFG)
    u.set_state(qs[1])
    t = 0.0
    while t < T - 1e-12:
        dt = min(u.dt_cfl(), T - t)
        assert u.step_dt(dt) == 0
        t += dt
    eu = u.get_state()[0][0]

    def composite(am):
        eta = np.repeat(np.repeat(am.patch_state(0, 0)[0], r, 0), r, 1)
        for k, (i0, j0, nx, ny) in enumerate(am.boxes[1]):
            eta[j0:j0 + ny, i0:i0 + nx] = am.patch_state(1, k)[0]
        return eta
    static, moved = run(0), run(4)
    e_static = np.abs(composite(static) - eu).max()
    e_moved = np.abs(composite(moved) - eu).max()
    assert e_moved < 0.5 * e_static, (e_moved, e_static)
    crest = int(np.argmax(eu[0]))
    assert any(i0 <= crest < i0 + nx for (i0, j0, nx, ny) in moved.boxes[1])


@pytest.mark.parametrize("seed,tol,tile,buffer", [(41, 0.005, 4, 1), (42, 0.02, 6, 2), (43, 0.001, 3, 0)])
def test_flagged_boxes_obey_the_hierarchy_rules(A, seed, tol, tile, buffer):
    """A12 produces box lists that A1 accepts (aligned to parent cells, inside
    one parent, two parent cells from its edges except at the domain boundary,
    disjoint: the constructor validates all of it), for several states and
    settings; every level-0 cell with a surface jump to a neighbour (both wet)
    lies under a level-1 box."""
    b, qs = W.amr_small_case(2, 24, 20, 2, 3, seed=seed, amp=0.3)
    am = A.AmrOracle(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, **CFG)
    am.set_state(qs)
    assert am.step(2) == 0
    boxes = am.flag_boxes(tol, tile, buffer)
    A.AmrOracle(b, 24, 20, 0.2, 2, boxes, model=2, **CFG)     # raises on a rule violation
    e = am.patch_state(0, 0)[0]
    p0 = am.levels[0][0]
    ny0, nx0 = e.shape
    wet = (e - p0["b"][A.NG:A.NG + ny0, A.NG:A.NG + nx0]) > CFG["dry_tol"]
    jx = (np.abs(np.diff(e, axis=1)) > tol) & wet[:, 1:] & wet[:, :-1]
    jy = (np.abs(np.diff(e, axis=0)) > tol) & wet[1:, :] & wet[:-1, :]
    jump = np.zeros(e.shape, dtype=bool)
    jump[:, 1:] |= jx
    jump[:, :-1] |= jx
    jump[1:, :] |= jy
    jump[:-1, :] |= jy
    cov = np.zeros(e.shape, dtype=bool)
    for (i0, j0, nx, ny) in boxes[0]:
        cov[j0 // 2:(j0 + ny) // 2, i0 // 2:(i0 + nx) // 2] = True
    assert cov[jump].all()
    assert sum(len(bl) for bl in boxes) > 0


@pytest.mark.parametrize("seed,tol,tile", [(51, 0.003, 4), (52, 0.01, 2), (53, 0.002, 5)])
def test_flag_driven_regrid_keeps_mass_and_steps_on(A, seed, tol, tile):
    """Over wet bathymetry, regridding to the flagged boxes (A11 + A12) keeps
    the mass to rounding, and the hierarchy steps on with exact mass."""
    b, qs = W.amr_small_case(2, 24, 20, 2, 3, seed=seed, amp=0.3, wetdry=False)
    am = A.AmrOracle(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, **CFG)
    am.set_state(qs)
    assert am.step(3) == 0
    m0 = am.mass()
    am.regrid(am.flag_boxes(tol, tile, 1))
    assert abs(am.mass() - m0) <= 1e-13 * m0
    assert am.step(3) == 0
    assert abs(am.mass() - m0 - am.clipped) <= 1e-13 * m0


def test_regrid_to_empty_levels_and_back(A):
    """A state at rest raises no flag: the flagged layout has no patches on the
    refined levels; the hierarchy steps on at rest, and regridding back to the
    original boxes (all cells interpolated from level 0) stays at rest."""
    b, qs = W.amr_small_case(2, 24, 20, 2, 3, seed=3, wetdry=False)
    rest = []
    for l, q in enumerate(qs):
        z = np.zeros_like(q)
        bl = b
        for _ in range(2 - l):
            bl = A.block_mean(bl, 2)
        z[0] = np.maximum(bl, 0.0)
        rest.append(z)
    am = A.AmrOracle(b, 24, 20, 0.2, 2, W.amr_boxes_small(), model=2, **CFG)
    am.set_state(rest)
    assert am.step(1) == 0
    boxes = am.flag_boxes(0.01, 4, 2)
    assert boxes == [[], []]
    am.regrid(boxes)
    assert am.step(2) == 0
    assert np.abs(am.patch_state(0, 0)[1:]).max() <= 1e-14
    am.regrid(W.amr_boxes_small())
    assert am.step(2) == 0
    for l, pats in enumerate(am.levels):
        for k in range(len(pats)):
            assert np.abs(am.patch_state(l, k)[1:]).max() <= 1e-14
