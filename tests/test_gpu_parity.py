"""GPU (C ABI, CUDA kernels) versus the FP64 CPU oracle, element by element.

FP64 bar: per-field relative L2 <= 1e-12 (and the time, time step and mass to
1e-12).  Mixed precision (FP32 bulk, FP64 critical): per-field tolerances on
relative L2 and max error of eta, hu, hv.  Sizes span several thread blocks with
ragged tails; full-size configurations are checked on sampled crops (one step of
the oracle with the GPU's time step around sampled cells) and by invariants.
"""
import numpy as np
import pytest

from paper_2606_12162_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


@pytest.fixture(scope="module")
def sgn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_12162_gb300 import build, sgn as S
    build.build()
    S.load()
    return S


def rel_l2(a, b, mask=None):
    out = []
    for k in range(a.shape[0]):
        x, y = a[k], b[k]
        if mask is not None:
            x, y = x[mask], y[mask]
        den = np.linalg.norm(y)
        num = np.linalg.norm(x - y)
        out.append(num / den if den > 0 else num)
    return np.array(out)


def pair(S, O, b, q, steps, precision=0, **cfg):
    s = S.Solver(b, precision=precision, **cfg)
    s.set_state(q)
    s.step(steps)
    qg, tg = s.get_state()
    o = O.Oracle(b, **cfg)
    o.set_state(q)
    rc = o.step(steps)
    assert rc == 0, o.status
    qo, to = o.get_state()
    return s, o, qg, tg, qo, to


CASES = [
    # model, nx, ny, bc, wetdry, steps
    (2, 37, 29, (0, 0, 0, 0), False, 30),
    (1, 70, 9, (1, 1, 0, 0), True, 30),
    (0, 130, 67, (2, 2, 0, 1), True, 25),
    (2, 66, 131, (0, 1, 2, 2), True, 20),
    (1, 2, 2, (0, 0, 0, 0), False, 5),
    (2, 5, 3, (1, 0, 1, 0), False, 8),
    (2, 257, 33, (1, 1, 1, 1), True, 12),
]


@pytest.mark.parametrize("model,nx,ny,bc,wetdry,steps", CASES)
def test_fp64_small_cases(sgn, oracle_mod, model, nx, ny, bc, wetdry, steps):
    b, q = W.random_small_case(model, nx, ny, seed=nx * 7 + ny, dx=0.05, wetdry=wetdry, amp=0.15)
    cfg = dict(dx=0.05, dy=0.04, model=model, bc=bc, h_star=0.6)
    s, o, qg, tg, qo, to = pair(sgn, oracle_mod, b, q, steps, **cfg)
    assert abs(tg - to) <= FP64_TOL * to
    err = rel_l2(qg, qo)
    assert (err <= FP64_TOL).all(), err
    f, dt, cr = s.status()
    assert f == 0
    assert abs(dt - o.last_dt) <= FP64_TOL * o.last_dt
    assert abs(cr - o.max_courant) <= 1e-10
    assert abs(s.mass() - o.mass()) <= FP64_TOL * o.mass()


@pytest.mark.parametrize("limiter,strang", [(0, 1), (2, 1), (1, 0)])
def test_fp64_options(sgn, oracle_mod, limiter, strang):
    b, q = W.random_small_case(1, 48, 40, seed=4, dx=0.1, wetdry=False)
    cfg = dict(dx=0.1, model=1, bc=(0, 0, 0, 0), limiter=limiter, strang=strang)
    _, _, qg, _, qo, _ = pair(sgn, oracle_mod, b, q, 20, **cfg)
    assert (rel_l2(qg, qo) <= FP64_TOL).all()


def test_fp64_phi_override_and_aux(sgn, oracle_mod):
    b, q = W.random_small_case(2, 60, 44, seed=8, dx=0.1, wetdry=True)
    phi = np.zeros(b.shape, np.uint8)
    phi[:, :30] = 1
    cfg = dict(dx=0.1, model=2, bc=(0, 0, 0, 0))
    s = sgn.Solver(b, phi_override=phi, **cfg)
    o = oracle_mod.Oracle(b, phi_override=phi, **cfg)
    c2g, phig = s.aux()
    c2o, phio = o.aux()
    assert np.array_equal(phig, phio) and np.array_equal(c2g, c2o)
    s2 = sgn.Solver(b, h_star=0.4, **cfg)
    o2 = oracle_mod.Oracle(b, h_star=0.4, **cfg)
    assert np.array_equal(s2.aux()[1], o2.aux()[1])
    assert np.array_equal(s2.aux()[0], o2.aux()[0])


@pytest.mark.parametrize("model", [2, 1])
def test_config1_full_size(sgn, oracle_mod, model):
    """256 x 256 planar solitary wave, walls, 200 steps (the first configuration)."""
    c = W.config1(model=model)
    cfg = dict(dx=c["dx"], model=model, bc=c["bc"], alpha=c["alpha"], cfl=c["cfl"])
    s, o, qg, tg, qo, to = pair(sgn, oracle_mod, c["b"], c["q"], c["steps"], **cfg)
    assert abs(tg - to) <= FP64_TOL * to
    err = rel_l2(qg, qo)
    assert (err <= FP64_TOL).all(), err
    m0 = oracle_mod.Oracle(c["b"], **cfg)
    m0.set_state(c["q"])
    assert abs(s.mass() - m0.mass()) <= 1e-13 * m0.mass()


def test_lake_at_rest_config2_bathymetry(sgn):
    """Ocean at rest over the beach + seamount of the second configuration stays
    exactly at rest in FP64 and in mixed precision (100 steps, 1024^2 crop)."""
    b, _, _ = W.config2_bathymetry(nx=1024, ny=1024, dx=40.0)
    for prec in (0, 1):
        s = sgn.Solver(b, model=2, dx=40.0, bc=(1, 1, 1, 1), h_star=20.0, precision=prec)
        s.set_state(W.rest_state(b, 2))
        s.step(100)
        qg, _ = s.get_state()
        wet = b < 0
        assert np.abs(qg[0][wet]).max() == 0.0
        assert np.abs(qg[1:]).max() == 0.0


def test_mixed_precision_small_against_oracle(sgn, oracle_mod):
    b, q = W.random_small_case(2, 96, 80, seed=12, dx=0.05, wetdry=True, amp=0.15)
    cfg = dict(dx=0.05, model=2, bc=(0, 0, 0, 0), h_star=0.6)
    s, o, qg, tg, qo, to = pair(sgn, oracle_mod, b, q, 40, precision=1, **cfg)
    wet = (qo[0] - b) > 1e-3
    err = rel_l2(qg[:3], qo[:3], wet)
    assert err[0] <= 1e-5 and err[1] <= 1e-3 and err[2] <= 1e-3, err
    assert abs(tg - to) <= 1e-5 * to


def test_config2_crop_mixed_and_fp64(sgn, oracle_mod):
    """A 512 x 512 crop of the second configuration (beach, seamount, landslide
    depression, wet/dry shoreline, SWE switch), 200 steps: FP64 within 1e-12,
    mixed precision within the stated tolerances, gauges identical."""
    c = W.config2(model=2, nx=512, ny=512, dx=80.0, ngauges=16)
    cfg = dict(dx=c["dx"], model=2, bc=c["bc"], h_star=c["h_star"], alpha=3.0)
    s, o, qg, tg, qo, to = pair(sgn, oracle_mod, c["b"], c["q"], 0, **cfg)
    s.add_gauges(c["gauges"], 256)
    o.add_gauges(c["gauges"], 256)
    s.step(200)
    assert o.step(200) == 0
    qg, tg = s.get_state()
    qo, to = o.get_state()
    assert (rel_l2(qg, qo) <= FP64_TOL).all(), rel_l2(qg, qo)
    gg, go = s.gauges(), o.gauges()
    assert gg.shape == go.shape
    assert np.abs(gg - go).max() <= 1e-11 * (1 + np.abs(go).max())
    sm = sgn.Solver(c["b"], precision=1, **cfg)
    sm.set_state(c["q"])
    sm.step(200)
    qm, _ = sm.get_state()
    wet = (qo[0] - c["b"]) > 1e-3
    err = rel_l2(qm[:3], qo[:3], wet)
    amp = np.abs(c["q"][0][c["b"] < 0]).max()
    assert err[0] <= 1e-4 and err[1] <= 1e-3 and err[2] <= 1e-3, err
    assert np.abs(qm[0] - qo[0]).max() <= 1e-3 * amp


def _crop_check(S, O, s, b, cfg, ncrops, seed, rad=6):
    """One step of the oracle on crops around sampled cells, with the GPU's state
    and time step, against the GPU's next state at the crop centres."""
    q0, _ = s.get_state()
    _, dt0, _ = s.status()
    s.step(1)
    _, dt, _ = s.status()
    q1, _ = s.get_state()
    rng = np.random.default_rng(seed)
    ny, nx = b.shape
    worst = 0.0
    for _ in range(ncrops):
        j = int(rng.integers(rad, ny - rad))
        i = int(rng.integers(rad, nx - rad))
        sl = (slice(j - rad, j + rad + 1), slice(i - rad, i + rad + 1))
        o = O.Oracle(b[sl], **cfg)
        o.set_state(q0[(slice(None),) + sl])
        assert o.step_dt(dt) in (0, -1)
        qc, _ = o.get_state()
        # cells at distance <= rad - 3 from the crop edge are exact
        inner = (slice(3, 2 * rad - 2), slice(3, 2 * rad - 2))
        a = q1[(slice(None),) + sl][(slice(None),) + inner]
        c = qc[(slice(None),) + inner]
        scale = np.abs(q1).max(axis=(1, 2))[:, None, None] + 1e-300
        worst = max(worst, float((np.abs(a - c) / scale).max()))
    return worst


def test_config2_full_size_sampled_crops(sgn, oracle_mod):
    """Full 4096 x 4096 second configuration (HSGN, FP64, the launch configuration
    the benchmark times): 20 steps on the GPU, then one step checked on 40 sampled
    crops against the oracle, and the mass is conserved (closed domain region)."""
    c = W.config2(model=2)
    cfg = dict(dx=c["dx"], model=2, bc=c["bc"], h_star=c["h_star"], alpha=3.0)
    s = sgn.Solver(c["b"], **cfg)
    s.set_state(c["q"])
    m0 = s.mass()
    s.step(20)
    worst = _crop_check(sgn, oracle_mod, s, c["b"], cfg, 40, 7)
    assert worst <= 1e-13, worst
    assert abs(s.mass() - m0) <= 1e-12 * m0
    f, _, cr = s.status()
    assert f == 0 and cr <= 1.0


def test_determinism_and_checkpoint(sgn):
    b, q = W.random_small_case(2, 150, 90, seed=21, dx=0.05, wetdry=True)
    cfg = dict(dx=0.05, model=2, bc=(0, 1, 0, 1), h_star=0.6)
    s = sgn.Solver(b, **cfg)
    s.set_state(q)
    s.step(40)
    a, ta = s.get_state()
    s2 = sgn.Solver(b, **cfg)
    s2.set_state(q)
    s2.step(20)
    mid, tm = s2.get_state()
    s3 = sgn.Solver(b, **cfg)
    s3.set_state(mid, tm)
    s3.step(20)
    c, tc = s3.get_state()
    assert np.array_equal(a, c) and ta == tc
    s.set_state(q)
    s.step(40)
    a2, _ = s.get_state()
    assert np.array_equal(a, a2)


def test_step_dt_matches_oracle(sgn, oracle_mod):
    b, q = W.random_small_case(1, 40, 30, seed=2, dx=0.05, wetdry=False)
    cfg = dict(dx=0.05, model=1, bc=(0, 0, 0, 0))
    s = sgn.Solver(b, **cfg)
    s.set_state(q)
    o = oracle_mod.Oracle(b, **cfg)
    o.set_state(q)
    for dt in (1e-3, 2e-3, 5e-4):
        s.step_dt(dt)
        assert o.step_dt(dt) == 0
    assert (rel_l2(s.get_state()[0], o.get_state()[0]) <= FP64_TOL).all()

    # the next CFL step is reported before it is taken, equal to the oracle's
    for _ in range(3):
        dn = s.next_dt()
        assert abs(dn - o.dt_cfl()) <= 1e-12 * dn
        s.step(1)
        assert o.step(1) == 0
        assert s.status()[1] == dn


def test_errors_reported(sgn):
    b, q = W.random_small_case(2, 32, 32, seed=3, dx=0.05, wetdry=False)
    s = sgn.Solver(b, model=2, dx=0.05)
    bad = q.copy()
    bad[1, 5, 5] = np.nan
    s.set_state(bad)
    assert s.step_rc(1) in (-5, -7)      # non-finite (or non-hyperbolic) reported, no fault
    s.set_state(q)
    with pytest.raises(sgn.SGNError) as e:
        s.step_dt(10.0)                  # far above the CFL limit
    assert e.value.code in (-6, -5, -4, -7)
    dry = np.full((8, 8), 1.0)
    s2 = sgn.Solver(dry, model=0, dx=1.0)
    assert s2.step_rc(1) == -8           # all dry
    with pytest.raises(sgn.SGNError):
        s.get_state_ptr(0, 1) if False else s.add_gauges([[1e9, 0.0]], 4)


def test_fp64_reciprocal_and_sqrt_against_ieee(sgn):
    """The kernels' FP64 reciprocal and square root (hardware approximation plus
    Newton-Raphson steps) stay within 2 ulp of CUDA's IEEE division and sqrt over
    a wide range of magnitudes."""
    import ctypes
    import torch
    rng = np.random.default_rng(0)
    x = np.concatenate([10.0 ** rng.uniform(-200, 200, 20000), rng.uniform(0.5, 2.0, 20000),
                        np.array([1.0, 2.0, 3.0, 1e-300, 1e300, 7.0 / 3.0])])
    xd = torch.from_numpy(x).cuda()
    err = torch.empty(2 * len(x), dtype=torch.float64, device="cuda")
    rc = sgn.load().sgn_math_check(ctypes.c_void_p(xd.data_ptr()), len(x), ctypes.c_void_p(err.data_ptr()))
    assert rc == 0
    e = err.cpu().numpy().reshape(-1, 2)
    assert e[:, 0].max() <= 2.0 and e[:, 1].max() <= 2.0, e.max(axis=0)


def test_fp32_reciprocal_and_sqrt_against_ieee(sgn):
    """The mixed path's FP32 reciprocal and square root (hardware approximation
    plus one Newton-Raphson step) stay within 2 ulp of CUDA's correctly rounded
    FP32 division and sqrt wherever x and 1/x are normal floats (the kernels
    never meet subnormal depths, speeds or sums; the approximations flush them
    to zero)."""
    import ctypes
    import torch
    rng = np.random.default_rng(1)
    x = np.concatenate([10.0 ** rng.uniform(-36, 36, 40000), rng.uniform(0.5, 2.0, 40000),
                        np.array([1.0, 2.0, 3.0, 1e-37, 8e37, 7.0 / 3.0])]).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    err = torch.empty(2 * len(x), dtype=torch.float64, device="cuda")
    rc = sgn.load().sgn_math_check_f32(ctypes.c_void_p(xd.data_ptr()), len(x), ctypes.c_void_p(err.data_ptr()))
    assert rc == 0
    e = err.cpu().numpy().reshape(-1, 2)
    assert e[:, 0].max() <= 2.0 and e[:, 1].max() <= 2.0, e.max(axis=0)


def _arrival_times(rec, frac=0.01):
    """First time at which |eta| reaches frac of the gauge's maximum |eta|."""
    t = rec[:, 0, 0]
    eta = np.abs(rec[:, :, 1])
    thr = frac * eta.max(axis=0)
    out = []
    for g in range(eta.shape[1]):
        idx = np.nonzero(eta[:, g] >= thr[g])[0]
        out.append(t[idx[0]] if len(idx) and thr[g] > 0 else np.nan)
    return np.array(out)


def test_config3_crop_fp64_and_mixed(sgn, oracle_mod):
    """1024 x 1024 crop of the third configuration (fractal bathymetry, ~20 % land,
    2 m uplift), 200 steps: the GPU FP64 path within 1e-12 of the oracle; the mixed
    path against the GPU FP64 path within relative L2 1e-3 (eta, hu, hv over wet
    cells), max |eta| error 1e-2 of the initial amplitude, gauge arrival times
    within one time step."""
    c = W.config3(model=2, crop=1024, ngauges=32)
    cfg = dict(dx=c["dx"], x0=c["x0"], y0=c["y0"], model=2, bc=c["bc"], h_star=c["h_star"], alpha=3.0)
    steps = 200
    # gauges on rings of 10-30 km around the source, where the wave arrives within
    # the run (wet cells only)
    cx, cy = c["source"]
    ring = []
    for r in (10e3, 20e3, 30e3):
        for a in np.linspace(0, 2 * np.pi, 8, endpoint=False):
            x, y = cx + r * np.cos(a), cy + r * np.sin(a)
            i, j = int((x - c["x0"]) / c["dx"]), int((y - c["y0"]) / c["dx"])
            if 0 <= i < 1024 and 0 <= j < 1024 and c["b"][j, i] < -50.0:
                ring.append((x, y))
    c["gauges"] = np.array(ring)
    s = sgn.Solver(c["b"], **cfg)
    s.set_state(c["q"])
    s.add_gauges(c["gauges"], steps + 4)
    s.step(steps)
    q64, t64 = s.get_state()
    g64 = s.gauges()
    o = oracle_mod.Oracle(c["b"], **cfg)
    o.set_state(c["q"])
    assert o.step(steps) == 0
    qo, to = o.get_state()
    assert (rel_l2(q64, qo) <= FP64_TOL).all(), rel_l2(q64, qo)
    sm = sgn.Solver(c["b"], precision=1, **cfg)
    sm.set_state(c["q"])
    sm.add_gauges(c["gauges"], steps + 4)
    sm.step(steps)
    qm, _ = sm.get_state()
    gm = sm.gauges()
    wet = (q64[0] - c["b"]) > 1e-3
    err = rel_l2(qm[:3], q64[:3], wet)
    assert (err <= 1e-3).all(), err
    assert np.abs(qm[0] - q64[0]).max() <= 1e-2 * 2.0
    dt = s.status()[1]
    ta, tb = _arrival_times(g64), _arrival_times(gm)
    ok = ~np.isnan(ta) & (np.abs(g64[:, :, 1]).max(axis=0) >= 0.01)
    assert ok.sum() >= 8
    assert np.nanmax(np.abs(ta[ok] - tb[ok])) <= dt * 1.0001


def test_config2_full_size_mixed_against_fp64(sgn):
    """Full 4096 x 4096 second configuration, 300 steps: mixed precision against
    the (oracle-checked) FP64 GPU path: relative L2 of eta <= 1e-4 and of hu, hv
    <= 1e-3 over wet cells, max |eta| error <= 1e-3 of the 5 m source amplitude."""
    c = W.config2(model=2)
    cfg = dict(dx=c["dx"], model=2, bc=c["bc"], h_star=c["h_star"], alpha=3.0)
    out = []
    for prec in (0, 1):
        s = sgn.Solver(c["b"], precision=prec, **cfg)
        s.set_state(c["q"])
        s.step(300)
        out.append(s.get_state()[0])
        del s
    q64, qm = out
    wet = (q64[0] - c["b"]) > 1e-3
    err = rel_l2(qm[:3], q64[:3], wet)
    assert err[0] <= 1e-4 and err[1] <= 1e-3 and err[2] <= 1e-3, err
    assert np.abs(qm[0] - q64[0]).max() <= 1e-3 * 5.0


def test_config2_full_size_mixed_against_fp64_1000_steps(sgn):
    """Full 4096 x 4096 second configuration over 1000 steps, each path on its
    own CFL steps, at the bar frozen from the measured run: relative L2 over wet
    cells eta <= 2e-4, hu, hv <= 1e-3; max |eta| error <= 5e-3 of the 5 m source
    amplitude; the 64 gauges' arrival times (first time |eta| reaches 1 % of
    its largest value there) within one time step."""
    c = W.config2(model=2)
    cfg = dict(dx=c["dx"], model=2, bc=c["bc"], h_star=c["h_star"], alpha=3.0)
    steps = 1000
    out, gauges = [], []
    for prec in (0, 1):
        s = sgn.Solver(c["b"], precision=prec, **cfg)
        s.set_state(c["q"])
        s.add_gauges(c["gauges"], steps + 4)
        s.step(steps)
        assert s.status()[0] == 0
        out.append(s.get_state()[0])
        gauges.append(s.gauges())
        if prec == 0:
            dt = s.status()[1]
        del s
    q64, qm = out
    wet = (q64[0] - c["b"]) > 1e-3
    err = rel_l2(qm[:3], q64[:3], wet)
    assert err[0] <= 2e-4 and err[1] <= 1e-3 and err[2] <= 1e-3, err
    assert np.abs(qm[0] - q64[0]).max() <= 5e-3 * 5.0
    g64, gm = gauges
    ta, tb = _arrival_times(g64), _arrival_times(gm)
    ok = ~np.isnan(ta) & ~np.isnan(tb) & (np.abs(g64[:, :, 1]).max(axis=0) >= 0.01)
    assert ok.sum() >= 32
    assert np.nanmax(np.abs(ta[ok] - tb[ok])) <= dt * 1.0001


def test_config3_full_size_mixed_against_fp64(sgn):
    """Full 8192 x 8192 third configuration (fractal bathymetry, 2 m uplift),
    400 steps, each path on its own CFL steps: the mixed path (one-pass kernel,
    the default on this grid) against the (oracle-checked) FP64 GPU path, at
    the configuration's bar: relative L2 over wet cells of eta, hu, hv <= 1e-3
    and max |eta| error <= 1e-2 of the 2 m uplift; both runs without a status
    flag.  (The 2000-step run of the configuration measures 1.7e-6 and 7.6e-6;
    the FP64 path takes about 0.13 s a step here, so the test keeps to 400.)"""
    c = W.config3(model=2)
    cfg = dict(dx=c["dx"], model=2, bc=c["bc"], h_star=c["h_star"], alpha=3.0, cfl=c["cfl"],
               dry_tol=c["dry_tol"])
    out = []
    for prec in (0, 1):
        s = sgn.Solver(c["b"], precision=prec, **cfg)
        s.set_state(c["q"])
        s.step(400)
        assert s.status()[0] == 0
        out.append(s.get_state()[0])
        del s
    q64, qm = out
    wet = (q64[0] - c["b"]) > 1e-3
    err = rel_l2(qm[:3], q64[:3], wet)
    assert err[0] <= 1e-3 and err[1] <= 1e-3 and err[2] <= 1e-3, err
    assert np.abs(qm[0] - q64[0]).max() <= 1e-2 * 2.0


def test_c2_override_matches_oracle(sgn, oracle_mod):
    """A prescribed relaxation field (sgn_set_c2; the constant-c^2 setting of
    the Sec. 5.3 steady-state test, here a varying positive field) gives the
    oracle's result with the same field."""
    b, q = W.random_small_case(2, 48, 36, seed=21, dx=0.05, wetdry=False)
    rng = np.random.default_rng(22)
    c2 = rng.uniform(20.0, 200.0, b.shape)
    cfg = dict(dx=0.05, model=2, bc=(1, 0, 1, 0))
    s = sgn.Solver(b, **cfg)
    s.set_c2(c2)
    s.set_state(q)
    s.step(15)
    o = oracle_mod.Oracle(b, **cfg)
    o.set_c2(c2)
    o.set_state(q)
    assert o.step(15) == 0
    assert (rel_l2(s.get_state()[0], o.get_state()[0]) <= FP64_TOL).all()
    assert np.allclose(s.aux()[0], c2, rtol=0, atol=0)
    with pytest.raises(sgn.SGNError):
        s.set_c2(-c2)
