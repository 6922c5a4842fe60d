"""Pin of the bathymetry sharpness sensor psi by its effect (App. F).

App. F runs an SGN solitary wave over the smoothed step
b(x) = 0.05 (erf(32 x) + 1) - H, H = 0.2 m: crossing the step generates
high-frequency oscillations that, on grids that do not resolve the step, can
grow into an instability; the sensor switches the non-hydrostatic bathymetry
coupling off at faces whose relative bathymetry jump is large, which
suppresses them, and leaves smooth or resolved bathymetry untouched.

Observable: the total variation of eta over the step region [-0.5, 1] m after
the wave has left it (t = 4, 5, 6 s; the crest is past x = 2 m by t = 4 s),
HSGN with alpha = 3, a = 0.02 m, on a grid of dx = 0.03 m (the step is about two
cells wide, so the steepest faces have xi ~ 0.3 > xi0 + xi1 and psi = 0 there).
Pinned:
  - with the sensor the residual variation is at least 3x smaller than without
    it at every output time (measured 4.1x, 14x, 30x);
  - without it the variation grows in time (the instability the appendix warns
    of), with it it decays;
  - at rest over the same step both stay exactly at rest (psi never touches the
    hydrostatic balance);
  - a planted mistake -- psi = 1 instead of 0 beyond the smoothstep band, i.e.
    no cut-off at sharp steps -- compiled into a copy of the oracle fails the
    first two.
"""
import importlib.util
import os
import subprocess

import numpy as np
import pytest
from scipy.special import erf

from paper_2606_12162_gb300 import workloads as W

H, A, DX, X0 = 0.2, 0.02, 0.03, -1.5
TIMES = (4.0, 5.0, 6.0)


def _setup(L0=-4.0, L1=6.0):
    nx = int(round((L1 - L0) / DX))
    x = L0 + (np.arange(nx) + 0.5) * DX
    X = np.tile(x, (2, 1))
    b = 0.05 * (erf(32.0 * X) + 1.0) - H
    # SGN solitary wave (App. B) on the deep side, depth H under it
    q = W.soliton_state(W.HSGN, X, np.zeros_like(X), np.full_like(X, -H), A, H, X0)
    return x, b, q


def _run(O, sensor, rest=False):
    x, b, q = _setup()
    if rest:
        q = W.rest_state(b, W.HSGN)
    kw = dict(dx=DX, model=W.HSGN, bc=(1, 1, 0, 0), h_star=0.0, alpha=3.0)
    if not sensor:
        kw["xi0"] = 1e9                 # psi = 1 at every face
    o = O.Oracle(b, **kw)
    o.set_state(q)
    out, t = {}, 0.0
    for te in TIMES:
        while t < te - 1e-12:
            dt = min(o.dt_cfl(), te - t)
            assert o.step_dt(dt) == 0
            t += dt
        out[te] = o.get_state()[0]
    return x, b, out


def _variation(O):
    """Total variation of eta over [-0.5, 1] m at the output times, with and without the sensor."""
    res = {}
    for sensor in (True, False):
        x, _, out = _run(O, sensor)
        win = (x > -0.5) & (x < 1.0)
        res[sensor] = np.array([np.abs(np.diff(out[te][0][0][win])).sum() for te in TIMES])
    return res


def _pin_holds(tv):
    on, off = tv[True], tv[False]
    return bool((off >= 3.0 * on).all() and off[-1] > 2.0 * off[0] and on[-1] < on[0])


def test_sensor_suppresses_step_oscillations(oracle_mod):
    tv = _variation(oracle_mod)
    assert _pin_holds(tv), tv


def test_sensor_keeps_rest_over_the_step(oracle_mod):
    for sensor in (True, False):
        _, b, out = _run(oracle_mod, sensor, rest=True)
        q = out[TIMES[-1]]
        assert np.abs(q[0]).max() == 0.0 and np.abs(q[1:]).max() == 0.0


def test_planted_sensor_mistake_fails_the_pin(tmp_path):
    """A copy of the oracle whose psi returns 1 beyond the smoothstep band."""
    here = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")
    src = open(os.path.join(here, "sgn_oracle.c")).read()
    i = src.index("double or_psi(")
    j = src.index("return 0.0;\n}", i)
    planted = src[:j] + "return 1.0;\n}" + src[j + len("return 0.0;\n}"):]
    (tmp_path / "sgn_oracle.c").write_text(planted)
    for f in os.listdir(here):
        if f.endswith(".h"):
            (tmp_path / f).write_text(open(os.path.join(here, f)).read())
    lib = str(tmp_path / "liboracle_planted.so")
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
                           "-o", lib, str(tmp_path / "sgn_oracle.c"), "-lm"])
    spec = importlib.util.spec_from_file_location("oracle_planted", os.path.join(here, "oracle.py"))
    P = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(P)
    P.LIB = lib
    P.build = lambda force=False: lib
    assert P.psi(-0.1, -0.2) == 1.0          # the planted branch is the one taken at this jump
    tv = _variation(P)
    assert not _pin_holds(tv), tv
