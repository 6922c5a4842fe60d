"""Pins of the well-prepared initial data (oracle/well_prepared.py, Sec. 3.2)
against closed forms that do not depend on it: the App. B solitary wave (exact
w and p of SGN on a flat bottom) and the mbSGN steady state of the Proposition
of Sec. 5.3 in the limit c^2 -> infinity (exact w and p over varying
bathymetry, which also decides the sign of u d_x b in the constraint, reading
G27); second-order convergence to both; the printed Eq. (constraint p 1D) does
not reproduce the solitary wave (reading G26); and mbHSGN started from
well-prepared data follows the travelling wave more closely than from p = 0."""
import numpy as np
import pytest

from paper_2606_12162_gb300 import workloads as W


@pytest.fixture(scope="module")
def WP(oracle_mod):
    from oracle import well_prepared
    return well_prepared


def _soliton_rows(N, L=40.0, a=0.2, H=1.0):
    dx = L / N
    x = (np.arange(N) + 0.5) * dx
    X, Y = np.meshgrid(x, np.arange(2) * dx)
    b = -H * np.ones_like(X)
    q = W.soliton_state(1, X, Y, b, a, H, 0.5 * L)
    return q, b, dx, x


def test_solitary_wave_w_and_p_second_order(WP):
    ew, ep = [], []
    for N in (200, 400, 800):
        q, b, dx, _ = _soliton_rows(N)
        qw = WP.well_prepared(q, b, dx)
        ew.append(np.abs(qw[3] - q[3]).max() / np.abs(q[3]).max())
        ep.append(np.abs(qw[4] - q[4]).max() / np.abs(q[4]).max())
    for e in (ew, ep):
        rates = np.log2(np.array(e[:-1]) / np.array(e[1:]))
        assert (rates > 1.8).all(), (e, rates)
    assert ep[-1] < 1e-3


def test_printed_relation_does_not_reproduce_the_solitary_wave(WP):
    """Eq. (constraint p 1D) as printed, evaluated with the exact d_t u = -c0 d_x u
    of the travelling wave: no convergence (reading G26)."""
    errs = []
    for N in (400, 800):
        q, b, dx, x = _soliton_rows(N)
        s = W.sgn_soliton(x, 0.0, 0.2, 1.0, 20.0)
        h, u, w = s["h"], s["u"], s["w"]
        D = lambda f: np.gradient(f, dx)
        ut = -s["c0"] * D(u)
        p_printed = -(2 / 3) * D(h * u * w) + (2 / 3) * D(h * u) * w + h / 3 * (-D(h * u) * D(u) + D(ut))
        errs.append(np.abs(p_printed - s["p"]).max() / np.abs(s["p"]).max())
    assert min(errs) > 0.5


def _mbsgn_steady(x, q=1.0, h0=1.0, b0=-1.0, g=9.81):
    """mbSGN steady state (Sec. 5.3 Proposition with c^2 -> infinity) for the
    prescribed w(x) = 2 a3 (x - a1) exp(-a2 (x - a1)^2) (a1 = 20, a2 = 17/5,
    a3 = 3/2) and p = (2/3) q w' (reading G25)."""
    from scipy.integrate import solve_ivp
    a1, a2, a3 = 20.0, 17.0 / 5.0, 1.5
    w = lambda s: 2 * a3 * (s - a1) * np.exp(-a2 * (s - a1) ** 2)
    w1 = lambda s: 2 * a3 * np.exp(-a2 * (s - a1) ** 2) * (1 - 2 * a2 * (s - a1) ** 2)
    w2 = lambda s: 2 * a3 * np.exp(-a2 * (s - a1) ** 2) * (-6 * a2 * (s - a1) + 4 * a2 ** 2 * (s - a1) ** 3)

    def rhs(s, y):
        h, b = y
        P, dP = (2 / 3) * q * w1(s), (2 / 3) * q * w2(s)
        hp = (-h * dP - (g * h + 1.5 * P) * (w(s) * h / q)) / (0.5 * g * h - q * q / h ** 2 + 0.25 * P)
        return [hp, -0.5 * hp + h * w(s) / q]

    sol = solve_ivp(rhs, (0.0, float(x[-1]) + 1.0), [h0, b0], t_eval=x, method="DOP853", rtol=1e-12, atol=1e-13)
    return sol.y[0], sol.y[1], w(x), (2 / 3) * q * w1(x)


def test_steady_state_over_bathymetry_second_order(WP):
    """Steady flow (d_t u = 0) over varying bathymetry: every b term of the
    relation is exercised; w and p converge to the exact ones at second order."""
    ew, ep = [], []
    for N in (400, 800, 1600):
        dx = 40.0 / N
        x = (np.arange(N) + 0.5) * dx
        h, b, w, p = _mbsgn_steady(x)
        qq = np.zeros((5, 2, N))
        B = np.tile(b, (2, 1))
        qq[0] = B + h
        qq[1] = 1.0
        qw = WP.well_prepared(qq, B, dx)
        ew.append(np.abs(qw[3, 0] - h * w).max() / np.abs(h * w).max())
        ep.append(np.abs(qw[4, 0] - h * p).max() / np.abs(h * p).max())
    for e in (ew, ep):
        rates = np.log2(np.array(e[:-1]) / np.array(e[1:]))
        assert (rates > 1.7).all(), (e, rates)


def test_well_prepared_start_follows_the_travelling_wave(WP, oracle_mod):
    """Sec. 3.2: mbHSGN (alpha = 5) from well-prepared data stays closer to the
    SGN solitary wave than from the same h, u with w = p = 0."""
    N = 400
    q, b, dx, x = _soliton_rows(N)
    s = W.sgn_soliton(x, 0.0, 0.2, 1.0, 20.0)
    ill = q.copy()
    ill[3:] = 0.0
    good = WP.well_prepared(ill, b, dx)
    T = 2.0
    errs = []
    for q0 in (good, ill):
        o = oracle_mod.Oracle(b, dx=dx, model=1, bc=(1, 1, 0, 0), alpha=5.0, h_star=0.0, dry_tol=1e-3)
        o.set_state(q0)
        t = 0.0
        while t < T - 1e-12:
            d = min(o.dt_cfl(), T - t)
            assert o.step_dt(d) == 0
            t += d
        h_ex = W.sgn_soliton(x, T, 0.2, 1.0, 20.0)["h"]
        errs.append(np.abs(o.get_state()[0][0, 0] - b[0] - h_ex).max())
    assert errs[0] < 0.5 * errs[1], errs
    del s
