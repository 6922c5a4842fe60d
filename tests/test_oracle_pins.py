"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Unit-level pins: the printed eigenstructure of App. C, the quasi-linear form of
Eq. (mbHSGN)/(HSGN), the f-wave decomposition identity, the bathymetry sensor,
the transition function (brute force), and the SDIRK(2,2) source integrator.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

GOLD = os.path.join(os.path.dirname(__file__), "golden")
G = 9.81


def _app_c():
    with open(os.path.join(GOLD, "app_c_eigenstructure.json")) as f:
        return json.load(f)


def _eval_matrix(rows, env):
    return np.array([[eval(e, {"__builtins__": {}}, env) for e in r] for r in rows], dtype=float)


def _random_state(rng, hsgn):
    h = rng.uniform(0.2, 3.0)
    st = dict(h=h, u=rng.uniform(-1, 1), v=rng.uniform(-1, 1), w=rng.uniform(-0.3, 0.3),
              sigma=rng.uniform(-0.3, 0.3) if hsgn else 0.0, p=rng.uniform(-0.5, 0.5),
              pb=rng.uniform(-0.5, 0.5) if hsgn else 0.0, c2=rng.uniform(0.0, 50.0), g=G)
    st["C"] = math.sqrt(G * h + st["p"] + st["c2"])
    return st


# Our wave order: fast-, r2, passive (v, w[, sigma, pb]), fast+.
PERM = {"mbhsgn": [0, 1, 3, 2, 4], "hsgn": [0, 1, 4, 3, 2, 5, 6]}


@pytest.mark.parametrize("name,model", [("mbhsgn", 1), ("hsgn", 2)])
def test_eigenvectors_match_app_c(oracle_mod, name, model):
    """R built by the oracle (with s1 = u - C, sN = u + C) times the printed R^-1
    of App. C is the identity, and the printed Jacobian has R as eigenvectors."""
    O = oracle_mod
    A = _app_c()[name]
    rng = np.random.default_rng(7)
    for _ in range(20):
        st = _random_state(rng, model == 2)
        roe = [st[k] for k in ("h", "u", "v", "w", "sigma", "p", "pb", "c2")]
        R = O.eigvecs(model, roe, st["u"] - st["C"], st["u"] + st["C"])
        Rp = _eval_matrix(A["R"], st)
        Rinv = _eval_matrix(A["Rinv"], st)
        perm = PERM[name]
        assert np.allclose(R, Rp[:, perm], atol=1e-14, rtol=0)
        assert np.allclose(Rinv[perm, :] @ R, np.eye(len(perm)), atol=1e-12)
        Jp = _eval_matrix(A["jacobian"], st)
        lam = np.array([eval(e, {"__builtins__": {}}, st) for e in A["eigenvalues"]])[perm]
        assert np.allclose(Jp @ R, R * lam[None, :], atol=1e-11)
        # the oracle's own quasi-linear matrix is the printed one
        J = O.jacobian(model, roe)
        assert np.allclose(J, Jp, atol=1e-13)


def _cfg(O, model, **kw):
    return O.make_config(4, 4, 1.0, model=model, **kw)


@pytest.mark.parametrize("model", [0, 1, 2])
def test_fwaves_sum_to_total_fluctuation(oracle_mod, model):
    """The f-waves recombine into the total fluctuation: sum_p Z_p = delta, and
    A^- + A^+ = delta (Sec. 4, f-wave decomposition)."""
    O = oracle_mod
    cfg = _cfg(O, model)
    rng = np.random.default_rng(11 + model)
    nv = O.NVAR[model]
    for _ in range(50):
        bL, bR = -rng.uniform(0.5, 3.0), -rng.uniform(0.5, 3.0)
        qL = np.zeros(nv); qR = np.zeros(nv)
        for q, b in ((qL, bL), (qR, bR)):
            h = rng.uniform(0.1, 2.0)
            q[0] = h + b
            q[1:] = h * rng.uniform(-0.4, 0.4, nv - 1)
        c2L, c2R = rng.uniform(0, 40), rng.uniform(0, 40)
        r = O.face(cfg, qL, qR, bL, bR, c2L, c2R)
        d = r["delta"]
        scale = np.abs(d).max() + 1e-30
        assert np.allclose(r["Z"].sum(axis=0), d, atol=1e-13 * scale)
        assert np.allclose(r["Am"] + r["Ap"], d, atol=1e-13 * scale)
        # Einfeldt speeds bracket the contact speed
        assert r["s"][0] <= r["s"][1] <= r["s"][-1]


def _prim_to_cons(model, h, b, prim):
    """prim = (u, v, w, sigma, p, pb) -> conserved (eta, hu, hv, ...)."""
    u, v, w, sg, p, pb = prim
    if model == 0:
        return np.array([h + b, h * u, h * v])
    if model == 1:
        return np.array([h + b, h * u, h * v, h * w, h * p])
    return np.array([h + b, h * u, h * v, h * w, h * sg, h * p, h * pb])


@pytest.mark.parametrize("name,model", [("mbhsgn", 1), ("hsgn", 2)])
def test_total_fluctuation_is_quasilinear_form(oracle_mod, name, model):
    """For a small jump dq (flat bottom, constant c^2) the total fluctuation tends to
    (dF/dq + A) dq with the Jacobian printed in App. C; for a small bathymetry jump
    db at rest in the conserved variables it tends to the bathymetry vector B db read
    off Eq. (mbHSGN)/(HSGN): (0, g h + 3p/2, 0, 0, -2 c^2 u) resp.
    (0, g h + p_b, 0, 0, 0, 0, -6 c^2 u), with the sensor psi -> 1."""
    O = oracle_mod
    A = _app_c()[name]
    cfg = _cfg(O, model, xi0=0.5, xi1=0.5)
    rng = np.random.default_rng(3)
    nv = O.NVAR[model]
    for _ in range(10):
        st = _random_state(rng, model == 2)
        prim = [st["u"], st["v"], st["w"], st["sigma"], st["p"], st["pb"]]
        b = -st["h"] - 0.5
        qL = _prim_to_cons(model, st["h"], b, prim)
        Jp = _eval_matrix(A["jacobian"], st)
        for k in range(nv):
            for eps in (1e-5, 1e-6):
                qR = qL.copy()
                qR[k] += eps
                r = O.face(cfg, qL, qR, b, b, st["c2"], st["c2"])
                # dq in (h, hu, ...) variables equals the eta jump for field 0
                err = np.abs(r["delta"] / eps - Jp[:, k]).max()
                assert err < 50 * eps * (1 + np.abs(Jp).max()), (k, eps, err)
        # bathymetry jump with h, hu, ... fixed (eta jumps by db as well)
        Bv = np.zeros(nv)
        Bv[1] = G * st["h"] + (1.5 * st["p"] if model == 1 else st["pb"])
        if model == 1:
            Bv[4] = -2.0 * st["c2"] * st["u"]
        else:
            Bv[6] = -6.0 * st["c2"] * st["u"]
        eps = 1e-7
        qR = qL.copy(); qR[0] += eps
        r = O.face(cfg, qL, qR, b, b + eps, st["c2"], st["c2"])
        assert np.abs(r["delta"] / eps - Bv).max() < 1e-4 * (1 + np.abs(Bv).max())


def test_swe_face_is_two_wave_hlle(oracle_mod):
    """With c^2 = 0 and no pressure the model is the SWE (Sec. 3.3: c^2 -> 0): only
    the two fast waves and the passive tangential wave carry the jump."""
    O = oracle_mod
    cfg = _cfg(O, 0)
    qL = np.array([0.3, 0.2, 0.05]); qR = np.array([0.1, -0.1, 0.02])
    r = O.face(cfg, qL, qR, -1.0, -1.2, 0.0, 0.0)
    hL, hR = 1.3, 1.3
    uL, uR = 0.2 / hL, -0.1 / hR
    # Einfeldt speeds of Sec. 4 with Roe averages
    hh = 0.5 * (hL + hR)
    uh = (math.sqrt(hR) * uR + math.sqrt(hL) * uL) / (math.sqrt(hR) + math.sqrt(hL))
    s1 = min(uh - math.sqrt(G * hh), uL - math.sqrt(G * hL))
    s2 = max(uh + math.sqrt(G * hh), uR + math.sqrt(G * hR))
    assert r["s"][0] == pytest.approx(s1, rel=1e-14) and r["s"][-1] == pytest.approx(s2, rel=1e-14)
    # HLLE f-wave amplitudes for (h, hu): beta1 + beta2 = d_h, s1 beta1 + s2 beta2 = d_hu
    d = r["delta"]
    b2 = (d[1] - s1 * d[0]) / (s2 - s1)
    assert r["Z"][-1][0] == pytest.approx(b2, rel=1e-13)
    # well-balanced momentum term: d_hu = Delta(hu^2/h) + g hhat Delta eta
    assert d[1] == pytest.approx((-0.1 * uR - 0.2 * uL) + G * hh * (0.1 - 0.3), rel=1e-13)


def test_sensor_psi(oracle_mod):
    """Sensor of Sec. 4: psi = 1 below xi0, 0 above xi0 + xi1, cubic smoothstep in
    between; C^1 at both ends; psi = 0 when b_i + b_{i-1} = 0 (reading)."""
    O = oracle_mod
    xi0, xi1 = 0.01, 0.05

    def at(xi):
        # b_R, b_L with 2|bR-bL|/|bR+bL| = xi
        bL = -1.0
        bR = bL * (2 + xi) / (2 - xi)
        return O.psi(bR, bL, xi0, xi1)

    assert at(0.0) == 1.0 and at(0.009) == 1.0
    assert at(0.07) == 0.0 and at(1.0) == 0.0
    assert at(xi0 + 0.5 * xi1) == pytest.approx(0.5, abs=1e-12)
    assert at(xi0 + 0.25 * xi1) == pytest.approx(1 - 3 * 0.0625 + 2 * 0.015625, abs=1e-12)
    e = 1e-6   # C^1: the deviation from the end values is quadratic in e
    assert abs(at(xi0 + e) - 1.0) < 4 * (e / xi1) ** 2 and abs(at(xi0 + xi1 - e)) < 4 * (e / xi1) ** 2
    assert O.psi(1.0, -1.0, xi0, xi1) == 0.0
    # symmetric in its arguments
    assert O.psi(-2.0, -2.05, xi0, xi1) == O.psi(-2.05, -2.0, xi0, xi1)


def test_transition_function_brute_force(oracle_mod):
    """phi_T of Eq. (transition_function) with n = 1 and n = 2 against a brute-force
    evaluation of the definition (reading: centres within n dx, eta0 = 0)."""
    O = oracle_mod
    rng = np.random.default_rng(5)
    ny, nx = 9, 11
    b = rng.uniform(-40.0, 5.0, size=(ny, nx))
    for n in (1, 2):
        for hstar in (0.0, 10.0, 20.0):
            o = O.Oracle(b, dx=1.0, model=1, h_star=hstar, n_transition=n, bc=(1, 1, 1, 1))
            c2, phi = o.aux()
            bp = np.pad(b, n, mode="edge")   # extrapolation boundaries copy the edge
            ref = np.zeros_like(phi)
            for j in range(ny):
                for i in range(nx):
                    vals = [max(0.0, -bp[j + n + dj, i + n + di])
                            for dj in range(-n, n + 1) for di in range(-n, n + 1) if di * di + dj * dj <= n * n]
                    ref[j, i] = 1 if min(vals) > hstar else 0
            assert np.array_equal(phi, ref)
            assert np.allclose(c2, 9.0 * G * np.maximum(0.0, -b) * ref, rtol=1e-15, atol=0)


GAM = 1.0 - 1.0 / math.sqrt(2.0)


def _R_stab(z):
    """Stability function of SDIRK(2,2) (two stages, gamma = 1 - 1/sqrt 2)."""
    return (1 + (1 - 2 * GAM) * z) / (1 - GAM * z) ** 2


def test_sdirk_mbhsgn_energy_factor(oracle_mod):
    """mbHSGN source: the exact flow conserves E = 4c^2 w^2/3 + p^2 (a rotation with
    omega = sqrt(3) c / h); one SDIRK(2,2) step scales E by |R(i omega tau)|^2."""
    O = oracle_mod
    rng = np.random.default_rng(1)
    for _ in range(20):
        h, c2, tau = rng.uniform(0.5, 5), rng.uniform(1, 100), rng.uniform(1e-3, 0.2)
        w, p = rng.uniform(-1, 1), rng.uniform(-1, 1)
        y = O.source(1, h, c2, tau, [w, p])
        E0 = 4 * c2 * w * w / 3 + p * p
        E1 = 4 * c2 * y[0] ** 2 / 3 + y[1] ** 2
        om = math.sqrt(3.0 * c2) / h
        assert E1 / E0 == pytest.approx(abs(_R_stab(1j * om * tau)) ** 2, rel=1e-12)


@pytest.mark.parametrize("model", [1, 2])
def test_sdirk_is_stability_function_and_second_order(oracle_mod, model):
    """On the linear source system y' = M y of Eq. (mbHSGN)/(HSGN) one SDIRK(2,2) step
    is R(tau M) y, and it converges at order 2 to the exact matrix exponential."""
    O = oracle_mod
    h, c2 = 1.3, 40.0
    if model == 1:
        M = np.array([[0, 1.5 / h], [-2 * c2 / h, 0]])
        y0 = np.array([0.2, -0.4])
    else:
        M = np.array([[0, 0, 0, 1 / h], [0, 0, 12 / h, -6 / h], [0, -c2 / h, 0, 0],
                      [-6 * c2 / h, 3 * c2 / h, 0, 0]])
        y0 = np.array([0.2, -0.1, 0.3, -0.4])
    n = len(y0)
    Id = np.eye(n)
    errs = []
    for tau in (0.004, 0.002, 0.001):
        y = O.source(model, h, c2, tau, y0)
        Rm = np.linalg.solve(Id - GAM * tau * M, np.linalg.solve(Id - GAM * tau * M, Id + (1 - 2 * GAM) * tau * M))
        assert np.allclose(y, Rm @ y0, rtol=1e-12, atol=1e-14)
        errs.append(np.abs(y - scipy.linalg.expm(tau * M) @ y0).max())
    r1, r2 = math.log2(errs[0] / errs[1]), math.log2(errs[1] / errs[2])
    assert 2.7 < r1 < 3.3 and 2.7 < r2 < 3.3  # local error O(tau^3) = global order 2


@pytest.mark.parametrize("model", [1, 2])
def test_uniform_current_is_steady_for_any_relaxation_field(oracle_mod, model):
    """Reading G24 (the relaxation term h c^2 d_x u with c^2 outside the
    derivative, as the relaxed divergence constraint d_t p + u d_x p = -c^2 d_x u
    + ... gives it) against the flux form d_x[h u (p + c^2)]: they differ by
    h u d_x c^2, which vanishes only for constant c^2.  A uniform current over a
    flat bottom (h, u uniform, w = sigma = p = p_b = 0) is the SGN solution with
    zero non-hydrostatic pressure, and with c^2 outside the derivative it is an
    exact steady solution of the relaxed systems for every c^2(x); the flux form
    would drive p by u h d_x c^2.  Face level: a face between two copies of the
    same current with different c^2 carries no fluctuation (the flux form gives
    delta_hp = h u (c2R - c2L)).  Whole step: with a smooth, strongly varying
    c^2 field (sgn_set_c2's setting, no SWE transition) the oracle keeps the
    current to round-off over 40 steps."""
    O = oracle_mod
    h, u, v = 1.3, 0.7, -0.2
    b = -h
    nv = O.NVAR[model]
    q = np.zeros(nv)
    q[0], q[1], q[2] = h + b, h * u, h * v
    cfg = _cfg(O, model)
    r = O.face(cfg, q, q, b, b, 20.0, 80.0)
    assert np.abs(r["delta"]).max() == 0.0
    assert np.abs(r["Am"]).max() == 0.0 and np.abs(r["Ap"]).max() == 0.0
    # the flux form's fluctuation of hp here would be h u (c2R - c2L) = 54.6: far from 0
    # whole step over a varying c^2 field, periodic in x and y
    nx, ny, dx = 96, 8, 0.05
    x = (np.arange(nx) + 0.5) * dx
    c2 = np.tile(60.0 + 45.0 * np.sin(2 * np.pi * x / (nx * dx)), (ny, 1))
    bb = np.full((ny, nx), b)
    qs = np.zeros((nv, ny, nx))
    qs[0], qs[1], qs[2] = h + b, h * u, h * v
    o = O.Oracle(bb, dx=dx, model=model, bc=(2, 2, 2, 2), h_star=0.0)
    o.set_c2(c2)
    o.set_state(qs)
    assert o.step(40) == 0
    qe, _ = o.get_state()
    assert np.abs(qe - qs).max() <= 1e-13 * (1 + np.abs(qs).max())
    assert np.abs(qe[3:]).max() <= 1e-13
