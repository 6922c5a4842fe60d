"""Exact solitary waves of the relaxed systems over a flat bottom (Sec. 5.2,
Table 1) -- test infrastructure, like the rest of oracle/: only tests/,
__graft_entry__.smoke() and bench.py's CPU baseline may import it.

The paper generates its solitary waves of mbHSGN and HSGN by integrating the
travelling-wave ODE of each system with an 8th-order Runge-Kutta method.  This
module writes those ODEs out from the 1-D equations (Eq. mbHSGN, Eq. HSGN of
Sec. 3) for a wave h(x - s t) on still water of depth H (b = -H), and
integrates them with scipy's DOP853 (an explicit 8th-order Runge-Kutta pair).

Travelling-wave relations, xi = x - s t, derivatives d/dxi written ':
  mass:      (h (u - s))' = 0            =>  h u = s (h - H)
  momentum:  (h u (u - s) + g h^2/2 + h p)' = 0
             =>  p(h) = g (H^2 - h^2) / (2 h) + s^2 H (h - H) / h^2
  every advected quantity q obeys (h (u - s) q)' = -s H q'.
mbHSGN (relaxation parameter lam = c^2):
  w'  = -3 p / (2 s H)
  h'  = 2 lam w / (s H (p_h(h) - lam / h))         (from the hp equation)
and w^2 = 3/2 Q(h) - 3 p(h)^2 / (4 lam) with Q(h) = int_H^h p(e)/e de is a first
integral.  A crest of height H + a (w = 0 there) fixes the speed:
  lam h (s^2 / h - g) = (s^2 H / h - g (H + h) / 2)^2,   h = H + a,
whose root nearest g h is taken (s^2 -> g (H + a), the SGN speed of App. B,
as lam -> infinity).  The profile is integrated from the crest (h = H + a,
w = 0), where the ODE is regular, and mirrored: h is even, w odd in xi.

HSGN: the same h u and p(h); with k = 1 / (s H):
  h'   = lam sigma k / (p_h(h) - lam / h)
  w'   = -k p_b
  sigma' = k (6 p_b - 12 p(h))
  p_b' = 6 lam k (w - sigma / 2)
The rest state has one real unstable direction (and a neutral oscillatory
pair), as the paper's construction from a perturbation along the unstable
manifold requires.  For a trial speed s the orbit leaving the rest state along
that direction is integrated to its crest (sigma = 0, i.e. h' = 0); s is
adjusted (root finding) until the crest height is H + a.  The system is
reversible (h, p_b even; w, sigma odd in xi), so the front is the mirror image
of the rear; w at the crest (returned) measures how far the orbit misses the
symmetric section and comes out at rounding level.
"""
import functools
import math

import numpy as np
from scipy.integrate import solve_ivp
from scipy.optimize import brentq

G = 9.81


def _p(h, s2, H, g):
    return g * (H * H - h * h) / (2.0 * h) + s2 * H * (h - H) / (h * h)


def _p_h(h, s2, H, g):
    return -g * (H * H + h * h) / (2.0 * h * h) + s2 * H * (2.0 * H - h) / h ** 3


def mbhsgn_speed2(a, H, lam, g=G):
    """s^2 of the mbHSGN solitary wave of crest height H + a (first integral at the crest)."""
    h = H + a
    A, B = H / h, g * (H + h) / 2.0
    b1 = 2.0 * A * B + lam
    c0 = B * B + lam * g * h
    disc = b1 * b1 - 4.0 * A * A * c0
    return 2.0 * c0 / (b1 + math.sqrt(disc))     # the smaller root, stably


def _dense_half(rhs, y0, L_half, rtol=1e-13, atol=1e-15):
    sol = solve_ivp(rhs, (0.0, L_half), y0, method="DOP853", rtol=rtol, atol=atol, dense_output=True)
    if sol.status != 0:
        raise RuntimeError("travelling-wave integration failed: " + sol.message)
    return sol.sol


def mbhsgn_wave(a, H, lam, L_half, g=G):
    """Returns (s, f) where f(xi) -> (h, hu, hw, hp) of the exact mbHSGN wave,
    valid for |xi| <= L_half."""
    s2 = mbhsgn_speed2(a, H, lam, g)
    s = math.sqrt(s2)

    def rhs(_, y):
        h, w = y
        return [2.0 * lam * w / (s * H * (_p_h(h, s2, H, g) - lam / h)), -1.5 * _p(h, s2, H, g) / (s * H)]

    half = _dense_half(rhs, [H + a, 0.0], L_half)

    def f(xi):
        xi = np.asarray(xi, dtype=np.float64)
        y = half(np.abs(xi).ravel()).reshape((2,) + xi.shape)
        h = y[0]
        w = np.sign(xi) * y[1]
        p = _p(h, s2, H, g)
        return h, s * (h - H), h * w, h * p

    return s, f


def mbhsgn_first_integral(h, w, s, H, lam, g=G):
    """w^2 - (3/2 Q(h) - 3 p^2 / (4 lam)); zero along the exact wave."""
    s2 = s * s
    Q = g * (H - H * H / (2.0 * h) - h / 2.0) + s2 * H * (1.0 / (2.0 * H) - 1.0 / h + H / (2.0 * h * h))
    p = _p(h, s2, H, g)
    return w * w - (1.5 * Q - 0.75 * p * p / lam)


def hsgn_linear_rates(s, H, lam, g=G):
    """Eigenvalues of the HSGN travelling-wave ODE linearised at the rest state."""
    s2 = s * s
    k = 1.0 / (s * H)
    ph = _p_h(H, s2, H, g)
    a1 = lam * k / (ph - lam / H)
    # variables (e, w, sigma, p_b), e = h - H; p ~ ph e
    M = np.array([[0.0, 0.0, a1, 0.0],
                  [0.0, 0.0, 0.0, -k],
                  [-12.0 * k * ph, 0.0, 0.0, 6.0 * k],
                  [0.0, 6.0 * lam * k, -3.0 * lam * k, 0.0]])
    return np.linalg.eigvals(M)


def _hsgn_rhs(s, H, lam, g):
    s2 = s * s
    k = 1.0 / (s * H)

    def rhs(_, y):
        h, w, sg, pb = y
        return [lam * sg * k / (_p_h(h, s2, H, g) - lam / h), -k * pb,
                k * (6.0 * pb - 12.0 * _p(h, s2, H, g)), 6.0 * lam * k * (w - 0.5 * sg)]
    return rhs


def _hsgn_unstable(s, H, lam, g):
    """Growth rate and unit eigenvector (e-component > 0) of the one real
    positive eigenvalue of the linearisation at rest."""
    s2 = s * s
    k = 1.0 / (s * H)
    ph = _p_h(H, s2, H, g)
    a1 = lam * k / (ph - lam / H)
    M = np.array([[0.0, 0.0, a1, 0.0], [0.0, 0.0, 0.0, -k], [-12.0 * k * ph, 0.0, 0.0, 6.0 * k],
                  [0.0, 6.0 * lam * k, -3.0 * lam * k, 0.0]])
    ev, V = np.linalg.eig(M)
    i = int(np.argmax(ev.real))
    if abs(ev[i].imag) > 1e-12 * abs(ev[i].real) or ev[i].real <= 0:
        raise ValueError("no real unstable direction at this speed")
    v = V[:, i].real
    v = v / np.linalg.norm(v)
    return ev[i].real, (v if v[0] > 0 else -v)


def _hsgn_to_crest(s, H, lam, g, eps):
    """Orbit leaving the rest state along its unstable direction (offset eps),
    integrated to the crest (sigma = 0 upward crossing, i.e. h' = 0)."""
    kap, v = _hsgn_unstable(s, H, lam, g)
    y0 = np.array([H, 0.0, 0.0, 0.0]) + eps * v
    ev = lambda _, y: y[2]
    ev.terminal, ev.direction = True, 1.0
    span = 5.0 * math.log(1.0 / eps) / kap + 50.0
    sol = solve_ivp(_hsgn_rhs(s, H, lam, g), (0.0, span), y0, method="DOP853", rtol=1e-13, atol=1e-16,
                    dense_output=True, events=ev)
    if sol.status != 1 or len(sol.t_events[0]) == 0:
        raise RuntimeError("no crest reached")
    return sol, sol.t_events[0][0], sol.y_events[0][0], kap, v


@functools.lru_cache(maxsize=16)
def hsgn_wave(a, H, lam, g=G, eps=1e-12):
    """Returns (s, f, crest) where f(xi) -> (h, hu, hw, hsigma, hp, hp_b) of the
    HSGN solitary wave of crest height H + a with its crest at xi = 0 (any xi;
    beyond the integrated orbit the linear unstable manifold), and crest is the
    ODE state (h, w, sigma, p_b) reached at the crest."""
    s_sgn = math.sqrt(g * (H + a))
    amp = lambda s: _hsgn_to_crest(s, H, lam, g, eps)[2][0] - H - a
    s = brentq(amp, s_sgn * 0.98, s_sgn * 1.02, xtol=1e-15, rtol=1e-15, maxiter=200)
    sol, xc, yc, kap, v = _hsgn_to_crest(s, H, lam, g, eps)
    s2 = s * s

    def rear(xi):          # xi <= 0: the integrated orbit, before it the linear manifold
        t = xc + xi
        y = np.empty((4,) + xi.shape)
        inside = t >= 0.0
        if inside.any():
            y[:, inside] = sol.sol(t[inside])
        if (~inside).any():
            y[:, ~inside] = (np.array([H, 0.0, 0.0, 0.0])[:, None] +
                             eps * v[:, None] * np.exp(kap * t[~inside])[None, :])
        return y

    def f(xi):
        xi = np.asarray(xi, dtype=np.float64)
        y = rear(-np.abs(xi).ravel()).reshape((4,) + xi.shape)
        sgn = np.where(xi > 0, -1.0, 1.0)      # w, sigma odd in xi
        h, w, sg, pb = y[0], sgn * y[1], sgn * y[2], y[3]
        p = _p(h, s2, H, g)
        return h, s * (h - H), h * w, h * sg, h * p, h * pb

    return s, f, yc


def periodic_state(model, x, f, x0, L, H):
    """State (nvar, ny, nx) of a wave profile f (from mbhsgn_wave, model 1, or
    hsgn_wave, model 2) with its crest at x0 on a periodic domain of length L,
    in the field order eta, hu, hv, hw[, hsigma], hp[, hp_b]; eta = h - H."""
    xi = (x - x0 + 0.5 * L) % L - 0.5 * L
    r = f(xi)
    q = np.zeros((5 if model == 1 else 7,) + np.shape(x))
    q[0] = r[0] - H
    q[1] = r[1]
    q[3:] = np.array(r[2:])
    return q
