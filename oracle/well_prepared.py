"""Well-prepared initial data for mbHSGN (Sec. 3.2): w from the mbSGN constraint
(Eq. (closed-form w mbSGN)) and p from the linear relation of Sec. 3.2 with
d_t u eliminated by Eq. (ut 1D), for data that vary along x only.

TEST INFRASTRUCTURE ONLY (like the rest of oracle/): the plain FP64 definition
the library's well-prepared kernel is checked against.

Reading G27: Eq. (closed-form w mbSGN) prints (w + u d_x b); Eq. (mbHSGN),
whose relaxation enforces the constraint, has (w - u d_x b), and so does the
kinematic condition (a linear vertical profile from u d_x b at the bottom):
w = -(h/2) d_x u + u d_x b is used.

Reading G26: Eq. (constraint p 1D) as printed is dimensionally inconsistent
(h d_x d_t u is not a pressure) and, evaluated on the exact solitary wave of
App. B, gives about -0.8 times its p.  The relation is re-derived from the
same two equations the paper names -- the hw equation of Eq. (Bristeau),
p = (2/3) [d_t(h w) + d_x(u h w)], and the constraint above -- with
d_t h = -d_x(h u):
    p = (2/3) D(h u w) - (2/3) D(h u) w + (h/3) D(h u) D u
        - (h^2/3) d_x d_t u + (2h/3) d_t u D b,
which reproduces the App. B solitary wave exactly (checked symbolically).
Eq. (ut 1D) is used as printed (it holds on that wave):
    d_t u = A + L[p],
    A    = (1/h) [ -D(h u^2 + g h^2 / 2) - g h D b + u D(h u) ],
    L[p] = -(1/h) [ D(h p) + (3/2) p D b ],
so that
    p + (h^2/3) d_x L[p] - (2h/3) L[p] D b = F - (h^2/3) D A + (2h/3) A D b,
    F = (2/3) D(h u w) - (2/3) D(h u) w + (h/3) D(h u) D u,
with d_x L[p] = -d_x[(1/h) d_x(h p)] - (3/2) D(p D b / h).

Discretisation (the paper leaves it open; the library uses the same one):
every row is extended by one copied cell at each end (zero gradient), D is the
central difference (f[i+1] - f[i-1]) / (2 dx); d_x[(1/h) d_x(h p)] is the
compact difference ((h p)[i+1] - (h p)[i]) / h[i+1/2] - ((h p)[i] - (h p)[i-1])
/ h[i-1/2], over dx^2, h[i+1/2] the mean of the two cells; p then solves one
tridiagonal system per row.
"""
import numpy as np
from scipy.linalg import solve_banded


def _ext(a):
    return np.concatenate([a[..., :1], a, a[..., -1:]], axis=-1)


def _D(ae, dx):
    """Central difference of an extended row (length n + 2) at the n cells."""
    return (ae[..., 2:] - ae[..., :-2]) / (2.0 * dx)


def well_prepared_row(h, u, b, dx, g=9.81):
    """w and p of one row (1-D arrays of the n cells).  Returns (w, p)."""
    n = h.size
    he, ue, be = _ext(h), _ext(u), _ext(b)
    Db = _D(be, dx)
    Du = _D(ue, dx)
    w = -0.5 * h * Du + u * Db                               # constraint, reading G27
    we = _ext(w)
    hu_e = he * ue
    Dhu = _D(hu_e, dx)
    F = (2.0 / 3.0) * _D(hu_e * we, dx) - (2.0 / 3.0) * Dhu * w + (h / 3.0) * Dhu * Du
    A = (-_D(he * ue * ue + 0.5 * g * he * he, dx) - g * h * Db + u * Dhu) / h
    DA = _D(_ext(A), dx)
    rhs = F - (h * h / 3.0) * DA + (2.0 * h / 3.0) * A * Db
    # tridiagonal operator M p = p + (h^2/3) d_x L[p] - (2h/3) L[p] D b (zero-gradient ends)
    Dbe = _ext(Db)
    hh = 0.5 * (he[1:] + he[:-1])                              # h at the n + 1 faces
    lo = np.zeros(n)                                           # coefficient of p[i-1]
    di = np.ones(n)                                            # coefficient of p[i]
    up = np.zeros(n)                                           # coefficient of p[i+1]
    for i in range(n):
        I = i + 1                                              # index in the extended row
        # -d_x[(1/h) d_x(h p)]  ->  -( (hp[I+1]-hp[I])/hh[I] - (hp[I]-hp[I-1])/hh[I-1] ) / dx^2
        cm = he[I - 1] / hh[I - 1] / dx ** 2
        cp = he[I + 1] / hh[I] / dx ** 2
        c0 = -he[I] * (1.0 / hh[I] + 1.0 / hh[I - 1]) / dx ** 2
        # dxL = -(cm p[I-1] + c0 p[I] + cp p[I+1]) - 1.5 (p[I+1] Db[I+1]/h[I+1] - p[I-1] Db[I-1]/h[I-1]) / (2 dx)
        dxL_m = -cm + 1.5 * Dbe[I - 1] / he[I - 1] / (2.0 * dx)
        dxL_0 = -c0
        dxL_p = -cp - 1.5 * Dbe[I + 1] / he[I + 1] / (2.0 * dx)
        # L[p][i] Db[i] = -(Db/h) [ (h[I+1] p[I+1] - h[I-1] p[I-1]) / (2 dx) + 1.5 p[I] Db ]
        L_m = (Db[i] / h[i]) * he[I - 1] / (2.0 * dx)
        L_0 = -(Db[i] / h[i]) * 1.5 * Db[i]
        L_p = -(Db[i] / h[i]) * he[I + 1] / (2.0 * dx)
        k1, k2 = h[i] * h[i] / 3.0, -2.0 * h[i] / 3.0
        cmi = k1 * dxL_m + k2 * L_m
        c0i = 1.0 + k1 * dxL_0 + k2 * L_0
        cpi = k1 * dxL_p + k2 * L_p
        # zero-gradient ends: the copied cell is the edge cell itself
        if i == 0:
            c0i += cmi
            cmi = 0.0
        if i == n - 1:
            c0i += cpi
            cpi = 0.0
        lo[i], di[i], up[i] = cmi, c0i, cpi
    ab = np.zeros((3, n))
    ab[0, 1:] = up[:-1]
    ab[1] = di
    ab[2, :-1] = lo[1:]
    p = solve_banded((1, 1), ab, rhs)
    return w, p


def well_prepared(q, b, dx, g=9.81, dry_tol=1e-3):
    """mbHSGN state q (5, ny, nx; eta, hu, hv, hw, hp) with hw and hp replaced by
    the well-prepared values of every row (x-direction relation; rows with a
    dry cell are left unchanged)."""
    q = np.array(q, dtype=np.float64, copy=True)
    for j in range(q.shape[1]):
        h = q[0, j] - b[j]
        if not (h > dry_tol).all():
            continue
        u = q[1, j] / h
        w, p = well_prepared_row(h, u, b[j], dx, g)
        q[3, j] = h * w
        q[4, j] = h * p
    return q
