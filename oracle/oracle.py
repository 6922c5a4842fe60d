"""ctypes wrapper of the FP64 CPU oracle (oracle/sgn_oracle.c).

Test infrastructure only: imported by tests/, by __graft_entry__.smoke() and by
bench.py's cpu_baseline / reference leg, never by the CUDA product path.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
SRC = [os.path.join(HERE, "sgn_oracle.c")]

SWE, MBHSGN, HSGN = 0, 1, 2
WALL, EXTRAP, PERIODIC = 0, 1, 2
MINMOD, MC, NOLIMIT = 0, 1, 2
NVAR = {SWE: 3, MBHSGN: 5, HSGN: 7}

ST_NEGDEPTH, ST_NONFINITE, ST_CFL, ST_NONHYP, ST_ALLDRY, ST_GAUGE_FULL = 1, 2, 4, 8, 16, 32

_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile liboracle.so in place (plain gcc, FP64, no FMA contraction)."""
    if not force and os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in SRC):
        return LIB
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-o", LIB + ".tmp"] + SRC + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


class Config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("bc", ctypes.c_int * 4), ("model", ctypes.c_int),
                ("alpha", ctypes.c_double), ("h_star", ctypes.c_double),
                ("n_transition", ctypes.c_int), ("xi0", ctypes.c_double), ("xi1", ctypes.c_double),
                ("cfl", ctypes.c_double), ("g", ctypes.c_double), ("dry_tol", ctypes.c_double),
                ("limiter", ctypes.c_int), ("strang", ctypes.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            L.or_create.restype = ctypes.c_void_p
            L.or_create.argtypes = [ctypes.POINTER(Config), dp, ctypes.c_void_p]
            L.or_destroy.argtypes = [ctypes.c_void_p]
            L.or_nvar.argtypes = [ctypes.c_void_p]
            L.or_set_state.argtypes = [ctypes.c_void_p, dp, ctypes.c_double]
            L.or_get_state.argtypes = [ctypes.c_void_p, dp, dp]
            L.or_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.or_step_dt.argtypes = [ctypes.c_void_p, ctypes.c_double]
            L.or_dt_cfl.argtypes = [ctypes.c_void_p]
            L.or_dt_cfl.restype = ctypes.c_double
            L.or_mass.argtypes = [ctypes.c_void_p]
            L.or_mass.restype = ctypes.c_double
            L.or_status.argtypes = [ctypes.c_void_p]
            L.or_status.restype = ctypes.c_uint
            L.or_last_dt.argtypes = [ctypes.c_void_p]
            L.or_last_dt.restype = ctypes.c_double
            L.or_max_courant.argtypes = [ctypes.c_void_p]
            L.or_max_courant.restype = ctypes.c_double
            L.or_get_aux.argtypes = [ctypes.c_void_p, dp, ctypes.c_void_p]
            L.or_add_gauges.argtypes = [ctypes.c_void_p, dp, ctypes.c_int, ctypes.c_int]
            L.or_gauges.argtypes = [ctypes.c_void_p, dp, ctypes.c_size_t]
            L.or_eigvecs.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
            L.or_jacobian.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp]
            L.or_face.argtypes = [ctypes.POINTER(Config), dp, dp, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, dp, dp, dp, dp, dp, dp]
            L.or_source.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
            L.or_psi.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.or_psi.restype = ctypes.c_double
            L.or_set_c2.argtypes = [ctypes.c_void_p, dp]
            L.or_create_frame.restype = ctypes.c_void_p
            L.or_create_frame.argtypes = [ctypes.POINTER(Config), dp, ctypes.c_void_p]
            L.or_set_frame.argtypes = [ctypes.c_void_p, dp, ctypes.c_double]
            L.or_get_frame.argtypes = [ctypes.c_void_p, dp]
            L.or_step_begin.argtypes = [ctypes.c_void_p, ctypes.c_double]
            L.or_step_end.argtypes = [ctypes.c_void_p, ctypes.c_double]
            L.or_get_theta.argtypes = [ctypes.c_void_p, dp]
            L.or_set_theta.argtypes = [ctypes.c_void_p, dp]
            L.or_face_mass.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
            L.or_max_speed.argtypes = [ctypes.c_void_p]
            L.or_max_speed.restype = ctypes.c_double
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_config(nx, ny, dx, dy=None, x0=0.0, y0=0.0, bc=(WALL, WALL, WALL, WALL), model=HSGN,
                alpha=3.0, h_star=0.0, n_transition=1, xi0=0.01, xi1=0.05, cfl=0.9, g=9.81,
                dry_tol=1e-3, limiter=MC, strang=1):
    c = Config()
    c.nx, c.ny = nx, ny
    c.x0, c.y0 = x0, y0
    c.dx = dx
    c.dy = dx if dy is None else dy
    for i in range(4):
        c.bc[i] = bc[i]
    c.model = model
    c.alpha, c.h_star, c.n_transition = alpha, h_star, n_transition
    c.xi0, c.xi1, c.cfl, c.g, c.dry_tol = xi0, xi1, cfl, g, dry_tol
    c.limiter, c.strang = limiter, strang
    return c


class Oracle:
    """One oracle solver instance on an nx*ny grid (state arrays shaped (nvar, ny, nx))."""

    def __init__(self, b, phi_override=None, **cfg):
        b = np.ascontiguousarray(b, dtype=np.float64)
        ny, nx = b.shape
        self.cfg = make_config(nx, ny, **cfg)
        self.nx, self.ny = nx, ny
        self._b = b
        ph = None
        if phi_override is not None:
            self._phi = np.ascontiguousarray(phi_override, dtype=np.uint8)
            ph = self._phi.ctypes.data
        self.h = lib().or_create(ctypes.byref(self.cfg), _dp(b), ph)
        if not self.h:
            raise ValueError("or_create rejected the configuration")
        self.nvar = lib().or_nvar(self.h)

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_destroy(self.h)
            self.h = None

    def set_state(self, q, t=0.0):
        q = np.ascontiguousarray(q, dtype=np.float64)
        assert q.shape == (self.nvar, self.ny, self.nx)
        if lib().or_set_state(self.h, _dp(q), float(t)):
            raise ValueError("or_set_state failed")

    def get_state(self):
        q = np.empty((self.nvar, self.ny, self.nx))
        t = ctypes.c_double()
        lib().or_get_state(self.h, _dp(q), ctypes.byref(t))
        return q, t.value

    def step(self, n=1):
        return lib().or_step(self.h, int(n))

    def step_dt(self, dt):
        return lib().or_step_dt(self.h, float(dt))

    def dt_cfl(self):
        return lib().or_dt_cfl(self.h)

    def mass(self):
        return lib().or_mass(self.h)

    @property
    def status(self):
        return lib().or_status(self.h)

    @property
    def last_dt(self):
        return lib().or_last_dt(self.h)

    @property
    def max_courant(self):
        return lib().or_max_courant(self.h)

    def aux(self):
        c2 = np.empty((self.ny, self.nx))
        phi = np.empty((self.ny, self.nx), dtype=np.uint8)
        lib().or_get_aux(self.h, _dp(c2), phi.ctypes.data)
        return c2, phi

    def set_c2(self, c2):
        c2 = np.ascontiguousarray(c2, dtype=np.float64)
        assert c2.shape == (self.ny, self.nx)
        if lib().or_set_c2(self.h, _dp(c2)):
            raise ValueError("or_set_c2 rejected the field")

    def add_gauges(self, xy, capacity):
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        self._ng = xy.shape[0]
        if lib().or_add_gauges(self.h, _dp(xy), xy.shape[0], int(capacity)):
            raise ValueError("gauge outside the grid")

    def gauges(self):
        n = lib().or_gauges(self.h, None, 0)
        out = np.empty((max(n, 1), self._ng, 4))
        lib().or_gauges(self.h, _dp(out), out.size)
        return out[:n]



class Patch:
    """One patch of a refined level in patch mode: the caller owns the ghost
    frame.  Frame arrays are (ny+4, nx+4) per field (two ghost layers)."""

    NG = 2

    def __init__(self, b_frame, phi_frame, **cfg):
        b_frame = np.ascontiguousarray(b_frame, dtype=np.float64)
        self.nyp, self.nxp = b_frame.shape
        self.nx, self.ny = self.nxp - 2 * self.NG, self.nyp - 2 * self.NG
        self.cfg = make_config(self.nx, self.ny, **cfg)
        self._b = b_frame
        self._phi = np.ascontiguousarray(phi_frame, dtype=np.uint8)
        self.h = lib().or_create_frame(ctypes.byref(self.cfg), _dp(self._b), self._phi.ctypes.data)
        if not self.h:
            raise ValueError("or_create_frame rejected the configuration")
        self.nvar = lib().or_nvar(self.h)

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_destroy(self.h)
            self.h = None

    def set_frame(self, q, t=0.0):
        q = np.ascontiguousarray(q, dtype=np.float64)
        assert q.shape == (self.nvar, self.nyp, self.nxp)
        lib().or_set_frame(self.h, _dp(q), float(t))

    def get_frame(self):
        q = np.empty((self.nvar, self.nyp, self.nxp))
        lib().or_get_frame(self.h, _dp(q))
        return q

    def step_begin(self, dt):
        return lib().or_step_begin(self.h, float(dt))

    def step_end(self, dt):
        return lib().or_step_end(self.h, float(dt))

    def get_theta(self):
        th = np.empty((self.nyp, self.nxp))
        lib().or_get_theta(self.h, _dp(th))
        return th

    def set_theta(self, th):
        th = np.ascontiguousarray(th, dtype=np.float64)
        lib().or_set_theta(self.h, _dp(th))

    def face_mass(self, d):
        out = np.empty((self.ny, self.nx + 1) if d == 0 else (self.ny + 1, self.nx))
        lib().or_face_mass(self.h, d, _dp(out))
        return out

    def max_speed(self):
        return lib().or_max_speed(self.h)

    @property
    def status(self):
        return lib().or_status(self.h)


def eigvecs(model, roe, s1, sN, g=9.81):
    nv = NVAR[model]
    R = np.zeros((nv, nv))
    roe = np.ascontiguousarray(roe, dtype=np.float64)
    lib().or_eigvecs(model, _dp(roe), g, s1, sN, _dp(R))
    return R


def jacobian(model, st, g=9.81):
    nv = NVAR[model]
    J = np.zeros((nv, nv))
    st = np.ascontiguousarray(st, dtype=np.float64)
    lib().or_jacobian(model, _dp(st), g, _dp(J))
    return J


def face(cfg, qL, qR, bL, bR, c2L, c2R):
    """One x-direction normal Riemann solve; returns dict of waves, speeds, fluctuations."""
    nv = NVAR[cfg.model]
    Z = np.zeros((nv, nv)); s = np.zeros(nv); Am = np.zeros(nv); Ap = np.zeros(nv)
    d = np.zeros(nv); F = np.zeros(1)
    qL = np.ascontiguousarray(qL, dtype=np.float64); qR = np.ascontiguousarray(qR, dtype=np.float64)
    act = lib().or_face(ctypes.byref(cfg), _dp(qL), _dp(qR), bL, bR, c2L, c2R,
                        _dp(Z), _dp(s), _dp(Am), _dp(Ap), _dp(d), _dp(F))
    return dict(Z=Z, s=s, Am=Am, Ap=Ap, delta=d, Fhat=F[0], active=act)


def source(model, h, c2, tau, aux):
    y = np.array(aux, dtype=np.float64)
    lib().or_source(model, h, c2, tau, _dp(y))
    return y


def psi(bR, bL, xi0=0.01, xi1=0.05):
    return lib().or_psi(bR, bL, xi0, xi1)
