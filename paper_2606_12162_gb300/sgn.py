"""ctypes binding of the C ABI in include/sgn.h (libsgn_gb300.so).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  PyTorch supplies device memory (through the allocator callback) and
the CUDA stream.  If the library has not been built this module raises; there is
no CPU fallback.
"""
import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libsgn_gb300.so")

SWE, MBHSGN, HSGN = 0, 1, 2
WALL, EXTRAP, PERIODIC = 0, 1, 2
FP64, MIXED = 0, 1
MINMOD, MC, NOLIMIT = 0, 1, 2
NVAR = {SWE: 3, MBHSGN: 5, HSGN: 7}

E_CODES = {0: "SGN_OK", -1: "SGN_EINVAL", -2: "SGN_ENOMEM", -3: "SGN_ECUDA", -4: "SGN_ENEGDEPTH",
           -5: "SGN_ENONFINITE", -6: "SGN_ECFL", -7: "SGN_ENONHYP", -8: "SGN_EALLDRY", -9: "SGN_ERANGE"}
ST_NEGDEPTH, ST_NONFINITE, ST_CFL, ST_NONHYP, ST_ALLDRY, ST_GAUGEFULL = 1, 2, 4, 8, 16, 32


class SGNError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s: %s (%s)" % (what, E_CODES.get(code, code), _strerror(code)))


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("x0", ctypes.c_double),
                ("y0", ctypes.c_double), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("bc", ctypes.c_int * 4)]


class Params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("h_star", ctypes.c_double), ("n_transition", ctypes.c_int),
                ("xi0", ctypes.c_double), ("xi1", ctypes.c_double), ("cfl", ctypes.c_double),
                ("g", ctypes.c_double), ("dry_tol", ctypes.c_double), ("limiter", ctypes.c_int),
                ("strang", ctypes.c_int), ("precision", ctypes.c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()
DP = ctypes.POINTER(ctypes.c_double)

# (name, restype, argtypes) of every entry point declared in include/sgn.h
SIGNATURES = [
    ("sgn_default_params", None, [ctypes.POINTER(Params)]),
    ("sgn_nvar", ctypes.c_int, [ctypes.c_int]),
    ("sgn_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("sgn_create", ctypes.c_int, [ctypes.POINTER(Grid), DP, ctypes.c_int, ctypes.POINTER(Params),
                                  ctypes.c_void_p, ctypes.POINTER(Allocator), ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_void_p)]),
    ("sgn_set_state", ctypes.c_int, [ctypes.c_void_p, DP, ctypes.c_double]),
    ("sgn_set_state_device", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double]),
    ("sgn_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, DP]),
    ("sgn_step_dt", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    ("sgn_get_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, DP, ctypes.c_size_t, DP]),
    ("sgn_get_state_device", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    ("sgn_add_gauges", ctypes.c_int, [ctypes.c_void_p, DP, ctypes.c_int, ctypes.c_int]),
    ("sgn_gauges", ctypes.c_int, [ctypes.c_void_p, DP, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int)]),
    ("sgn_clear_gauges", ctypes.c_int, [ctypes.c_void_p]),
    ("sgn_status", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint), DP, DP]),
    ("sgn_next_dt", ctypes.c_int, [ctypes.c_void_p, DP]),
    ("sgn_mass", ctypes.c_int, [ctypes.c_void_p, DP]),
    ("sgn_get_aux", ctypes.c_int, [ctypes.c_void_p, DP, ctypes.c_void_p]),
    ("sgn_well_prepare", ctypes.c_int, [ctypes.c_void_p]),
    ("sgn_set_c2", ctypes.c_int, [ctypes.c_void_p, DP]),
    ("sgn_set_profiling", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("sgn_kernel_times", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_char_p), DP,
                                        ctypes.POINTER(ctypes.c_long), ctypes.c_int]),
    ("sgn_launches_per_step", ctypes.c_int, [ctypes.c_void_p]),
    ("sgn_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), DP]),
    ("sgn_set_tuning", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    ("sgn_get_tuning", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    ("sgn_destroy", None, [ctypes.c_void_p]),
    ("sgn_math_check", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("sgn_math_check_f32", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("sgn_mass_static", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]),
]
MASS_SCRATCH_MAX = 65536
TUNE_N, TUNE_OPTS = 8, 3
TUNE_SLOTS = ("prep", "face_x", "face_y", "trans_x", "trans_y", "theta", "update", "schedule")


def mass_static(eta, b, dx, dy, out, stream=None):
    """Allocation-free mass of eta/b (CUDA float64 tensors, (ny, nx)) into out (a
    CUDA float64 tensor with one element); returns the C ABI's error code."""
    ny, nx = eta.shape[-2], eta.shape[-1]
    return load().sgn_mass_static(ctypes.c_void_p(eta.data_ptr()), ctypes.c_void_p(b.data_ptr()), nx, ny,
                                  float(dx), float(dy), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(stream) if stream else None)


def load():
    """Load libsgn_gb300.so; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libsgn_gb300.so is missing: build it with "
                                   "paper_2606_12162_gb300.build.build() (nvcc, sm_103a)")
            L = ctypes.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _strerror(code):
    try:
        return load().sgn_strerror(code).decode()
    except Exception:
        return "?"


def _ck(code, what):
    if code != 0:
        raise SGNError(code, what)


def _dp(a):
    return a.ctypes.data_as(DP)


def default_params(**kw):
    p = Params()
    load().sgn_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError("unknown parameter %s" % k)
        setattr(p, k, v)
    return p


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator, kept alive until freed."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.live = {}
        # allocations still granted (None: no limit) -- lets a test make the
        # library run out of device memory at a chosen point
        self.allow = None
        self.c_alloc = ALLOC_FN(self._alloc)
        self.c_free = FREE_FN(self._free)
        self.struct = Allocator(self.c_alloc, self.c_free, None)

    def _alloc(self, nbytes, ctx):
        if self.allow is not None:
            if self.allow <= 0:
                return None
            self.allow -= 1
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:
            return None
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, ptr, ctx):
        self.live.pop(ptr, None)


class Solver:
    """One solver handle.  b: (ny, nx) bathymetry; states are (nvar, ny, nx) float64."""

    def __init__(self, b, model=HSGN, dx=1.0, dy=None, x0=0.0, y0=0.0, bc=(WALL,) * 4,
                 precision=FP64, phi_override=None, stream=None, torch_alloc=True, **params):
        L = load()
        b = np.ascontiguousarray(b, dtype=np.float64)
        ny, nx = b.shape
        self.nx, self.ny, self.model = nx, ny, model
        self.nvar = NVAR[model]
        g = Grid()
        g.nx, g.ny, g.x0, g.y0, g.dx = nx, ny, x0, y0, dx
        g.dy = dx if dy is None else dy
        for i in range(4):
            g.bc[i] = bc[i]
        self.params = default_params(precision=precision, **params)
        self._alloc = None
        aptr = None
        if torch_alloc:
            import torch
            self._alloc = _TorchAllocator(torch.device("cuda", torch.cuda.current_device()))
            aptr = ctypes.byref(self._alloc.struct)
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        ph = None
        if phi_override is not None:
            self._phi = np.ascontiguousarray(phi_override, dtype=np.uint8)
            ph = self._phi.ctypes.data
        h = ctypes.c_void_p()
        _ck(L.sgn_create(ctypes.byref(g), _dp(b), model, ctypes.byref(self.params), ph, aptr,
                         ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)), "sgn_create")
        self.h = h
        self._ng = 0

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().sgn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, q, t=0.0):
        q = np.ascontiguousarray(q, dtype=np.float64)
        if q.shape != (self.nvar, self.ny, self.nx):
            raise ValueError("state must have shape %s" % ((self.nvar, self.ny, self.nx),))
        _ck(load().sgn_set_state(self.h, _dp(q), float(t)), "sgn_set_state")

    def set_state_ptr(self, ptr, t=0.0):
        """q in host memory given by address (e.g. a pinned torch tensor)."""
        _ck(load().sgn_set_state(self.h, ctypes.cast(ptr, DP), float(t)), "sgn_set_state")

    def set_state_device(self, tensor, t=0.0):
        assert tensor.is_cuda and tensor.dtype.is_floating_point and tensor.element_size() == 8
        assert tensor.numel() == self.nvar * self.nx * self.ny and tensor.is_contiguous()
        _ck(load().sgn_set_state_device(self.h, ctypes.c_void_p(tensor.data_ptr()), float(t)),
            "sgn_set_state_device")

    def step(self, n=1):
        t = ctypes.c_double()
        _ck(load().sgn_step(self.h, int(n), ctypes.byref(t)), "sgn_step")
        return t.value

    def step_rc(self, n=1):
        """As step() but returns the error code instead of raising."""
        t = ctypes.c_double()
        return load().sgn_step(self.h, int(n), ctypes.byref(t))

    def step_dt(self, dt):
        _ck(load().sgn_step_dt(self.h, float(dt)), "sgn_step_dt")

    def get_state(self, field_mask=0):
        nsel = self.nvar if field_mask == 0 else bin(field_mask).count("1")
        out = np.empty((nsel, self.ny, self.nx))
        t = ctypes.c_double()
        _ck(load().sgn_get_state(self.h, int(field_mask), _dp(out), out.size, ctypes.byref(t)), "sgn_get_state")
        return out, t.value

    def get_state_ptr(self, ptr, n):
        _ck(load().sgn_get_state(self.h, 0, ctypes.cast(ptr, DP), int(n), None), "sgn_get_state")

    def get_state_device(self, tensor):
        _ck(load().sgn_get_state_device(self.h, ctypes.c_void_p(tensor.data_ptr()), tensor.numel()),
            "sgn_get_state_device")

    def add_gauges(self, xy, capacity):
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
        _ck(load().sgn_add_gauges(self.h, _dp(xy), xy.shape[0], int(capacity)), "sgn_add_gauges")
        self._ng = xy.shape[0]

    def gauges(self):
        n = ctypes.c_int()
        _ck(load().sgn_gauges(self.h, None, 0, ctypes.byref(n)), "sgn_gauges")
        out = np.empty((n.value, self._ng, 4))
        if n.value:
            _ck(load().sgn_gauges(self.h, _dp(out), out.size, ctypes.byref(n)), "sgn_gauges")
        return out

    def clear_gauges(self):
        _ck(load().sgn_clear_gauges(self.h), "sgn_clear_gauges")

    def status(self):
        f = ctypes.c_uint()
        dt = ctypes.c_double()
        cr = ctypes.c_double()
        _ck(load().sgn_status(self.h, ctypes.byref(f), ctypes.byref(dt), ctypes.byref(cr)), "sgn_status")
        return f.value, dt.value, cr.value

    def next_dt(self):
        """The CFL time step the next step() will take."""
        dt = ctypes.c_double()
        _ck(load().sgn_next_dt(self.h, ctypes.byref(dt)), "sgn_next_dt")
        return dt.value

    def mass(self):
        m = ctypes.c_double()
        _ck(load().sgn_mass(self.h, ctypes.byref(m)), "sgn_mass")
        return m.value

    def aux(self):
        c2 = np.empty((self.ny, self.nx))
        phi = np.empty((self.ny, self.nx), dtype=np.uint8)
        _ck(load().sgn_get_aux(self.h, _dp(c2), phi.ctypes.data), "sgn_get_aux")
        return c2, phi

    def set_c2(self, c2):
        """Replace c^2 of every cell (ny, nx); call before set_state."""
        c2 = np.ascontiguousarray(c2, dtype=np.float64)
        if c2.shape != (self.ny, self.nx):
            raise ValueError("c2 must have shape %s" % ((self.ny, self.nx),))
        _ck(load().sgn_set_c2(self.h, _dp(c2)), "sgn_set_c2")

    def well_prepare(self):
        """Replace hw and hp by the well-prepared values of Sec. 3.2 (mbHSGN)."""
        _ck(load().sgn_well_prepare(self.h), "sgn_well_prepare")

    def set_profiling(self, on):
        _ck(load().sgn_set_profiling(self.h, int(bool(on))), "sgn_set_profiling")

    def kernel_times(self):
        n = 16
        names = (ctypes.c_char_p * n)()
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_long * n)()
        k = load().sgn_kernel_times(self.h, names, ms, cnt, n)
        return {names[i].decode(): (ms[i], cnt[i]) for i in range(min(k, n)) if names[i]}

    def launches_per_step(self):
        return load().sgn_launches_per_step(self.h)

    def autotune(self, reps=20):
        """Time the launch-shape options of each step kernel and the two
        schedules on the current state, keep the fastest (state unchanged).
        Returns (choice list, ms table TUNE_N x TUNE_OPTS)."""
        ch = (ctypes.c_int * TUNE_N)()
        ms = (ctypes.c_double * (TUNE_N * TUNE_OPTS))()
        _ck(load().sgn_autotune(self.h, int(reps), ch, ms), "sgn_autotune")
        return list(ch), np.array(ms[:]).reshape(TUNE_N, TUNE_OPTS)

    def set_tuning(self, choice):
        ch = (ctypes.c_int * TUNE_N)(*[int(c) for c in choice])
        _ck(load().sgn_set_tuning(self.h, ch), "sgn_set_tuning")

    def tuning(self):
        """Current tuning: {slot: (option, (bx, by))}; the schedule slot has (0, 0)."""
        ch, bx, by = (ctypes.c_int * TUNE_N)(), (ctypes.c_int * TUNE_N)(), (ctypes.c_int * TUNE_N)()
        _ck(load().sgn_get_tuning(self.h, ch, bx, by), "sgn_get_tuning")
        return {TUNE_SLOTS[k]: (ch[k], (bx[k], by[k])) for k in range(TUNE_N)}
