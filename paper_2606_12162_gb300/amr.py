"""Python binding of include/sgn_amr.h (the refined hierarchy): ctypes
marshalling only; every stage runs in the library's kernels."""
import ctypes

import numpy as np

from . import sgn

DP = ctypes.POINTER(ctypes.c_double)
AMR_SIGS = [
    ("sgn_amr_create", ctypes.c_int, [ctypes.POINTER(sgn.Grid), DP, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                      ctypes.POINTER(sgn.Params), ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    ("sgn_amr_destroy", None, [ctypes.c_void_p]),
    ("sgn_amr_npatches", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("sgn_amr_set_patch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, DP]),
    ("sgn_amr_get_patch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, DP]),
    ("sgn_amr_get_level_device", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    ("sgn_amr_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, DP]),
    ("sgn_amr_step_dt", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    ("sgn_amr_next_dt", ctypes.c_int, [ctypes.c_void_p, DP]),
    ("sgn_amr_mass", ctypes.c_int, [ctypes.c_void_p, DP, DP]),
    ("sgn_amr_status", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint)]),
    ("sgn_amr_info", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                                    ctypes.POINTER(ctypes.c_longlong)]),
    ("sgn_amr_launches_per_step", ctypes.c_int, [ctypes.c_void_p]),
    ("sgn_amr_regrid", ctypes.c_int, [ctypes.c_void_p, DP, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]),
    ("sgn_amr_regrid_flagged", ctypes.c_int, [ctypes.c_void_p, DP, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_int)]),
    ("sgn_amr_get_boxes", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.c_int]),
    ("sgn_amr_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), DP]),
    ("sgn_amr_set_tuning", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    ("sgn_amr_set_retake", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("sgn_amr_retakes", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)]),
]
_ready = False


def lib():
    global _ready
    L = sgn.load()
    if not _ready:
        for name, res, args in AMR_SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _ready = True
    return L


def _ck(rc, what):
    if rc != 0:
        raise sgn.SGNError(rc, what)


class Hierarchy:
    """Refined hierarchy on the GPU.  boxes: for levels 1..L-1, lists of
    (i0, j0, nx, ny) in that level's cells; b_finest: bathymetry of the finest
    level.  Patch states are (nvar, ny, nx) float64 arrays."""

    def __init__(self, b_finest, nx0, ny0, dx0, r, boxes, model=sgn.HSGN, bc=(sgn.WALL,) * 4,
                 precision=sgn.FP64, stream=None, torch_alloc=True, **params):
        L = lib()
        self.L = len(boxes) + 1
        self.r, self.model = r, model
        self.nvar = sgn.NVAR[model]
        b = np.ascontiguousarray(b_finest, dtype=np.float64)
        R = r ** (self.L - 1)
        if b.shape != (ny0 * R, nx0 * R):
            raise ValueError("b_finest must have shape %s" % ((ny0 * R, nx0 * R),))
        g = sgn.Grid()
        g.nx, g.ny, g.dx, g.dy = nx0, ny0, dx0, dx0
        for i in range(4):
            g.bc[i] = bc[i]
        self.params = sgn.default_params(precision=precision, **params)
        self._alloc = None
        aptr = None
        if torch_alloc:
            import torch
            self._alloc = sgn._TorchAllocator(torch.device("cuda", torch.cuda.current_device()))
            aptr = ctypes.byref(self._alloc.struct)
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
        self.boxes = [[(0, 0, nx0, ny0)]] + [[tuple(int(v) for v in bx) for bx in bl] for bl in boxes]
        nb = (ctypes.c_int * max(1, self.L - 1))(*[len(bl) for bl in boxes])
        flat = [int(v) for bl in boxes for bx in bl for v in bx]
        bx = (ctypes.c_int * max(1, len(flat)))(*flat)
        h = ctypes.c_void_p()
        _ck(L.sgn_amr_create(ctypes.byref(g), b.ctypes.data_as(DP), self.L, r, nb, bx, model,
                             ctypes.byref(self.params), aptr, ctypes.c_void_p(stream) if stream else None,
                             ctypes.byref(h)), "sgn_amr_create")
        self.h = h
        self.nx0, self.ny0 = nx0, ny0

    def regrid(self, b_finest, boxes):
        """New patches of levels 1..L-1 (same layout as at creation) with the
        state carried over; b_finest is the bathymetry given at creation."""
        if len(boxes) != self.L - 1:
            raise ValueError("need box lists for %d levels" % (self.L - 1))
        b = np.ascontiguousarray(b_finest, dtype=np.float64)
        R = self.r ** (self.L - 1)
        if b.shape != (self.ny0 * R, self.nx0 * R):
            raise ValueError("b_finest must have shape %s" % ((self.ny0 * R, self.nx0 * R),))
        nb = (ctypes.c_int * max(1, self.L - 1))(*[len(bl) for bl in boxes])
        flat = [int(v) for bl in boxes for bx in bl for v in bx]
        bx = (ctypes.c_int * max(1, len(flat)))(*flat)
        _ck(lib().sgn_amr_regrid(self.h, b.ctypes.data_as(DP), nb, bx), "sgn_amr_regrid")
        self.boxes = [self.boxes[0]] + [[tuple(int(v) for v in x) for x in bl] for bl in boxes]

    def regrid_flagged(self, b_finest, tol, tile=8, buffer=2):
        """Flag-driven regridding (surface jump above tol); returns the number
        of boxes per level >= 1."""
        b = np.ascontiguousarray(b_finest, dtype=np.float64)
        nb = (ctypes.c_int * max(1, self.L - 1))()
        _ck(lib().sgn_amr_regrid_flagged(self.h, b.ctypes.data_as(DP), float(tol), int(tile), int(buffer), nb),
            "sgn_amr_regrid_flagged")
        self.boxes = [self.boxes[0]] + [self.get_boxes(l) for l in range(1, self.L)]
        return list(nb)[:self.L - 1]

    def get_boxes(self, level):
        n = lib().sgn_amr_get_boxes(self.h, int(level), None, 0)
        if n < 0:
            raise sgn.SGNError(n, "sgn_amr_get_boxes")
        out = (ctypes.c_int * max(1, 4 * n))()
        _ck(0 if lib().sgn_amr_get_boxes(self.h, int(level), out, n) == n else -1, "sgn_amr_get_boxes")
        return [tuple(out[4 * k:4 * k + 4]) for k in range(n)]

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().sgn_amr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def npatches(self, level):
        return lib().sgn_amr_npatches(self.h, level)

    def set_patch(self, level, k, q):
        i0, j0, nx, ny = self.boxes[level][k]
        q = np.ascontiguousarray(q, dtype=np.float64)
        if q.shape != (self.nvar, ny, nx):
            raise ValueError("patch state must have shape %s" % ((self.nvar, ny, nx),))
        _ck(lib().sgn_amr_set_patch(self.h, level, k, q.ctypes.data_as(DP)), "sgn_amr_set_patch")

    def get_patch(self, level, k):
        i0, j0, nx, ny = self.boxes[level][k]
        out = np.empty((self.nvar, ny, nx))
        _ck(lib().sgn_amr_get_patch(self.h, level, k, out.ctypes.data_as(DP)), "sgn_amr_get_patch")
        return out

    def get_level_device(self, level, out):
        """Every patch of `level` into the first fields of `out`, a contiguous
        FP64 CUDA tensor of shape (nfields, NY_l, NX_l); cells without a patch
        keep their values."""
        import torch
        R = self.r ** level
        if (out.dtype != torch.float64 or not out.is_cuda or not out.is_contiguous() or out.dim() != 3
                or tuple(out.shape[1:]) != (self.ny0 * R, self.nx0 * R)):
            raise ValueError("out must be a contiguous float64 CUDA tensor (nfields, %d, %d)"
                             % (self.ny0 * R, self.nx0 * R))
        _ck(lib().sgn_amr_get_level_device(self.h, level, int(out.shape[0]), ctypes.c_void_p(out.data_ptr())),
            "sgn_amr_get_level_device")
        return out

    def set_state(self, qs):
        """qs[l]: dense (nvar, NY_l, NX_l) state of level l; each patch takes its box."""
        for l, bl in enumerate(self.boxes):
            for k, (i0, j0, nx, ny) in enumerate(bl):
                self.set_patch(l, k, qs[l][:, j0:j0 + ny, i0:i0 + nx])

    def step(self, n=1):
        t = ctypes.c_double()
        _ck(lib().sgn_amr_step(self.h, int(n), ctypes.byref(t)), "sgn_amr_step")
        return t.value

    def step_rc(self, n=1):
        t = ctypes.c_double()
        return lib().sgn_amr_step(self.h, int(n), ctypes.byref(t))

    def step_dt(self, dt0):
        _ck(lib().sgn_amr_step_dt(self.h, float(dt0)), "sgn_amr_step_dt")

    def next_dt(self):
        d = ctypes.c_double()
        _ck(lib().sgn_amr_next_dt(self.h, ctypes.byref(d)), "sgn_amr_next_dt")
        return d.value

    def mass(self):
        """(mass over the uncovered cells of all levels, water added by clipped reflux)."""
        m, c = ctypes.c_double(), ctypes.c_double()
        _ck(lib().sgn_amr_mass(self.h, ctypes.byref(m), ctypes.byref(c)), "sgn_amr_mass")
        return m.value, c.value

    def status(self):
        f = ctypes.c_uint()
        _ck(lib().sgn_amr_status(self.h, ctypes.byref(f)), "sgn_amr_status")
        return f.value

    def info(self):
        """Per level: interior cells of all patches, cells of the level's atlas."""
        c = (ctypes.c_longlong * self.L)()
        a = (ctypes.c_longlong * self.L)()
        _ck(lib().sgn_amr_info(self.h, c, a), "sgn_amr_info")
        return list(c), list(a)

    def launches_per_step(self):
        return lib().sgn_amr_launches_per_step(self.h)

    def set_retake(self, max_retakes):
        """Retake level-0 steps that break the CFL limit (0: off)."""
        _ck(lib().sgn_amr_set_retake(self.h, int(max_retakes)), "sgn_amr_set_retake")

    def retakes(self):
        n = ctypes.c_longlong()
        _ck(lib().sgn_amr_retakes(self.h, ctypes.byref(n)), "sgn_amr_retakes")
        return n.value

    def autotune(self, reps=20):
        """Tune every level's launch shapes and schedule (state unchanged).
        Returns (choice per level, ms table per level)."""
        n = self.L * sgn.TUNE_N
        ch = (ctypes.c_int * n)()
        ms = (ctypes.c_double * (n * sgn.TUNE_OPTS))()
        _ck(lib().sgn_amr_autotune(self.h, int(reps), ch, ms), "sgn_amr_autotune")
        return (np.array(ch[:]).reshape(self.L, sgn.TUNE_N),
                np.array(ms[:]).reshape(self.L, sgn.TUNE_N, sgn.TUNE_OPTS))

    def set_tuning(self, choice):
        """choice: L x TUNE_N option indices (one tuning per level)."""
        c = np.asarray(choice, dtype=np.int64).reshape(-1)
        ch = (ctypes.c_int * len(c))(*[int(v) for v in c])
        if len(c) != self.L * sgn.TUNE_N:
            raise ValueError("need %d options" % (self.L * sgn.TUNE_N))
        _ck(lib().sgn_amr_set_tuning(self.h, ch), "sgn_amr_set_tuning")
