"""C ABI checks that need no GPU: the library builds, loads, exports every entry
point declared in include/sgn.h (and nothing else), and rejects invalid
arguments on the host before touching the device."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sgn.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2606_12162_gb300 import build, sgn
    build.build()
    return sgn, sgn.load()


def header_functions(prefix="sgn_", header=HEADER):
    src = open(header).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(%s[a-z0-9_]+)\s*\(" % prefix, src)))


def test_header_declares_the_abi():
    fns = header_functions()
    for required in ("sgn_create", "sgn_set_state", "sgn_step", "sgn_get_state", "sgn_gauges", "sgn_destroy"):
        assert required in fns


def test_library_exports_exactly_the_headers(lib):
    from paper_2606_12162_gb300 import corrector, sgn
    out = subprocess.run(["nm", "-D", "--defined-only", sgn.LIB_PATH], capture_output=True, text=True).stdout
    exported = sorted(set(re.findall(r"\bT ([a-z]+_[a-z0-9_]+)$", out, flags=re.M)))
    from paper_2606_12162_gb300 import amr
    declared = header_functions("sgn_") + header_functions("sgn_", os.path.join(ROOT, "include", "sgn_amr.h")) + \
        header_functions("lc_", os.path.join(ROOT, "include", "lc.h"))
    assert exported == sorted(declared)
    # every declared entry point resolves through ctypes and has a binding signature
    names = {n for n, _, _ in sgn.SIGNATURES} | {n for n, _, _ in corrector.LC_SIGS} | \
        {n for n, _, _ in amr.AMR_SIGS}
    for fn in declared:
        getattr(lib[1], fn)
        assert fn in names


def test_defaults_and_enums(lib):
    S, L = lib
    p = S.default_params()
    assert p.alpha == 3.0 and p.xi0 == 0.01 and p.xi1 == 0.05 and p.cfl == 0.9
    assert p.g == 9.81 and p.n_transition == 1 and p.limiter == S.MC and p.strang == 1
    assert [L.sgn_nvar(m) for m in (0, 1, 2)] == [3, 5, 7]
    assert L.sgn_nvar(9) == -1
    for code in range(0, -10, -1):
        assert L.sgn_strerror(code)


def _grid(S, nx=8, ny=8, dx=1.0, bc=(0, 0, 0, 0)):
    g = S.Grid()
    g.nx, g.ny, g.dx, g.dy = nx, ny, dx, dx
    for i in range(4):
        g.bc[i] = bc[i]
    return g


@pytest.mark.parametrize("bad", ["null_out", "null_b", "small", "dx", "bc", "periodic_pair", "model",
                                 "cfl", "ntrans", "precision", "limiter"])
def test_create_rejects_invalid_arguments(lib, bad):
    S, L = lib
    b = np.full((8, 8), -1.0)
    g = _grid(S)
    p = S.default_params()
    model = 2
    out = ctypes.c_void_p()
    outp = ctypes.byref(out)
    bp = b.ctypes.data_as(S.DP)
    if bad == "null_out":
        outp = None
    elif bad == "null_b":
        bp = None
    elif bad == "small":
        g.nx = 1
    elif bad == "dx":
        g.dx = 0.0
    elif bad == "bc":
        g.bc[2] = 7
    elif bad == "periodic_pair":
        g.bc[0] = 2
    elif bad == "model":
        model = 5
    elif bad == "cfl":
        p.cfl = 1.5
    elif bad == "ntrans":
        p.n_transition = 3
    elif bad == "precision":
        p.precision = 4
    elif bad == "limiter":
        p.limiter = 9
    rc = L.sgn_create(ctypes.byref(g), bp, model, ctypes.byref(p), None, None, None, outp)
    assert rc == -1


def test_null_handles_are_rejected(lib):
    S, L = lib
    x = np.zeros(4)
    assert L.sgn_step(None, 1, None) == -1
    assert L.sgn_set_state(None, x.ctypes.data_as(S.DP), 0.0) == -1
    assert L.sgn_get_state(None, 0, x.ctypes.data_as(S.DP), 4, None) == -1
    assert L.sgn_mass(None, x.ctypes.data_as(S.DP)) == -1
    assert L.sgn_status(None, None, None, None) == -1
    assert L.sgn_next_dt(None, x.ctypes.data_as(S.DP)) == -1
    assert L.sgn_well_prepare(None) == -1
    assert L.sgn_set_c2(None, x.ctypes.data_as(S.DP)) == -1
    L.sgn_destroy(None)


def test_create_without_gpu_reports_an_error_code(lib):
    """With no CUDA device the library returns SGN_ECUDA instead of crashing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    S, L = lib
    b = np.full((8, 8), -1.0)
    out = ctypes.c_void_p()
    rc = L.sgn_create(ctypes.byref(_grid(S)), b.ctypes.data_as(S.DP), 2, ctypes.byref(S.default_params()),
                      None, None, None, ctypes.byref(out))
    assert rc == -3 and not out.value


def test_amr_create_rejects_invalid_arguments(lib):
    """Refined hierarchy: argument checks on the host, before any device call."""
    S, L = lib
    from paper_2606_12162_gb300 import amr
    amr.lib()
    b = np.full((16, 16), -1.0)
    nb = (ctypes.c_int * 1)(1)
    bx = (ctypes.c_int * 4)(4, 4, 8, 8)
    out = ctypes.c_void_p()
    p = S.default_params()
    dp = b.ctypes.data_as(S.DP)

    def create(g, nlev=2, ratio=2, bb=dp, nbx=nb, box=bx, outp=ctypes.byref(out)):
        return L.sgn_amr_create(ctypes.byref(g), bb, nlev, ratio, nbx, box, 2, ctypes.byref(p), None, None, outp)

    assert create(_grid(S), outp=None) == -1
    assert create(_grid(S), nlev=0) == -1
    assert create(_grid(S), nlev=9) == -1
    assert create(_grid(S), ratio=1) == -1
    assert create(_grid(S), bb=None) == -1
    assert create(_grid(S), nbx=None) == -1
    assert create(_grid(S, bc=(2, 2, 0, 0))) == -1          # periodic
    g = _grid(S)
    g.dy = 2.0                                                 # dx != dy
    assert create(g) == -1
    assert L.sgn_amr_step(None, 1, None) == -1
    assert L.sgn_amr_npatches(None, 0) == -1
    L.sgn_amr_destroy(None)
    import torch
    if not torch.cuda.is_available():
        assert create(_grid(S)) == -3 and not out.value
