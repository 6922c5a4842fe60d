"""Learned coarse-to-fine corrector: binding of include/lc.h, training-pair
generation with the solver itself, training, inference and fallback.

The corrector stands in for the finest refinement level of the paper's AMR: from
a coarse state (eta, hu, hv, b, phi_T) it predicts the fine-grid (ratio r)
correction of eta, hu, hv relative to the piecewise-constant prolongation.
Training pairs come from coarse and fine runs of this library's solver on the
same seeded scenario (fractal bathymetry, Gaussian sources).  Forward, backward,
loss and Adam are the library's CUDA kernels; PyTorch only holds device buffers.
"""
import ctypes
import math
import time

import numpy as np

from . import sgn, workloads as W

DP = ctypes.c_void_p
LC_SIGS = [
    ("lc_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_long,
                                 ctypes.c_ulonglong, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("lc_destroy", None, [ctypes.c_void_p]),
    ("lc_num_params", ctypes.c_long, [ctypes.c_void_p]),
    ("lc_get_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long]),
    ("lc_set_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long]),
    ("lc_forward", ctypes.c_int, [ctypes.c_void_p, DP, ctypes.c_int, ctypes.c_int, DP]),
    ("lc_train_step", ctypes.c_int, [ctypes.c_void_p, DP, DP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.c_float,
                                     ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    ("lc_make_input", ctypes.c_int, [DP, DP, DP, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, DP, ctypes.c_void_p]),
    ("lc_make_target", ctypes.c_int, [DP, DP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                      ctypes.c_float, DP, ctypes.c_void_p]),
    ("lc_apply", ctypes.c_int, [DP, DP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                ctypes.c_int, DP, ctypes.c_void_p]),
    ("lc_restrict", ctypes.c_int, [DP, ctypes.c_int, ctypes.c_int, ctypes.c_int, DP, ctypes.c_void_p]),
]
_ready = False

# scales of the normalised inputs and outputs: surface [m], momentum [m^2/s], bathymetry [m]
S_ETA, S_Q, S_B = 1.0, 100.0, 1000.0


def lib():
    global _ready
    L = sgn.load()
    if not _ready:
        for name, res, args in LC_SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _ready = True
    return L


def _ck(rc, what):
    if rc != 0:
        raise RuntimeError("%s failed (%d)" % (what, rc))


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream or None


class Net:
    """The corrector network (depth 3x3 conv layers, BF16 weights, FP32 accumulation)."""

    def __init__(self, cin=5, width=32, depth=5, r=4, nout=3, max_hw=256 * 256, seed=5000):
        self.cin, self.width, self.depth, self.r, self.nout = cin, width, depth, r, nout
        self.cout = nout * r * r
        self.max_hw = max_hw
        h = ctypes.c_void_p()
        _ck(lib().lc_create(cin, width, depth, self.cout, max_hw, seed, _stream(), ctypes.byref(h)), "lc_create")
        self.h = h
        self.n = lib().lc_num_params(h)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().lc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layers(self):
        return [(self.cin if l == 0 else self.width, self.cout if l == self.depth - 1 else self.width)
                for l in range(self.depth)]

    def params(self):
        out = np.empty(self.n, dtype=np.float32)
        _ck(lib().lc_get_params(self.h, out.ctypes.data, self.n), "lc_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _ck(lib().lc_set_params(self.h, p.ctypes.data, self.n), "lc_set_params")

    def forward(self, x):
        import torch
        _, H, Wd = x.shape
        y = torch.empty((self.cout, H, Wd), dtype=torch.float32, device=x.device)
        _ck(lib().lc_forward(self.h, _p(x), H, Wd, _p(y)), "lc_forward")
        return y

    def train_step(self, x, t, lr, fw=(1.0, 1.0, 1.0), want_grad=False):
        _, H, Wd = x.shape
        fwa = (ctypes.c_float * self.nout)(*fw)
        loss = ctypes.c_double()
        g = np.empty(self.n, dtype=np.float32) if want_grad else None
        _ck(lib().lc_train_step(self.h, _p(x), _p(t), H, Wd, self.r, self.nout, fwa, float(lr), ctypes.byref(loss),
                                g.ctypes.data if want_grad else None), "lc_train_step")
        return (loss.value, g) if want_grad else loss.value


# ----------------------------------------------------------------------------
def scenario_bathymetry(nc, r, seed=5001, depth=6000.0, smooth_cells=2.0):
    """Fine fractal bathymetry (seed 5001, |k|^-2 spectrum) low-pass filtered with a
    Gaussian of smooth_cells coarse cells, so that the coarse grid resolves the
    bathymetry (the raw field has grid-scale cliffs of ~1 km at 2 km spacing), and
    its r x r block-mean restriction."""
    from scipy.ndimage import gaussian_filter
    raw = W.fractal_bathymetry(nc * r, seed, depth=depth, land_frac=0.15)
    bf = gaussian_filter(raw, smooth_cells * r, mode="nearest")
    bf = np.minimum(bf, 500.0)
    bc = bf.reshape(nc, r, nc, r).mean(axis=(1, 3))
    return bf, bc


def source_state(model, b, dx, cx, cy, amp, rad):
    n = b.shape[0]
    x, y = W.cell_centres(n, n, dx, dx)
    q = np.zeros((W.NVAR[model], n, n))
    q[0] = W.apply_surface(b, amp * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / rad ** 2))
    return q


def generate_pairs(nc=512, r=4, dxc=2000.0, scenarios=range(40), times=(60.0, 120.0, 180.0, 240.0, 300.0),
                   model=W.HSGN, precision=sgn.MIXED, seed=5001):
    """Coarse/fine solver pairs: for each scenario (source seed 5002 + s: amplitude
    U[0.5, 5] m, radius U[10, 50] km, centre over water deeper than 1000 m) run the
    coarse (nc^2, dxc) and fine ((r nc)^2, dxc/r) solvers to each snapshot time and
    keep (input, target, coarse state, fine state) on the device."""
    import torch
    bf, bc = scenario_bathymetry(nc, r, seed)
    nf = nc * r
    dxf = dxc / r
    cfg = dict(model=model, bc=(1, 1, 1, 1), h_star=20.0, alpha=3.0, precision=precision)
    sc = sgn.Solver(bc, dx=dxc, **cfg)
    sf = sgn.Solver(bf, dx=dxf, **cfg)
    _, phic = sc.aux()
    bcd = torch.from_numpy(np.ascontiguousarray(bc)).cuda()
    phid = torch.from_numpy(np.ascontiguousarray(phic)).cuda()
    nv = W.NVAR[model]
    qc = torch.empty((nv, nc, nc), dtype=torch.float64, device="cuda")
    qf = torch.empty((nv, nf, nf), dtype=torch.float64, device="cuda")
    pairs = []
    L = lib()
    st = _stream()
    for s in scenarios:
        rng = np.random.default_rng(5002 + s)
        deep = np.argwhere(bc < -1000.0)
        j, i = deep[rng.integers(len(deep))]
        cx, cy = (i + 0.5) * dxc, (j + 0.5) * dxc
        amp, rad = rng.uniform(0.5, 5.0), rng.uniform(10e3, 50e3)
        qf0 = source_state(model, bf, dxf, cx, cy, amp, rad)
        qc0 = np.zeros((nv, nc, nc))
        qc0[0] = qf0[0].reshape(nc, r, nc, r).mean(axis=(1, 3))
        sf.set_state(qf0)
        sc.set_state(qc0)
        tnow = {id(sc): 0.0, id(sf): 0.0}
        for T in times:
            for sv in (sc, sf):
                tnow[id(sv)] = advance_to(sv, tnow[id(sv)], T)
            sc.get_state_device(qc)
            sf.get_state_device(qf)
            x = torch.empty((5, nc, nc), dtype=torch.float32, device="cuda")
            tg = torch.empty((3, nf, nf), dtype=torch.float32, device="cuda")
            _ck(L.lc_make_input(_p(qc), _p(bcd), _p(phid), nc, nc, S_ETA, S_Q, S_B, _p(x), st), "lc_make_input")
            _ck(L.lc_make_target(_p(qf), _p(qc), nc, nc, r, S_ETA, S_Q, _p(tg), st), "lc_make_target")
            pairs.append(dict(x=x, t=tg, qc=qc[:3].clone(), qf=qf[:3].clone(), scenario=s, time=T))
    return pairs, dict(bc=bc, bf=bf, dxc=dxc, r=r)


def advance_to(sv, t, T):
    """Step a solver from time t to exactly T: CFL steps while more than two
    steps remain, then equal fixed steps of at most 0.9 x the last CFL step."""
    while T - t > 1e-9:
        dtl = sv.status()[1]
        if dtl <= 0.0 or T - t > 2.0 * dtl:
            t = sv.step(1)
            continue
        k = int(math.ceil((T - t) / (0.9 * dtl)))
        h = (T - t) / k
        for _ in range(k):
            sv.step_dt(h)
        t = T
    return t


def train(net, pairs, iters=2000, crop=64, lr=1e-3, seed=0, fw=(1.0, 1.0, 1.0), log=None):
    """Adam on random crops of the training pairs (crop x crop coarse cells)."""
    import torch
    rng = np.random.default_rng(seed)
    r = net.r
    losses = []
    t0 = time.perf_counter()
    for it in range(iters):
        p = pairs[int(rng.integers(len(pairs)))]
        nc = p["x"].shape[-1]
        c = min(crop, nc)
        j, i = int(rng.integers(0, nc - c + 1)), int(rng.integers(0, nc - c + 1))
        x = p["x"][:, j:j + c, i:i + c].contiguous()
        t = p["t"][:, j * r:(j + c) * r, i * r:(i + c) * r].contiguous()
        lr_it = lr * 0.5 * (1.0 + math.cos(math.pi * it / iters))
        losses.append(net.train_step(x, t, lr_it, fw))
        if log and (it % 200 == 0 or it == iters - 1):
            log("iter %d loss %.4e (%.1f s)" % (it, losses[-1], time.perf_counter() - t0))
    torch.cuda.synchronize()
    return np.array(losses)


def predict_fine(net, pair, use_net=True):
    """Fine-grid eta, hu, hv: prolongation of the coarse state plus the network's
    correction (or the plain prolongation)."""
    import torch
    nc = pair["x"].shape[-1]
    r = net.r
    y = net.forward(pair["x"]) if use_net else None
    out = torch.empty((3, nc * r, nc * r), dtype=torch.float64, device="cuda")
    _ck(lib().lc_apply(_p(pair["qc"]), _p(y) if use_net else None, nc, nc, r, S_ETA, S_Q, int(use_net), _p(out),
                       _stream()), "lc_apply")
    return out


def evaluate(net, pairs, block=8, bound=0.05, indicator_thr=0.02):
    """Relative L2 error of eta at the fine level, prolongation vs corrected, and
    the fallback: per block of block x block coarse cells, blocks whose corrected
    error (relative L2 against the fine solve, over the block) exceeds `bound` fall
    back to the fine solve.  Also the a-priori indicator of the paper's refinement
    flag, |d eta| between coarse neighbours > indicator_thr [m], and how many of
    the over-bound blocks it flags (recall)."""
    import torch
    r = net.r
    rows = []
    for p in pairs:
        qf = p["qf"]
        eta_f = qf[0]
        pp = predict_fine(net, p, use_net=False)[0]
        pn = predict_fine(net, p, use_net=True)[0]
        e_p = torch.linalg.norm(pp - eta_f).item()
        e_n = torch.linalg.norm(pn - eta_f).item()
        nf = eta_f.shape[0]
        nb = nf // (block * r)
        bsz = block * r
        d2 = ((pn - eta_f) ** 2)[:nb * bsz, :nb * bsz].reshape(nb, bsz, nb, bsz).sum(dim=(1, 3))
        ref2 = ((eta_f - eta_f.mean()) ** 2)[:nb * bsz, :nb * bsz].reshape(nb, bsz, nb, bsz).sum(dim=(1, 3))
        sig = (eta_f.abs().max().item() ** 2) * bsz * bsz * 1e-6
        rel = torch.sqrt(d2 / (ref2 + sig))
        over = rel > bound
        # hybrid: fine solve on the fallback blocks, corrected field elsewhere
        mask = over.repeat_interleave(bsz, 0).repeat_interleave(bsz, 1)
        hyb = pn.clone()
        hyb[:nb * bsz, :nb * bsz][mask] = eta_f[:nb * bsz, :nb * bsz][mask]
        e_h = torch.linalg.norm(hyb - eta_f).item()
        ec = p["qc"][0]
        gx = (ec[:, 1:] - ec[:, :-1]).abs()
        gy = (ec[1:, :] - ec[:-1, :]).abs()
        flag = torch.zeros_like(ec, dtype=torch.bool)
        flag[:, 1:] |= gx > indicator_thr
        flag[:, :-1] |= gx > indicator_thr
        flag[1:, :] |= gy > indicator_thr
        flag[:-1, :] |= gy > indicator_thr
        ncb = nb * block
        fb = flag[:ncb, :ncb].reshape(nb, block, nb, block).any(dim=3).any(dim=1)
        recall = (fb & over).sum().item() / max(over.sum().item(), 1)
        rows.append(dict(scenario=p["scenario"], time=p["time"], err_prolong=e_p, err_net=e_n, err_hybrid=e_h,
                         gain=e_p / max(e_n, 1e-300), fallback_frac=over.float().mean().item(),
                         indicator_frac=fb.float().mean().item(), indicator_recall=recall))
    return rows
