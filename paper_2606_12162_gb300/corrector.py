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
    ("lc_sync", ctypes.c_int, [ctypes.c_void_p]),
    ("lc_fallback_tiles", ctypes.c_int, [DP, DP, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_int, DP, ctypes.c_void_p]),
    ("lc_train_step", ctypes.c_int, [ctypes.c_void_p, DP, DP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.c_float,
                                     ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    ("lc_make_input", ctypes.c_int, [DP, DP, DP, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, DP, ctypes.c_void_p]),
    ("lc_make_target", ctypes.c_int, [DP, DP, DP, DP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                      ctypes.c_float, DP, ctypes.c_void_p]),
    ("lc_apply", ctypes.c_int, [DP, DP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                ctypes.c_int, DP, ctypes.c_void_p]),
    ("lc_restrict", ctypes.c_int, [DP, ctypes.c_int, ctypes.c_int, ctypes.c_int, DP, ctypes.c_void_p]),
]
_ready = False

# scales of the normalised inputs and outputs: surface [m], momentum [m^2/s],
# bathymetry [m] (surface and momentum at the size of the fine/coarse
# differences of the waves, so that the targets are of order 0.1-1)
S_ETA, S_Q, S_B = 0.1, 10.0, 1000.0


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

    def sync(self):
        """Wait for the network's kernels; raises if one reported a failure."""
        _ck(lib().lc_sync(self.h), "lc_sync")

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


def scenario_source(bc, dxc, s):
    """Source of scenario s (seed 5002 + s): centre of a coarse cell deeper than
    1000 m, amplitude U[0.5, 5] m, radius U[10, 50] km."""
    rng = np.random.default_rng(5002 + s)
    deep = np.argwhere(bc < -1000.0)
    j, i = deep[rng.integers(len(deep))]
    return (i + 0.5) * dxc, (j + 0.5) * dxc, rng.uniform(0.5, 5.0), rng.uniform(10e3, 50e3)


def generate_pairs(nc=512, r=4, dxc=2000.0, scenarios=range(40), times=(60.0, 120.0, 180.0, 240.0, 300.0),
                   model=W.HSGN, precision=sgn.MIXED, seed=5001, keep_fine=None, gauges=0, stats=None):
    """Coarse/fine solver pairs: for each scenario (scenario_source) run the
    coarse (nc^2, dxc) and fine ((r nc)^2, dxc/r) solvers to each snapshot time
    and keep (input, target, coarse state[, fine state]) on the device.

    keep_fine(s) -> bool selects the scenarios whose fine eta, hu, hv are kept
    (default: all).  With gauges > 0 both solvers record that many gauges
    (gauge_positions, seed 5100 + s), returned per scenario in stats["gauges"].
    stats (a dict) also receives the wall time and step count of every coarse
    and fine advance, the scenarios kept ("ok") and those dropped because a
    solve reported an error ("failed")."""
    import torch
    bf, bc = scenario_bathymetry(nc, r, seed)
    nf = nc * r
    dxf = dxc / r
    cfg = dict(model=model, bc=(1, 1, 1, 1), h_star=20.0, alpha=3.0, precision=precision)
    sc = sgn.Solver(bc, dx=dxc, **cfg)
    sf = sgn.Solver(bf, dx=dxf, **cfg)
    _, phic = sc.aux()
    bcd = torch.from_numpy(np.ascontiguousarray(bc)).cuda()
    bfd = torch.from_numpy(np.ascontiguousarray(bf)).cuda()
    phid = torch.from_numpy(np.ascontiguousarray(phic)).cuda()
    nv = W.NVAR[model]
    qc = torch.empty((nv, nc, nc), dtype=torch.float64, device="cuda")
    qf = torch.empty((nv, nf, nf), dtype=torch.float64, device="cuda")
    pairs = []
    L = lib()
    st = _stream()
    if stats is not None:
        for k in ("coarse_s", "fine_s", "coarse_steps", "fine_steps", "ok", "failed"):
            stats.setdefault(k, [])
        stats.setdefault("gauges", {})
    for s in scenarios:
        cx, cy, amp, rad = scenario_source(bc, dxc, s)
        # the same source evaluated on each grid (a restriction of the fine
        # state would put water on coarse cells that hold fine land)
        qf0 = source_state(model, bf, dxf, cx, cy, amp, rad)
        qc0 = source_state(model, bc, dxc, cx, cy, amp, rad)
        sf.set_state(qf0)
        sc.set_state(qc0)
        sf.cfl_dt = sc.cfl_dt = 0.0
        if gauges:
            gxy = gauge_positions(bc, dxc, cx, cy, gauges, 5100 + s)
            for sv in (sc, sf):
                sv.clear_gauges()
                sv.add_gauges(gxy, 4096)
        tnow = {id(sc): 0.0, id(sf): 0.0}
        mine, mypairs, failed = [], [], None
        for T in times:
            for sv, key in ((sc, "coarse"), (sf, "fine")):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                try:
                    tnow[id(sv)], nst = advance_to(sv, tnow[id(sv)], T)
                except sgn.SGNError as e:
                    failed = dict(scenario=s, solver=key, target=T, error=str(e))
                    break
                torch.cuda.synchronize()
                mine.append((key, time.perf_counter() - t0, nst))
            if failed:
                break
            sc.get_state_device(qc)
            sf.get_state_device(qf)
            x = torch.empty((5, nc, nc), dtype=torch.float32, device="cuda")
            tg = torch.empty((3, nf, nf), dtype=torch.float32, device="cuda")
            _ck(L.lc_make_input(_p(qc), _p(bcd), _p(phid), nc, nc, S_ETA, S_Q, S_B, _p(x), st), "lc_make_input")
            _ck(L.lc_make_target(_p(qf), _p(qc), _p(bfd), _p(bcd), nc, nc, r, S_ETA, S_Q, _p(tg), st), "lc_make_target")
            keep = keep_fine is None or keep_fine(s)
            mypairs.append(dict(x=x, t=tg, qc=qc[:3].clone(), qf=qf[:3].clone() if keep else None, scenario=s,
                                time=T, centre=(int(cy / dxc), int(cx / dxc))))
        if failed:
            # a scenario whose solve reports an error is dropped whole (and counted)
            if stats is not None:
                stats["failed"].append(failed)
            continue
        pairs.extend(mypairs)
        if stats is not None:
            for key, dt_, nst in mine:
                stats[key + "_s"].append(dt_)
                stats[key + "_steps"].append(nst)
            stats["ok"].append(s)
            if gauges:
                stats["gauges"][s] = dict(xy=gxy, coarse=sc.gauges(), fine=sf.gauges())
    sc.close()
    sf.close()
    return pairs, dict(bc=bc, bf=bf, dxc=dxc, r=r, phic=phic)


def gauge_positions(bc, dxc, cx, cy, n, seed, rmin=20e3, rmax=150e3):
    """n gauge positions: centres of coarse ocean cells (b < -100 m) 20-150 km
    from the source, drawn with the given seed."""
    nc = bc.shape[0]
    x, y = W.cell_centres(nc, nc, dxc, dxc)
    d = np.hypot(x - cx, y - cy)
    jj, ii = np.nonzero((bc < -100.0) & (d > rmin) & (d < rmax))
    rng = np.random.default_rng(seed)
    pick = rng.choice(len(ii), size=min(n, len(ii)), replace=False)
    return np.stack([x[jj[pick], ii[pick]], y[jj[pick], ii[pick]]], axis=1)


def arrival_times(rec, frac=0.1, floor=0.01):
    """First recorded time at which |eta| at a gauge reaches max(frac x its
    largest |eta|, floor [m]); NaN where it never does.
    rec: [record][gauge][t, eta, hu, hv]."""
    t = rec[:, :, 0]
    e = np.abs(rec[:, :, 1])
    thr = np.maximum(frac * e.max(axis=0), floor)
    out = np.full(rec.shape[1], np.nan)
    for g in range(rec.shape[1]):
        k = np.nonzero(e[:, g] >= thr[g])[0]
        if len(k) and e[:, g].max() >= floor:
            out[g] = t[k[0], g]
    return out


def advance_to(sv, t, T):
    """Step a solver from time t to exactly T without exceeding the CFL step.
    Far from T, batches of CFL steps, each batch at most half the remaining
    interval over the largest step seen (the step shrinks briefly when a thin
    layer runs up a shore and then recovers, so the last step is no bound);
    within two CFL steps of T, fixed steps no longer than the solver's next CFL
    step.  A fresh state (cfl_dt reset to 0 on the solver object after
    set_state) starts with a few single steps.  Returns (T, steps taken)."""
    n = 0
    dmax = getattr(sv, "cfl_dt", 0.0)
    warm = 4 if dmax <= 0.0 else 0
    while T - t > 1e-9:
        rem = T - t
        if warm == 0 and dmax > 0.0 and rem > 4.0 * dmax:
            k = max(1, int(0.5 * rem / dmax) - 1)
            t = sv.step(k)
            n += k
            dmax = max(dmax, sv.status()[1])
            if t > T + 1e-9:
                raise RuntimeError("advance_to passed the target time (%.6g > %.6g)" % (t, T))
            continue
        dn = sv.next_dt()
        if dn <= 0.0:
            raise RuntimeError("advance_to: no CFL step (every cell dry)")
        if rem <= dn:
            sv.step_dt(rem)
            t = T
        elif rem <= 2.0 * dn:
            sv.step_dt(0.5 * rem)
            t += 0.5 * rem
        else:
            t = sv.step(1)
            dmax = max(dmax, sv.status()[1])
            warm = max(0, warm - 1)
        n += 1
    sv.cfl_dt = dmax
    return T, n


def train(net, pairs, iters=2000, crop=64, lr=1e-3, seed=0, fw=(1.0, 1.0, 1.0), log=None, near=0.8):
    """Adam on crops of the training pairs (crop x crop coarse cells): with
    probability `near` a crop whose centre lies within crop/2 of the scenario's
    source (where the waves are: far from them the target is zero), otherwise
    anywhere."""
    import torch
    rng = np.random.default_rng(seed)
    r = net.r
    losses = []
    t0 = time.perf_counter()
    for it in range(iters):
        p = pairs[int(rng.integers(len(pairs)))]
        nc = p["x"].shape[-1]
        c = min(crop, nc)
        if "centre" in p and rng.random() < near:
            cj, ci = p["centre"]
            j = int(np.clip(cj - c // 2 + rng.integers(-(c // 2), c // 2 + 1), 0, nc - c))
            i = int(np.clip(ci - c // 2 + rng.integers(-(c // 2), c // 2 + 1), 0, nc - c))
        else:
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


def evaluate(net, pairs, block=8, bound=0.05, indicator_thr=0.02, ocean_f=None, ocean_c=None):
    """Error of the fine-level surface over the ocean (ocean_f: fine cells with
    b < 0 whose coarse cell has b < 0 as well; all cells if None: on land the
    surface is bathymetry, not a wave), plain prolongation vs corrected,
    relative to the surface's own norm over the ocean; and the fallback: blocks
    of block x block coarse cells whose RMS corrected error over their ocean
    exceeds `bound` x the RMS of the fine surface over the whole ocean fall
    back to the fine solve.  Also the a-priori indicator of the paper's
    refinement flag, |d eta| > indicator_thr [m] between neighbouring coarse
    ocean cells (ocean_c), and how many of the over-bound blocks it flags."""
    import torch
    r = net.r
    rows = []
    for p in pairs:
        qf = p["qf"]
        eta_f = qf[0]
        m = torch.ones_like(eta_f) if ocean_f is None else ocean_f.to(eta_f.dtype)
        pp = predict_fine(net, p, use_net=False)[0]
        pn = predict_fine(net, p, use_net=True)[0]
        e_p = torch.linalg.norm((pp - eta_f) * m).item()
        e_n = torch.linalg.norm((pn - eta_f) * m).item()
        ref = torch.linalg.norm(eta_f * m).item()
        nf = eta_f.shape[0]
        nb = nf // (block * r)
        bsz = block * r
        cut = (slice(0, nb * bsz), slice(0, nb * bsz))
        d2 = (((pn - eta_f) * m) ** 2)[cut].reshape(nb, bsz, nb, bsz).sum(dim=(1, 3))
        nblk = m[cut].reshape(nb, bsz, nb, bsz).sum(dim=(1, 3)).clamp(min=1.0)
        rms_all = ref / max(m.sum().item(), 1.0) ** 0.5
        over = torch.sqrt(d2 / nblk) > bound * rms_all
        # hybrid: fine solve on the fallback blocks, corrected field elsewhere
        mask = over.repeat_interleave(bsz, 0).repeat_interleave(bsz, 1)
        hyb = pn.clone()
        hyb[cut][mask] = eta_f[cut][mask]
        e_h = torch.linalg.norm((hyb - eta_f) * m).item()
        ec = p["qc"][0]
        oc = torch.ones_like(ec, dtype=torch.bool) if ocean_c is None else ocean_c
        gx = ((ec[:, 1:] - ec[:, :-1]).abs() > indicator_thr) & oc[:, 1:] & oc[:, :-1]
        gy = ((ec[1:, :] - ec[:-1, :]).abs() > indicator_thr) & oc[1:, :] & oc[:-1, :]
        flag = torch.zeros_like(ec, dtype=torch.bool)
        flag[:, 1:] |= gx
        flag[:, :-1] |= gx
        flag[1:, :] |= gy
        flag[:-1, :] |= gy
        ncb = nb * block
        fb = flag[:ncb, :ncb].reshape(nb, block, nb, block).any(dim=3).any(dim=1)
        recall = (fb & over).sum().item() / max(over.sum().item(), 1)
        rows.append(dict(scenario=p["scenario"], time=p["time"], err_prolong=e_p, err_net=e_n, err_hybrid=e_h,
                         rel_prolong=e_p / max(ref, 1e-300), rel_net=e_n / max(ref, 1e-300),
                         rel_hybrid=e_h / max(ref, 1e-300),
                         gain=e_p / max(e_n, 1e-300), fallback_frac=over.float().mean().item(),
                         indicator_frac=fb.float().mean().item(), indicator_recall=recall))
    return rows



def ocean_masks(meta):
    """(fine cells with b < 0 whose coarse cell has b < 0, coarse cells with
    b < 0) as device booleans."""
    import torch
    r = meta["r"]
    bc = meta["bc"]
    pc = np.repeat(np.repeat(bc < 0.0, r, axis=0), r, axis=1)
    return torch.from_numpy((meta["bf"] < 0.0) & pc).cuda(), torch.from_numpy(bc < 0.0).cuda()


def correct(net, qc, bcd, phid, out=None):
    """Fine-level eta, hu, hv (3, r nc, r nc) from a coarse device state qc (its
    first three fields are read): input assembly, the network and the corrected
    prolongation, all library kernels on the current stream."""
    import torch
    nc = qc.shape[-1]
    r = net.r
    x = torch.empty((5, nc, nc), dtype=torch.float32, device="cuda")
    st = _stream()
    L = lib()
    _ck(L.lc_make_input(_p(qc), _p(bcd), _p(phid), nc, nc, S_ETA, S_Q, S_B, _p(x), st), "lc_make_input")
    y = net.forward(x)
    if out is None:
        out = torch.empty((3, nc * r, nc * r), dtype=torch.float64, device="cuda")
    _ck(L.lc_apply(_p(qc), _p(y), nc, nc, r, S_ETA, S_Q, 1, _p(out), st), "lc_apply")
    return out


def _tile_cuts(n, tile):
    """Tiles of `tile` cells from the low corner, a one-cell remainder joined to
    the tile before it: (start, width) pairs."""
    cuts, x = [], 0
    while x < n:
        w = min(tile, n - x)
        if n - (x + w) == 1:
            w += 1
        cuts.append((x, w))
        x += w
    return cuts


def fallback_boxes(eta, b, thr, hmin, tile, buffer, r):
    """Level-1 boxes of the runtime fallback from a coarse surface eta and
    bathymetry b (H x W FP64 device tensors): the paper's refinement flag
    (Sec. 6.3), a surface jump |eta - eta_n| > thr between neighbouring cells,
    counted only between cells deeper than hmin (away from the shore, where the
    relaxed system runs as SWE anyway and where a coarse cell partly over land
    would take its children's mean depth under a patch), widened by `buffer`
    cells; every tile (tile x tile squares from the low corner, a one-cell
    remainder joined to the square before it) holding a widened flag and no
    cell shallower than hmin becomes a box (in fine cells).  The flags and the
    tile selection run in lc_fallback_tiles."""
    import torch
    H, Wd = eta.shape[-2], eta.shape[-1]
    cy, cx = _tile_cuts(H, tile), _tile_cuts(Wd, tile)
    sel = torch.empty((len(cy), len(cx)), dtype=torch.uint8, device=eta.device)
    _ck(lib().lc_fallback_tiles(_p(eta), _p(b), H, Wd, float(thr), float(hmin), int(tile), int(buffer), _p(sel),
                                _stream()), "lc_fallback_tiles")
    sh = sel.cpu().numpy()
    boxes = []
    for ty, (y0, h_) in enumerate(cy):
        for tx, (x0, w_) in enumerate(cx):
            if sh[ty, tx]:
                boxes.append((x0 * r, y0 * r, w_ * r, h_ * r))
    return boxes


def hybrid_run(net, meta, s, times, on_snapshot, thr=0.05, tile=16, buffer=4, regrid_every=8, model=W.HSGN,
               uniform_input=True, hmin=20.0):
    """The learned form with its runtime fallback to the plain fine solve, on
    scenario s: a two-level refined hierarchy whose level 0 is the coarse grid
    and whose level-1 patches (ratio r, the fine grid's spacing and bathymetry)
    cover the cells the paper's refinement flag marks on the coarse state
    (fallback_boxes: a surface jump above `thr` [m] between neighbouring cells
    deeper than `hmin`, widened by `buffer` coarse cells, tile x tile boxes)
    and follow the flow by a regrid every `regrid_every` level-0 steps.  The
    flag is computed from the coarse state alone, never from the fine
    solution.  At each output time T (reached exactly, as
    advance_to does) the fine-level surface is the network's corrected
    prolongation of the coarse state outside the patches and the patches' own
    fine solve inside.  With uniform_input the network reads a separate plain
    coarse solve advanced beside the hierarchy -- the state it was trained on;
    otherwise it reads level 0, which holds the patches' average where they
    cover it.  net = None gives the plain prolongation outside the patches;
    on_snapshot(T, fine) receives it (3 x r nc x r nc FP64 on the device, eta,
    hu, hv; valid during the call).  Returns the wall time split into stepping,
    regridding and snapshots (network and assembly), the level-0 steps, the
    regrids, and the patch share of the fine grid at each output time."""
    import torch
    from . import amr
    bf, bc, dxc, r = meta["bf"], meta["bc"], meta["dxc"], meta["r"]
    nc = bc.shape[0]
    nf = nc * r
    nv = W.NVAR[model]
    cx, cy, amp, rad = scenario_source(bc, dxc, s)
    h = amr.Hierarchy(bf, nc, nc, dxc, r, [[]], model=model, bc=(1, 1, 1, 1), precision=sgn.MIXED, h_star=20.0,
                      alpha=3.0)
    q0 = source_state(model, bc, dxc, cx, cy, amp, rad)
    h.set_patch(0, 0, q0)
    sc = None
    if uniform_input:
        sc = sgn.Solver(bc, dx=dxc, model=model, bc=(1, 1, 1, 1), h_star=20.0, alpha=3.0, precision=sgn.MIXED)
        sc.set_state(q0)
        sc.cfl_dt = 0.0
        tc = 0.0
    bcd = torch.from_numpy(np.ascontiguousarray(bc)).cuda()
    phid = torch.from_numpy(np.ascontiguousarray(meta["phic"])).cuda()
    qcd = torch.empty((nv, nc, nc), dtype=torch.float64, device="cuda")
    e0 = torch.empty((1, nc, nc), dtype=torch.float64, device="cuda")
    out = torch.empty((3, nf, nf), dtype=torch.float64, device="cuda")
    res = dict(step_s=0.0, regrid_s=0.0, snapshot_s=0.0, steps=0, regrids=0, patch_frac=[], patches=[])
    # as advance_to: single steps first (the step after a new state is computed
    # by that step), then batches sized by the largest step seen
    t, since, warm, dmax = 0.0, regrid_every, 4, 0.0

    def clock():
        torch.cuda.synchronize()
        return time.perf_counter()

    try:
        for T in times:
            while T - t > 1e-9:
                if since >= regrid_every:
                    c0 = clock()
                    h.get_level_device(0, e0)
                    h.regrid(bf, [fallback_boxes(e0[0], bcd, thr, hmin, tile, buffer, r)])
                    res["regrid_s"] += clock() - c0
                    res["regrids"] += 1
                    since = 0
                rem = T - t
                c0 = clock()
                if warm == 0 and dmax > 0.0 and rem > 4.0 * dmax:
                    k = max(1, min(regrid_every - since, int(0.5 * rem / dmax) - 1))
                    t = h.step(k)
                    if t > T + 1e-9:
                        raise RuntimeError("hybrid_run passed the output time (%.6g > %.6g)" % (t, T))
                else:
                    dn = h.next_dt()
                    k = 1
                    if warm > 0 or dn <= 0.0 or rem > 2.0 * dn:
                        tb = t
                        t = h.step(1)
                        dmax = max(dmax, t - tb)
                        warm = max(0, warm - 1)
                        if t > T + 1e-9:
                            raise RuntimeError("hybrid_run passed the output time (%.6g > %.6g)" % (t, T))
                    elif rem <= dn:
                        h.step_dt(rem)
                        t = T
                    else:
                        h.step_dt(0.5 * rem)
                        t += 0.5 * rem
                if k > 1 or warm == 0:
                    dmax = max(dmax, h.next_dt())
                res["step_s"] += clock() - c0
                res["steps"] += k
                since += k
            # fine-level surface: network outside the patches, fine solve inside
            c0 = clock()
            if sc is not None:
                tc, _ = advance_to(sc, tc, T)
                sc.get_state_device(qcd)
            else:
                h.get_level_device(0, qcd)
            if net is not None:
                correct(net, qcd, bcd, phid, out)
            else:
                _ck(lib().lc_apply(_p(qcd), None, nc, nc, r, S_ETA, S_Q, 0, _p(out), _stream()), "lc_apply")
            h.get_level_device(1, out)            # the patches' fine solve over the network's field
            area = sum(bx * by for (_, _, bx, by) in h.get_boxes(1))
            res["snapshot_s"] += clock() - c0
            res["patch_frac"].append(area / float(nf * nf))
            res["patches"].append(h.npatches(1))
            on_snapshot(T, out)
    finally:
        h.close()
        if sc is not None:
            sc.close()
    return res


def _rel_l2(a, b):
    import torch
    return (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()


def experiment(nc=1024, r=4, dxc=2000.0, n_train=32, n_held=8, times=(60.0, 120.0, 180.0, 240.0, 300.0),
               iters=6000, crop=128, lr=1e-3, width=32, depth=5, block=16, bound=0.1, gauges=64, fp64_check=True,
               log=print):
    """Generate the coarse/fine pairs, train the corrector on scenarios below
    n_train, evaluate it on the others, and time the ways of getting the
    fine-level surface at the snapshot times: the plain fine solve (mixed
    precision), the plain fine solve in FP64 (first held-out scenario) and the
    coarse solve plus the corrector.  Returns a dict of results."""
    import torch
    res = dict(nc=nc, r=r, nf=nc * r, dxc=dxc, n_train=n_train, n_held=n_held, times=list(times), iters=iters,
               crop=crop, width=width, depth=depth, block=block, bound=bound)
    stats = {}
    t0 = time.perf_counter()
    pairs, meta = generate_pairs(nc, r, dxc, range(n_train + n_held), times, keep_fine=lambda s: s >= n_train,
                                 gauges=gauges, stats=stats)
    res["generate_s"] = time.perf_counter() - t0
    res["failed"] = stats["failed"]
    ok = stats["ok"]
    log("pairs: %d in %.1f s, dropped scenarios: %d" % (len(pairs), res["generate_s"], len(stats["failed"])))
    trn = [p for p in pairs if p["scenario"] < n_train]
    held = [p for p in pairs if p["scenario"] >= n_train]
    if not trn or not held:
        raise RuntimeError("no usable scenarios: %s" % res["failed"])
    net = Net(cin=5, width=width, depth=depth, r=r, max_hw=nc * nc, seed=5000)
    res["params"] = int(net.n)
    t0 = time.perf_counter()
    losses = train(net, trn, iters, crop, lr, log=log)
    res["train_s"] = time.perf_counter() - t0
    res["loss_first50"] = float(losses[:50].mean())
    res["loss_last50"] = float(losses[-50:].mean())
    ocean_f, ocean_c = ocean_masks(meta)
    rows = evaluate(net, held, block, bound, ocean_f=ocean_f, ocean_c=ocean_c)
    res["rows"] = rows
    for k in ("rel_prolong", "rel_net", "rel_hybrid", "gain", "fallback_frac", "indicator_frac",
              "indicator_recall"):
        v = np.array([row[k] for row in rows])
        res[k + "_median"] = float(np.median(v))
        res[k + "_min"] = float(v.min())
        res[k + "_max"] = float(v.max())
    # inference time per snapshot (input assembly, network, corrected prolongation)
    bcd = torch.from_numpy(np.ascontiguousarray(meta["bc"])).cuda()
    phid = torch.from_numpy(np.ascontiguousarray(meta["phic"])).cuda()
    out = torch.empty((3, nc * r, nc * r), dtype=torch.float64, device="cuda")
    for _ in range(3):
        correct(net, held[0]["qc"], bcd, phid, out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record()
    for k in range(reps):
        correct(net, held[k % len(held)]["qc"], bcd, phid, out)
    e1.record()
    torch.cuda.synchronize()
    t_inf = e0.elapsed_time(e1) / reps * 1e-3
    res["inference_ms"] = t_inf * 1e3
    res["inference_gflop"] = 2.0 * sum(ci * co * 9 for ci, co in net.layers()) * nc * nc * 1e-9
    # throughput: fine-level cell-updates delivered per second of wall time
    nt = len(times)
    nsc = len(ok)
    cs = np.array(stats["coarse_s"]).reshape(nsc, nt).sum(axis=1)
    fs = np.array(stats["fine_s"]).reshape(nsc, nt).sum(axis=1)
    cst = np.array(stats["coarse_steps"]).reshape(nsc, nt).sum(axis=1)
    fst = np.array(stats["fine_steps"]).reshape(nsc, nt).sum(axis=1)
    nf2 = float(nc * r) ** 2
    fine_updates = nf2 * fst
    res["fine_steps_median"] = float(np.median(fst))
    res["coarse_steps_median"] = float(np.median(cst))
    res["fine_mixed_cups"] = float(np.sum(fine_updates) / np.sum(fs))
    learned_s = cs + nt * t_inf
    res["learned_cups"] = float(np.sum(fine_updates) / np.sum(learned_s))
    # fallback cost model: the fine solve over the fallback share of the domain
    ff = res["fallback_frac_median"]
    res["learned_with_fallback_cups"] = float(np.sum(fine_updates) / np.sum(learned_s + ff * fs))
    # gauge arrival times, coarse vs fine (held-out scenarios)
    if gauges:
        d, dtc = [], []
        for s in [v for v in ok if v >= n_train]:
            g = stats["gauges"][s]
            ta, tb = arrival_times(g["coarse"]), arrival_times(g["fine"])
            keep = np.isfinite(ta) & np.isfinite(tb)
            d.extend(np.abs(ta[keep] - tb[keep]).tolist())
            dtc.append(float(np.median(np.diff(g["coarse"][:, 0, 0]))))
        d = np.array(d)
        res["arrival_gauges"] = int(d.size)
        res["arrival_abs_diff_median_s"] = float(np.median(d)) if d.size else None
        res["arrival_abs_diff_max_s"] = float(d.max()) if d.size else None
        res["coarse_dt_median_s"] = float(np.median(dtc)) if dtc else None
    # FP64 fine solve of the first held-out scenario
    if fp64_check:
        s = held[0]["scenario"]
        cx, cy, amp, rad = scenario_source(meta["bc"], dxc, s)
        bf = meta["bf"]
        dxf = dxc / r
        sv = sgn.Solver(bf, dx=dxf, model=W.HSGN, bc=(1, 1, 1, 1), h_star=20.0, alpha=3.0, precision=sgn.FP64)
        sv.set_state(source_state(W.HSGN, bf, dxf, cx, cy, amp, rad))
        sv.cfl_dt = 0.0
        q64 = torch.empty((W.NVAR[W.HSGN], nc * r, nc * r), dtype=torch.float64, device="cuda")
        tt, nst, wall = 0.0, 0, 0.0
        e_mixed, e_net, e_pro = [], [], []
        try:
            for T, p in zip(times, [p for p in held if p["scenario"] == s]):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                tt, k = advance_to(sv, tt, T)
                torch.cuda.synchronize()
                wall += time.perf_counter() - t0
                nst += k
                sv.get_state_device(q64)
                e_mixed.append(_rel_l2(p["qf"][0] * ocean_f, q64[0] * ocean_f))
                e_net.append(_rel_l2(predict_fine(net, p, True)[0] * ocean_f, q64[0] * ocean_f))
                e_pro.append(_rel_l2(predict_fine(net, p, False)[0] * ocean_f, q64[0] * ocean_f))
        except sgn.SGNError as e:
            res["fp64_error"] = dict(scenario=s, time=tt, error=str(e))
        sv.close()
        if e_mixed:
            res["fine_fp64_cups"] = nf2 * nst / wall
            res["fp64_rel_l2_eta_fine_mixed_max"] = float(max(e_mixed))
            res["fp64_rel_l2_eta_learned_max"] = float(max(e_net))
            res["fp64_rel_l2_eta_prolong_max"] = float(max(e_pro))
    res["weights"] = net.params()
    return res


def main(argv=None):
    """Command line: run the corrector experiment and write a JSON summary
    (and the trained FP32 parameters as .npy)."""
    import argparse
    import json
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--nc", type=int, default=1024)
    ap.add_argument("--r", type=int, default=4)
    ap.add_argument("--dxc", type=float, default=2000.0)
    ap.add_argument("--train", type=int, default=32)
    ap.add_argument("--held", type=int, default=8)
    ap.add_argument("--iters", type=int, default=6000)
    ap.add_argument("--crop", type=int, default=128)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--block", type=int, default=16)
    ap.add_argument("--bound", type=float, default=0.1)
    ap.add_argument("--gauges", type=int, default=64)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--out", default=None, help="JSON summary path")
    ap.add_argument("--weights", default=None, help="trained parameters (.npy)")
    ap.add_argument("--profile", type=int, default=0, metavar="N",
                    help="instead of the experiment: one forward pass and one training step of the network on "
                         "random N x N inputs (a small, fixed launch sequence for a profiler)")
    a = ap.parse_args(argv)
    if a.profile:
        import torch
        lib()
        n = a.profile
        net = Net(cin=5, width=32, depth=5, r=a.r, max_hw=n * n, seed=5000)
        g = torch.Generator(device="cuda").manual_seed(0)
        x = torch.randn((5, n, n), device="cuda", generator=g)
        t = torch.randn((3, n * a.r, n * a.r), device="cuda", generator=g)
        net.forward(x)
        net.train_step(x, t, 0.0)
        torch.cuda.synchronize()
        print("profile run done: %d x %d" % (n, n))
        return
    res = experiment(nc=a.nc, r=a.r, dxc=a.dxc, n_train=a.train, n_held=a.held, iters=a.iters, crop=a.crop,
                     lr=a.lr, block=a.block, bound=a.bound, gauges=a.gauges, fp64_check=not a.no_fp64,
                     log=lambda m: print(m, flush=True))
    w = res.pop("weights")
    if a.weights:
        np.save(a.weights, w)
    txt = json.dumps(res, indent=1, default=float)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt)
    print(json.dumps({k: v for k, v in res.items() if k != "rows"}, default=float))


if __name__ == "__main__":
    main()
