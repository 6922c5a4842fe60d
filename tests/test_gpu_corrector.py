"""Learned corrector on the GPU: its forward/backward kernels against the FP64
NumPy reference, its data kernels against NumPy, and what the trained network
gains over the plain prolongation on held-out scenarios (with the fallback to
the fine solve where its error exceeds the bound)."""
import numpy as np
import pytest

from paper_2606_12162_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_12162_gb300 import build, corrector
    build.build()
    corrector.lib()
    return corrector


def test_gradients_match_fp64_reference(C):
    import torch
    from oracle import conv_ref as R
    rng = np.random.default_rng(3)
    net = C.Net(cin=5, width=8, depth=3, r=2, nout=3, max_hw=64 * 64, seed=7)
    p = net.params()
    x = rng.standard_normal((5, 20, 24)).astype(np.float32)
    t = rng.standard_normal((3, 40, 48)).astype(np.float32)
    fw = (1.0, 0.3, 0.3)
    loss, g = net.train_step(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), 0.0, fw, want_grad=True)
    # the kernels multiply BF16 weights by BF16-rounded activations and
    # gradients on the tensor cores (FP32 accumulation, FP32 biases); the FP64
    # reference rounds the same operands
    pr = p.astype(np.float64)
    off = 0
    for ci, co in net.layers():
        pr[off:off + ci * co * 9] = R.bf16_round(p[off:off + ci * co * 9])
        off += ci * co * 9 + co
    lref, gref = R.loss_and_grad(pr, net.layers(), x, t, 2, 3, fw, quant=R.bf16_round)
    assert abs(loss - lref) <= 1e-5 * lref
    assert np.abs(g - gref).max() <= 1e-4 * np.abs(gref).max()
    # forward alone
    yd = net.forward(torch.from_numpy(x).cuda())
    net.sync()                      # no convolution gave up waiting for its tensor-core work
    y = yd.cpu().numpy()
    yref = R.forward(pr, net.layers(), x, quant=R.bf16_round)[-1]
    assert np.abs(y - yref).max() <= 1e-4 * np.abs(yref).max()


@pytest.mark.parametrize("cin,width,depth,r,nout,H,W", [(5, 32, 3, 4, 3, 37, 70), (5, 16, 2, 2, 3, 9, 33),
                                                       (7, 48, 3, 2, 4, 16, 32), (5, 32, 3, 4, 3, 67, 300)])
def test_tensor_core_layers_match_reference(C, cin, width, depth, r, nout, H, W):
    """The tensor-core convolutions at the channel counts of the full network
    (5 -> 32 -> 48 with ratio 4 and 3 fields, the 48-channel gradient into 32
    channels, 7 -> 48 -> 16) and at ragged tile edges (tiles of 4 rows x 128
    columns: 67 x 300 spans 17 x 3 of them): loss and gradients within 1e-4 of the FP64 reference with the
    same BF16 operand rounding; the same step twice gives the same bits."""
    import torch
    from oracle import conv_ref as R
    rng = np.random.default_rng(cin + width + H)
    net = C.Net(cin=cin, width=width, depth=depth, r=r, nout=nout, max_hw=H * W, seed=3)
    p = net.params()
    x = rng.standard_normal((cin, H, W)).astype(np.float32)
    t = rng.standard_normal((nout, H * r, W * r)).astype(np.float32)
    fw = tuple([1.0] + [0.5] * (nout - 1))
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    loss, g = net.train_step(xd, td, 0.0, fw, want_grad=True)
    loss2, g2 = net.train_step(xd, td, 0.0, fw, want_grad=True)
    assert loss == loss2 and np.array_equal(g, g2)
    pr = p.astype(np.float64)
    off = 0
    for ci, co in net.layers():
        pr[off:off + ci * co * 9] = R.bf16_round(p[off:off + ci * co * 9])
        off += ci * co * 9 + co
    lref, gref = R.loss_and_grad(pr, net.layers(), x, t, r, nout, fw, quant=R.bf16_round)
    assert abs(loss - lref) <= 1e-5 * lref
    assert np.abs(g - gref).max() <= 1e-4 * np.abs(gref).max()


def test_data_kernels(C):
    import torch
    L = C.lib()
    rng = np.random.default_rng(4)
    nc, r = 12, 4
    qc = rng.standard_normal((3, nc, nc))
    qf = rng.standard_normal((3, nc * r, nc * r))
    b = rng.uniform(-100, 20, (nc, nc))
    phi = (b < -30).astype(np.uint8)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x = torch.empty((5, nc, nc), dtype=torch.float32, device="cuda")
    assert L.lc_make_input(C._p(d(qc)), C._p(d(b)), C._p(d(phi)), nc, nc, 2.0, 50.0, 100.0, C._p(x), None) == 0
    t = torch.empty((3, nc * r, nc * r), dtype=torch.float32, device="cuda")
    assert L.lc_make_target(C._p(d(qf)), C._p(d(qc)), None, None, nc, nc, r, 2.0, 50.0, C._p(t), None) == 0
    bfine = rng.uniform(-50, 20, (nc * r, nc * r))
    tm = torch.empty((3, nc * r, nc * r), dtype=torch.float32, device="cuda")
    assert L.lc_make_target(C._p(d(qf)), C._p(d(qc)), C._p(d(bfine)), C._p(d(b)), nc, nc, r, 2.0, 50.0, C._p(tm),
                            None) == 0
    y = torch.from_numpy(rng.standard_normal((3 * r * r, nc, nc)).astype(np.float32)).cuda()
    out = torch.empty((3, nc * r, nc * r), dtype=torch.float64, device="cuda")
    assert L.lc_apply(C._p(d(qc)), C._p(y), nc, nc, r, 2.0, 50.0, 1, C._p(out), None) == 0
    fine = torch.from_numpy(qf[0].copy()).cuda()
    co = torch.empty((nc, nc), dtype=torch.float64, device="cuda")
    assert L.lc_restrict(C._p(fine), nc, nc, r, C._p(co), None) == 0
    torch.cuda.synchronize()
    xr = np.stack([np.where(b < 0, qc[0], 0) / 2.0, qc[1] / 50.0, qc[2] / 50.0, b / 100.0, phi])
    assert np.allclose(x.cpu().numpy(), xr, rtol=1e-6, atol=1e-7)
    P = np.repeat(np.repeat(qc, r, axis=1), r, axis=2)
    s = np.array([2.0, 50.0, 50.0])[:, None, None]
    assert np.allclose(t.cpu().numpy(), (qf - P) / s, rtol=1e-6, atol=1e-6)
    tmr = (qf - P) / s
    land = (bfine >= 0.0) | np.repeat(np.repeat(b >= 0.0, r, 0), r, 1)
    tmr[0] = np.where(land, 0.0, tmr[0])                 # no surface target on land
    assert np.allclose(tm.cpu().numpy(), tmr, rtol=1e-6, atol=1e-6)
    from oracle import conv_ref as R
    assert np.allclose(out.cpu().numpy(), P + s * R.shuffle(y.cpu().numpy().astype(np.float64), r, 3), rtol=1e-12)
    assert np.allclose(co.cpu().numpy(), qf[0].reshape(nc, r, nc, r).mean(axis=(1, 3)), rtol=1e-13)


def test_trained_corrector_gains_over_prolongation(C):
    """Coarse 64^2 at 2 km, fine 256^2 at 500 m (ratio 4) over a seeded fractal
    bathymetry: 6 training scenarios x 3 snapshots, 2 held-out scenarios.  The
    trained network brings the surface closer to the fine solve than the plain
    prolongation (median gain over the held-out snapshots above 1.2, none more
    than 2 % worse), and the hybrid with the fine solve on the blocks over the
    bound is no worse than the network.  Errors are taken over the ocean (land
    keeps eta = b and carries no wave).  The full-size experiment (config 5) is
    run by python -m paper_2606_12162_gb300.corrector."""
    pairs, meta = C.generate_pairs(nc=64, r=4, dxc=2000.0, scenarios=range(8), times=(60.0, 120.0, 180.0))
    train = [p for p in pairs if p["scenario"] < 6]
    held = [p for p in pairs if p["scenario"] >= 6]
    net = C.Net(cin=5, width=16, depth=4, r=4, nout=3, max_hw=64 * 64, seed=11)
    losses = C.train(net, train, iters=2000, crop=32, lr=2e-3)
    assert losses[-50:].mean() < 0.5 * losses[:50].mean()
    ocean_f, ocean_c = C.ocean_masks(meta)
    rows = C.evaluate(net, held, block=8, bound=0.1, ocean_f=ocean_f, ocean_c=ocean_c)
    gains = np.array([r_["gain"] for r_ in rows])
    assert np.median(gains) > 1.2, gains
    assert (gains > 0.98).all(), gains
    for r_ in rows:
        assert r_["err_hybrid"] <= r_["err_net"] + 1e-12, r_


def test_runtime_fallback_hybrid_small(C):
    """The learned form with its runtime fallback (hybrid_run): patches of the
    plain fine solve where the a-priori surface-jump flag fires on the coarse
    state (deep water), the trained network's corrected prolongation elsewhere.
    Coarse 64^2 at 2 km, fine 256^2 at 500 m, 6 training and 2 held-out
    scenarios.  Bound, at every held-out snapshot: the hybrid's surface error
    (relative L2 over the ocean against the full fine solve) is at most 1.05 x
    the network's alone and below the plain prolongation's; the patches cover
    part of the grid, not all of it, and the fine solve never ran where no flag
    fired (the flags see the coarse state only)."""
    import torch
    times = (60.0, 120.0, 180.0)
    pairs, meta = C.generate_pairs(nc=64, r=4, dxc=2000.0, scenarios=range(8), times=times)
    train = [p for p in pairs if p["scenario"] < 6]
    held = [p for p in pairs if p["scenario"] >= 6]
    net = C.Net(cin=5, width=16, depth=4, r=4, nout=3, max_hw=64 * 64, seed=11)
    C.train(net, train, iters=2000, crop=32, lr=2e-3)
    ocean_f, ocean_c = C.ocean_masks(meta)
    rows = {(r_["scenario"], r_["time"]): r_ for r_ in C.evaluate(net, held, block=8, bound=0.1, ocean_f=ocean_f,
                                                                    ocean_c=ocean_c)}
    m = ocean_f.to(torch.float64)
    for s in sorted({p["scenario"] for p in held}):
        ref = {p["time"]: p["qf"][0] for p in held if p["scenario"] == s}
        errs = {}

        def cb(T, fine):
            errs[T] = (torch.linalg.norm((fine[0] - ref[T]) * m) / torch.linalg.norm(ref[T] * m)).item()

        res = C.hybrid_run(net, meta, s, times, cb, thr=0.02, tile=8, buffer=2, regrid_every=4)
        assert len(errs) == len(times) and res["regrids"] >= 2
        assert max(res["patch_frac"]) < 0.9
        for T in times:
            r_ = rows[(s, T)]
            assert errs[T] <= 1.05 * r_["rel_net"] + 1e-12, (s, T, errs[T], r_["rel_net"])
            assert errs[T] < r_["rel_prolong"], (s, T, errs[T], r_["rel_prolong"])


def test_fallback_boxes_follow_the_flag(C):
    """fallback_boxes: a deep-water surface jump above the threshold yields a box
    over it (tile-aligned, in fine cells); jumps at or below it, jumps in
    shallow water and tiles holding a shallow cell yield none."""
    import torch
    nc, r = 32, 4
    b = torch.full((nc, nc), -100.0, dtype=torch.float64, device="cuda")
    eta = torch.zeros_like(b)
    eta[10, 5] = 0.05                                  # jump of 5 cm in deep water
    eta[25, 25] = 0.01                                 # below the threshold
    boxes = C.fallback_boxes(eta, b, 0.02, 20.0, 8, 1, r)
    assert boxes == [(0, 32, 32, 32)]                  # the 8 x 8 tile holding (10, 5), in fine cells
    b[8:16, 0:8] = -10.0                               # that tile in shallow water: no box
    assert C.fallback_boxes(eta, b, 0.02, 20.0, 8, 1, r) == []


def test_fallback_tiles_match_their_definition(C):
    """lc_fallback_tiles against the flag written out in NumPy (a cell and a
    face neighbour both deeper than hmin with surfaces more than thr apart;
    dilation by `buffer` in the Chebyshev metric; tiles with a remainder of one
    cell joined to the tile before; no shallow cell in a selected tile), on
    noisy surfaces with four raised cells over deep water with a shallow
    rectangle, for several tile and buffer sizes (each case selects some tiles
    and rejects others both for lack of a flag and for shallow cells)."""
    import torch
    rng = np.random.default_rng(17)
    for (H, Wd, tile, buffer) in ((37, 50, 8, 1), (33, 33, 16, 0), (70, 45, 16, 3), (9, 13, 4, 2)):
        eta = rng.normal(0.0, 0.005, (H, Wd))
        for _ in range(4):
            eta[rng.integers(H), rng.integers(Wd)] += 0.1
        b = np.full((H, Wd), -100.0)
        y0, x0 = rng.integers(H // 2), rng.integers(Wd // 2)
        b[y0:y0 + max(2, H // 4), x0:x0 + max(2, Wd // 4)] = -5.0
        d = eta - b > 20.0
        f = np.zeros((H, Wd), dtype=bool)
        jx = (np.abs(eta[:, 1:] - eta[:, :-1]) > 0.05) & d[:, 1:] & d[:, :-1]
        jy = (np.abs(eta[1:, :] - eta[:-1, :]) > 0.05) & d[1:, :] & d[:-1, :]
        f[:, 1:] |= jx
        f[:, :-1] |= jx
        f[1:, :] |= jy
        f[:-1, :] |= jy
        fw = np.zeros_like(f)
        for y, x in zip(*np.nonzero(f)):
            fw[max(0, y - buffer):y + buffer + 1, max(0, x - buffer):x + buffer + 1] = True
        want = []
        for (y0, h_) in C._tile_cuts(H, tile):
            for (x0, w_) in C._tile_cuts(Wd, tile):
                if fw[y0:y0 + h_, x0:x0 + w_].any() and d[y0:y0 + h_, x0:x0 + w_].all():
                    want.append((x0 * 4, y0 * 4, w_ * 4, h_ * 4))
        got = C.fallback_boxes(torch.from_numpy(eta).cuda(), torch.from_numpy(b).cuda(), 0.05, 20.0, tile, buffer, 4)
        assert got == want, (H, Wd, tile, buffer)
        assert 0 < len(want) < len(C._tile_cuts(H, tile)) * len(C._tile_cuts(Wd, tile))


def test_experiment_pipeline_small(C):
    """The whole experiment driver at a small size: pairs with gauges, training,
    evaluation, inference timing, throughput figures and the FP64 fine check."""
    res = C.experiment(nc=48, r=4, n_train=2, n_held=1, times=(60.0, 120.0), iters=60, crop=16, block=8,
                       gauges=8, fp64_check=True, log=lambda m: None)
    for k in ("rel_net_median", "gain_median", "inference_ms", "fine_mixed_cups", "learned_cups",
              "learned_with_fallback_cups", "fine_fp64_cups", "fp64_rel_l2_eta_fine_mixed_max",
              "fp64_rel_l2_eta_learned_max"):
        assert np.isfinite(res[k]) and res[k] >= 0.0, (k, res[k])
    assert len(res["rows"]) == 2
    assert res["fine_steps_median"] > res["coarse_steps_median"] > 0
    # the mixed fine solve stays close to the FP64 fine solve
    assert res["fp64_rel_l2_eta_fine_mixed_max"] < 1e-3
    assert res["weights"].size == res["params"]
