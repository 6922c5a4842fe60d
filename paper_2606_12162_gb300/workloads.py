"""Seeded synthetic workloads: bathymetry, initial states and gauge positions.

This module holds initial data only (closed-form solitary waves, Gaussians,
synthetic bathymetries); none of the solver's arithmetic.  It is the one module
that both the CUDA path's tests/benchmarks and the CPU oracle's tests draw their
inputs from.

State layout everywhere: float64 array of shape (nvar, ny, nx), fields
eta, hu, hv [, hw] [, h sigma], hp [, h p_b]; eta = h + b relative to the still
level eta0 = 0.  Bathymetry b is negative under water.
"""
import math

import numpy as np

SWE, MBHSGN, HSGN = 0, 1, 2
NVAR = {SWE: 3, MBHSGN: 5, HSGN: 7}
G = 9.81


def field_index(model):
    """Field positions of the auxiliary variables for a model (None if absent)."""
    if model == MBHSGN:
        return dict(hw=3, hs=None, hp=4, hpb=None)
    if model == HSGN:
        return dict(hw=3, hs=4, hp=5, hpb=6)
    return dict(hw=None, hs=None, hp=None, hpb=None)


def cell_centres(nx, ny, dx, dy, x0=0.0, y0=0.0):
    x = x0 + (np.arange(nx) + 0.5) * dx
    y = y0 + (np.arange(ny) + 0.5) * dy
    return np.meshgrid(x, y)


def rest_state(b, model):
    """Lake at rest: eta = max(0, b), everything else zero."""
    q = np.zeros((NVAR[model],) + b.shape)
    q[0] = np.maximum(0.0, b)
    return q


# --------------------------------------------------------------------------
# App. B: solitary wave of SGN (flat bottom, depth H).  The printed pressure has
# prefactor 1/2 and ((2H-h) sech')^2; the form used here, 2/3 * ... *
# [(2H-h) sech'^2 + h sech sech''], is the one that satisfies the travelling-wave
# momentum balance of SGN (checked symbolically).  Over a flat bottom the SGN
# constraints give sigma = 2w and the bottom pressure p_b = 3p/2.
def sgn_soliton(xi_coord, t, a, H, x0, nu=1.0, g=G):
    ell = math.sqrt((H ** 3 / a + H ** 2) * 4.0 / 3.0)
    c0 = nu * math.sqrt(0.75) * ell / H * math.sqrt(g * H ** 3 / (0.75 * ell ** 2 - H ** 2))
    xi = (xi_coord - c0 * t - x0) / ell
    sech = 1.0 / np.cosh(xi)
    tanh = np.tanh(xi)
    d1 = -sech * tanh                       # sech'
    d2 = sech * tanh ** 2 - sech ** 3       # sech''
    h = H + a * sech ** 2
    u = c0 * (1.0 - H / h)
    w = -a * c0 * H / (ell * h) * sech * d1
    p = (2.0 / 3.0) * a * c0 ** 2 * H ** 2 / (ell ** 2 * h ** 2) * ((2.0 * H - h) * d1 ** 2 + h * sech * d2)
    return dict(h=h, u=u, w=w, p=p, sigma=2.0 * w, pb=1.5 * p, ell=ell, c0=c0)


def soliton_state(model, x, y, b, a, H, x0, direction=0, nu=1.0, t=0.0):
    """Planar SGN soliton on depth H travelling along x (direction 0) or y (1)."""
    coord = x if direction == 0 else y
    s = sgn_soliton(coord, t, a, H, x0, nu)
    q = np.zeros((NVAR[model],) + x.shape)
    h = s["h"]
    q[0] = h + b
    q[1 + direction] = h * s["u"]
    fi = field_index(model)
    if fi["hw"] is not None:
        q[fi["hw"]] = h * s["w"]
        q[fi["hp"]] = h * s["p"]
    if fi["hs"] is not None:
        q[fi["hs"]] = h * s["sigma"]
        q[fi["hpb"]] = h * s["pb"]
    return q


def apply_surface(b, bump):
    """Add a surface perturbation over the ocean (b < 0) keeping h >= 0 (eta >= b);
    land keeps eta = b."""
    eta = np.where(b < 0.0, np.maximum(bump, b), b)
    return eta


# --------------------------------------------------------------------------
# Config 1: 256 x 256, dx = 0.05 m, flat bottom depth 1 m, planar SGN soliton
# a = 0.1 m at x0 = 4.8 m travelling in +x, reflective walls, CFL 0.9, 200 steps.
def config1(model=HSGN, nx=256, ny=256, dx=0.05, a=0.1, H=1.0, x0=4.8):
    x, y = cell_centres(nx, ny, dx, dx)
    b = np.full((ny, nx), -H)
    q = soliton_state(model, x, y, b, a, H, x0)
    return dict(b=b, q=q, dx=dx, dy=dx, x0=0.0, y0=0.0, bc=(0, 0, 0, 0), model=model,
                alpha=3.0, h_star=0.0, cfl=0.9, steps=200, dry_tol=1e-3, gauges=None)


# --------------------------------------------------------------------------
# Config 2: 4096 x 4096, dx = 10 m.  b = -200 m for x < 26 km, then a 1:50 beach
# (shoreline at 36 km, dry land up to +99 m), plus a Gaussian seamount of height
# 100 m and radius 500 m (centre seeded, seed 2001).  Initial surface: Gaussian
# depression of -5 m, radius 1 km (centre seeded on the slope, seed 2002).
# Extrapolation boundaries, h* = 20 m, 1000 steps, 64 gauges within 3 km of the
# source (seed 2003).
def config2_bathymetry(nx=4096, ny=4096, dx=10.0, seamount=None):
    x, y = cell_centres(nx, ny, dx, dx)
    L = nx * dx
    scale = L / 40960.0
    xs = 26000.0 * scale
    b = np.where(x < xs, -200.0, -200.0 + (x - xs) / 50.0)
    if seamount is None:
        rng = np.random.default_rng(2001)
        seamount = (rng.uniform(5000, 20000) * scale, rng.uniform(5000, 36000) * scale)
    r2 = (x - seamount[0]) ** 2 + (y - seamount[1]) ** 2
    b = b + 100.0 * np.exp(-r2 / 500.0 ** 2)
    return b, x, y


def config2(model=HSGN, nx=4096, ny=4096, dx=10.0, ngauges=64):
    b, x, y = config2_bathymetry(nx, ny, dx)
    L = nx * dx
    scale = L / 40960.0
    rng = np.random.default_rng(2002)
    cx, cy = rng.uniform(33500, 35000) * scale, rng.uniform(8000, 33000) * scale
    r2 = (x - cx) ** 2 + (y - cy) ** 2
    q = np.zeros((NVAR[model], ny, nx))
    q[0] = apply_surface(b, -5.0 * np.exp(-r2 / 1000.0 ** 2))
    grng = np.random.default_rng(2003)
    wet = (q[0] - b) > 1.0
    near = wet & (r2 < 3000.0 ** 2)
    jj, ii = np.nonzero(near)
    pick = grng.choice(len(ii), size=min(ngauges, len(ii)), replace=False)
    gxy = np.stack([x[jj[pick], ii[pick]], y[jj[pick], ii[pick]]], axis=1)
    return dict(b=b, q=q, dx=dx, dy=dx, x0=0.0, y0=0.0, bc=(1, 1, 1, 1), model=model,
                alpha=3.0, h_star=20.0, cfl=0.9, steps=1000, dry_tol=1e-3, gauges=gxy,
                source=(cx, cy))


# --------------------------------------------------------------------------
# Config 3: 8192 x 8192, dx = 500 m, fractal bathymetry: isotropic Gaussian
# random field with power spectrum |k|^-2 (seed 3001), mapped so that the 80th
# percentile is 0 (about 20 % land) and the minimum is -6000 m, land capped at
# +500 m; Gaussian uplift 2 m, radius 30 km at a cell deeper than 3000 m (seed
# 3002); h* = 20 m, extrapolation boundaries, 2000 steps, 64 gauges (seed 3003).
def fractal_bathymetry(n, seed, depth=6000.0, land_frac=0.2, land_cap=500.0, smooth=0.0):
    """Isotropic Gaussian random field with amplitude spectrum |k|^-1, mapped so
    that land_frac of the cells lie above 0 and the deepest is -depth, land
    capped at land_cap.  smooth > 0: the spectrum is first multiplied by a
    Gaussian low-pass of that width in cells (exp(-2 pi^2 smooth^2 |k|^2), k in
    cycles per cell), which removes one-cell pinnacles the grid cannot resolve."""
    rng = np.random.default_rng(seed)
    kx = np.fft.fftfreq(n)
    k = np.sqrt(kx[None, :] ** 2 + kx[:, None] ** 2)
    k[0, 0] = 1.0
    amp = 1.0 / k
    amp[0, 0] = 0.0
    if smooth > 0.0:
        amp *= np.exp(-2.0 * np.pi ** 2 * smooth ** 2 * k ** 2)
    spec = amp * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    f = np.real(np.fft.ifft2(spec))
    q80 = np.quantile(f, 1.0 - land_frac)
    fmin = f.min()
    b = (f - q80) / (q80 - fmin) * depth
    return np.minimum(b, land_cap)


def config3(model=HSGN, n=8192, dx=500.0, ngauges=64, crop=None, smooth=2.0):
    # low-passed at two cells: the raw field has isolated one-cell pinnacles
    # (e.g. 37 m deep amid 2000 m) on which the relaxed system loses
    # hyperbolicity within a few hundred steps in either precision
    b = fractal_bathymetry(n, 3001, smooth=smooth)
    x, y = cell_centres(n, n, dx, dx)
    rng = np.random.default_rng(3002)
    deep = np.argwhere(b < -3000.0)
    j, i = deep[rng.integers(len(deep))]
    cx, cy = x[j, i], y[j, i]
    if crop is not None:
        # a crop of size crop x crop centred on the source (kept inside the grid)
        i0 = int(min(max(i - crop // 2, 0), n - crop))
        j0 = int(min(max(j - crop // 2, 0), n - crop))
        b = b[j0:j0 + crop, i0:i0 + crop]
        x = x[j0:j0 + crop, i0:i0 + crop]
        y = y[j0:j0 + crop, i0:i0 + crop]
        xo, yo = i0 * dx, j0 * dx
    else:
        xo, yo = 0.0, 0.0
    r2 = (x - cx) ** 2 + (y - cy) ** 2
    q = np.zeros((NVAR[model],) + b.shape)
    q[0] = apply_surface(b, 2.0 * np.exp(-r2 / 30000.0 ** 2))
    grng = np.random.default_rng(3003)
    jj, ii = np.nonzero((q[0] - b) > 1.0)
    pick = grng.choice(len(ii), size=min(ngauges, len(ii)), replace=False)
    gxy = np.stack([x[jj[pick], ii[pick]], y[jj[pick], ii[pick]]], axis=1)
    return dict(b=b, q=q, dx=dx, dy=dx, x0=xo, y0=yo, bc=(1, 1, 1, 1), model=model,
                alpha=3.0, h_star=20.0, cfl=0.9, steps=2000, dry_tol=1e-3, gauges=gxy,
                source=(cx, cy))


# --------------------------------------------------------------------------
# Small seeded cases used by the parity tests.
def smooth_random_bathymetry(nx, ny, seed, lo=-2.0, hi=0.6, modes=4):
    """Smooth random bathymetry crossing the still level (wet/dry shoreline)."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    f = np.zeros_like(X)
    for _ in range(modes):
        kx, ky = rng.integers(1, 4, size=2)
        ph = rng.uniform(0, 2 * np.pi, size=2)
        f += rng.uniform(0.3, 1.0) * np.cos(np.pi * kx * X + ph[0]) * np.cos(np.pi * ky * Y + ph[1])
    f = (f - f.min()) / (f.max() - f.min() + 1e-300)
    return lo + (hi - lo) * f


def gaussian_hump_state(model, b, x, y, xc, yc, amp, radius):
    q = np.zeros((NVAR[model],) + b.shape)
    q[0] = apply_surface(b, amp * np.exp(-((x - xc) ** 2 + (y - yc) ** 2) / radius ** 2))
    return q


def random_small_case(model, nx, ny, seed, dx=0.1, wetdry=True, amp=0.2):
    """A seeded small case: smooth random bathymetry (crossing the still level when
    wetdry), a Gaussian hump plus random small velocities and auxiliaries."""
    rng = np.random.default_rng(seed)
    x, y = cell_centres(nx, ny, dx, dx)
    if wetdry:
        b = smooth_random_bathymetry(nx, ny, seed + 1)
    else:
        b = -1.0 - 0.3 * smooth_random_bathymetry(nx, ny, seed + 1, 0.0, 1.0)
    xc, yc = rng.uniform(0.3, 0.7) * nx * dx, rng.uniform(0.3, 0.7) * ny * dx
    q = gaussian_hump_state(model, b, x, y, xc, yc, amp, 0.2 * min(nx, ny) * dx)
    h = q[0] - b
    wet = h > 1e-3
    q[1] = np.where(wet, h * rng.uniform(-0.2, 0.2) * np.sin(x), 0.0)
    q[2] = np.where(wet, h * rng.uniform(-0.2, 0.2) * np.cos(y), 0.0)
    fi = field_index(model)
    if fi["hw"] is not None:
        q[fi["hw"]] = np.where(wet, h * 0.01 * np.sin(2 * x + y), 0.0)
        q[fi["hp"]] = np.where(wet, h * 0.05 * np.cos(x - 2 * y), 0.0)
    if fi["hs"] is not None:
        q[fi["hs"]] = np.where(wet, h * 0.02 * np.cos(x + y), 0.0)
        q[fi["hpb"]] = np.where(wet, h * 0.03 * np.sin(x * y), 0.0)
    return b, q


def amr_small_case(model, nx0, ny0, r, nlevels, seed, dx0=0.2, wetdry=True, amp=0.2):
    """Seeded input of a small refined hierarchy: random_small_case on the finest
    grid (nx0 r^(L-1) x ny0 r^(L-1), spacing dx0 / r^(L-1)) and, for every level,
    the state on that level's full grid as r x r block means of the next finer
    one.  Returns (b_finest, [q_0, ..., q_{L-1}])."""
    R = r ** (nlevels - 1)
    b, q = random_small_case(model, nx0 * R, ny0 * R, seed, dx=dx0 / R, wetdry=wetdry, amp=amp)
    qs = [q]
    for _ in range(nlevels - 1):
        f = qs[0]
        nv, ny, nx = f.shape
        qs.insert(0, f.reshape(nv, ny // r, r, nx // r, r).mean(axis=(2, 4)))
    return b, qs


def amr_boxes_small():
    """A three-level hierarchy (ratio 2) over a 24 x 20 level-0 grid: two level-1
    patches sharing a face plus a third one touching the domain boundary, and a
    level-2 patch in each of the first two (boxes in each level's cell indices)."""
    lvl1 = [(8, 8, 16, 12), (24, 8, 8, 12), (0, 28, 12, 12)]
    lvl2 = [(20, 20, 16, 12), (52, 20, 8, 8)]
    return [lvl1, lvl2]


def amr_boxes_small_moved():
    """A second layout over the grid of amr_boxes_small (for regridding): one
    level-1 patch kept, one reshaped, one moved away from the boundary; a
    level-2 patch shifted half over its old place and one in the moved patch."""
    lvl1 = [(8, 8, 16, 12), (24, 12, 8, 8), (28, 24, 12, 12)]
    lvl2 = [(24, 20, 16, 12), (60, 52, 12, 16)]
    return [lvl1, lvl2]


# --------------------------------------------------------------------------
# Config 4: three refinement levels, ratio 4, level 0 1024 x 1024 at 2 km over
# a fractal bathymetry with a sloping coast strip; patches of seeded sizes
# 16..128 cells (multiples of 8) along the advancing front of a ring wave.
def config4_bathymetry(n0=1024, r=4, levels=3, seed=4001, depth=6000.0):
    """Finest-level bathymetry (n0 r^(L-1))^2: a fractal field (|k|^-2, seed
    4001) on a 4x coarser grid, low-pass filtered (Gaussian, 4 cells of that
    grid: the level-0 spacing, so that level 0 resolves the coasts), bilinearly
    refined, plus a coast strip rising 1:100 to at most +50 m over the last 8 %
    of the domain in x."""
    from scipy.ndimage import gaussian_filter
    R = r ** (levels - 1)
    nf = n0 * R
    nb = nf // 4
    base = gaussian_filter(fractal_bathymetry(nb, seed, depth=depth, land_frac=0.1), 4.0, mode="nearest")
    t = (np.arange(nf) + 0.5) / 4.0 - 0.5
    i0 = np.clip(np.floor(t).astype(np.int64), 0, nb - 2)
    w = np.clip(t - i0, 0.0, 1.0)
    rows = base[i0] * (1.0 - w)[:, None] + base[i0 + 1] * w[:, None]
    b = rows[:, i0] * (1.0 - w)[None, :] + rows[:, i0 + 1] * w[None, :]
    del rows
    dxf = 2000.0 / R
    x = (np.arange(nf) + 0.5) * dxf
    xc = 0.92 * nf * dxf
    b += np.where(x > xc, (x - xc) / 100.0, 0.0)[None, :]
    np.minimum(b, 50.0, out=b)
    return b


def _seeded_cuts(rng, a0, a1, sizes):
    """Cut [a0, a1) into consecutive lengths drawn from `sizes`; the last piece
    takes the remainder (split in two if it would exceed the largest size)."""
    cuts, x = [], a0
    lo, hi = min(sizes), max(sizes)
    while x < a1:
        w = int(rng.choice(sizes))
        if a1 - (x + w) < lo:
            w = a1 - x
            if w > hi:
                h1 = (w // 2) // 8 * 8
                cuts.append((x, h1))
                x, w = x + h1, w - h1
        cuts.append((x, w))
        x += w
    return cuts


def config4_boxes(n0=1024, r=4, levels=3, seed=4001, centre=(0.45, 0.5), radius=300e3, width=70e3, dx0=2000.0,
                  sizes=tuple(range(16, 129, 8))):
    """Patches along the front of a ring wave (radius 300 km, a flagged band
    70 km wide around it: the |d eta| flag of an expanding ring).  The region a
    level may refine (the whole grid for level 1; each level-1 box two level-1
    cells inside its edges for level 2) is cut into rows and columns of seeded
    sizes 16..128 cells (multiples of 8); every tile holding a flagged cell
    becomes a box.  Returns [level-1 boxes, level-2 boxes]."""
    rng = np.random.default_rng(seed)
    cx, cy = centre[0] * n0 * dx0, centre[1] * n0 * dx0

    def flagged(level, X, Y):
        d = dx0 / r ** level
        rr = np.hypot((X + 0.5) * d - cx, (Y + 0.5) * d - cy)
        return np.abs(rr - radius) < 0.5 * width

    out = []
    parents = [(0, 0, n0, n0)]
    for level in range(1, levels):
        Np = n0 * r ** (level - 1)
        boxes = []
        for (pi0, pj0, pnx, pny) in parents:
            m0 = 0 if level == 1 else 2 * r
            a0 = pi0 * r + (0 if pi0 == 0 else m0)
            a1 = (pi0 + pnx) * r - (0 if pi0 + pnx == Np else m0)
            b0 = pj0 * r + (0 if pj0 == 0 else m0)
            b1 = (pj0 + pny) * r - (0 if pj0 + pny == Np else m0)
            a0, b0 = (a0 + 7) // 8 * 8, (b0 + 7) // 8 * 8
            a1, b1 = a1 // 8 * 8, b1 // 8 * 8
            if a1 - a0 < min(sizes) or b1 - b0 < min(sizes):
                continue
            for (j0, h) in _seeded_cuts(rng, b0, b1, sizes):
                for (i0, w) in _seeded_cuts(rng, a0, a1, sizes):
                    ys, xs = np.mgrid[j0:j0 + h:8, i0:i0 + w:8]
                    if flagged(level, xs + 4, ys + 4).any():
                        boxes.append((int(i0), int(j0), int(w), int(h)))
        out.append(boxes)
        parents = boxes
    return out


def config4(model=HSGN, n0=1024, r=4, levels=3, amp=2.0, radius=30e3, centre=(0.45, 0.5), boxes=None):
    """Config 4 input: finest bathymetry, boxes, and the initial state of every
    patch (Gaussian uplift of 2 m, radius 30 km, at the ring centre, over the
    ocean only), states[level][patch] of shape (nvar, ny, nx)."""
    dx0 = 2000.0
    b = config4_bathymetry(n0, r, levels)
    if boxes is None:
        boxes = config4_boxes(n0, r, levels, centre=centre, dx0=dx0)
    cx, cy = centre[0] * n0 * dx0, centre[1] * n0 * dx0
    allboxes = [[(0, 0, n0, n0)]] + boxes
    R = r ** (levels - 1)
    states = []
    for level, bxs in enumerate(allboxes):
        d = dx0 / r ** level
        f = r ** (levels - 1 - level)      # finest cells per cell of this level
        lv = []
        for (i0, j0, nx, ny) in bxs:
            blk = b[j0 * f:(j0 + ny) * f, i0 * f:(i0 + nx) * f]
            bb = blk.reshape(ny, f, nx, f).mean(axis=(1, 3)) if f > 1 else blk
            x = (np.arange(i0, i0 + nx) + 0.5) * d
            y = (np.arange(j0, j0 + ny) + 0.5) * d
            rr2 = (x[None, :] - cx) ** 2 + (y[:, None] - cy) ** 2
            q = np.zeros((NVAR[model], ny, nx))
            q[0] = apply_surface(bb, amp * np.exp(-rr2 / radius ** 2))
            lv.append(q)
        states.append(lv)
    del R
    return dict(b=b, boxes=boxes, states=states, n0=n0, r=r, dx0=dx0, bc=(1, 1, 1, 1), model=model,
                alpha=3.0, h_star=20.0, cfl=0.9, dry_tol=1e-2)
