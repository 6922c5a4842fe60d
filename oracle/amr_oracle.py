"""Plain block-structured refinement (Berger-Oliger-Colella, as the paper runs
the method in GeoClaw: patches, refinement ratio r, subcycling in time, Sec. 4)
around the oracle's patch step.

TEST INFRASTRUCTURE ONLY: like the rest of oracle/, used by tests/ to check the
batched CUDA hierarchy; it shares no code with it.  Pure-Python loops over the
ghost cells, registers and covered cells: small hierarchies only.

The paper relies on GeoClaw's refinement without restating it; the definitions
below are the readings the CUDA hierarchy implements as well.

 A1 Hierarchy.  Level 0 is one patch covering the nx0 x ny0 grid (spacing dx0);
    level l >= 1 holds disjoint boxes (i0, j0, nx, ny) in level-l cell indices
    (spacing dx0 / r^l), aligned to whole parent cells, each inside a single
    level-(l-1) patch and at least two parent cells from its edges except along
    the domain boundary.  Every patch has a frame of two ghost layers.
 A2 Bathymetry of the finest level is given; a coarser level's cell is the mean
    of its r x r children (summed row by row, divided by r^2).  phi_T of a level
    follows the uniform-grid rule on that level's full grid; frames take b and
    phi_T of their cell, or of the cell the boundary condition maps them to.
 A3 Ghost cells of a level-l patch, level-l cell (X, Y): outside the domain, the
    boundary condition maps them into the patch's own frame (wall: mirror with
    negated normal momentum; extrapolation: copy), filled after the others;
    inside another patch of the level: copy of its cell; otherwise
    interpolation from the parent at time weight a (A4).
 A4 Interpolation: each coarse value is first interpolated in time,
    (1 - a) q_old + a q_new; if the coarse cell is dry the ghost cell is at
    rest (eta = max(its own b, 0), the still level; all else 0), so that a
    sub-cell below the still level inside a dry coarse cell does not drain the
    fine patch; otherwise the surface eta and the primitives (u, v, w, sigma,
    p, p_b) are each the coarse value plus minmod-limited slopes times the
    sub-cell offset ((s + 1/2)/r - 1/2 in coarse cells), a one-sided difference
    counting only towards a wet coarse neighbour inside the domain (else that
    slope is 0); eta is raised to the ghost cell's own b where it falls below
    it, and each conserved field is the ghost depth times its primitive (zero
    when that depth is at most dry_tol), bounded in magnitude by the coarse
    cell's own conserved value (time-interpolated) and set to zero where the two
    differ in sign.  Interpolating velocities keeps a thin interpolated layer
    from getting a large velocity; the bound keeps a deep sub-cell of a coarse
    cell that is mostly dry (small mean depth, unreliable velocity) from getting
    a large momentum.
 A5 Subcycling: a level-l step of dt_l is followed by r steps of dt_l / r of
    level l + 1 at time weights k / r, k = 0..r-1, then average-down and reflux.
 A6 Positivity factors of ghost cells copied from a patch of the same level are
    taken from that patch (so both sides of a shared face move the same mass);
    all other ghost cells keep 1.
 A7 Reflux of mass: at each coarse face between a cell covered by a finer patch
    and an uncovered one, the uncovered cell's surface is corrected by the
    difference between the coarse mass flux and the fine mass fluxes through the
    same face summed over the fine faces and substeps (all corrections of a
    cell summed first).  Where that would leave a negative depth (a cell
    drying next to a finer patch whose interpolated ghost cells carry no
    positivity factor) the depth is set to zero and the water this adds is
    counted in `clipped`, so mass + 0 = initial mass + clipped exactly.  The
    other rows are not refluxed (the relaxed systems are not in conservation
    form).
 A8 Average-down: every field of a covered coarse cell becomes the mean of its
    r x r children (as in A2).
 A10 A coarse cell that is partly dry holds the mean depth of its children
    after average-down, which exceeds the coarse rest depth max(-b_c, 0): the
    lake at rest is exact when no such cell borders an uncovered cell (mass is
    exact in every case).
 A9 Time step: dt_0 = min over levels of CFL r^l / smax_l, smax_l the largest
    cell speed over the interior cells of level l after each of its steps since
    the previous level-0 step (dt_l = dt_0 / r^l).
 A11 Regridding: new boxes for levels 1..L-1 (same rules as A1).  Level 0 is
    kept; coarse to fine, each interior cell of a new patch takes the value of
    the old patch of its level that covered it, else the A4 interpolation from
    its new parent at the current time (weight 0, old = new state); then every
    level is averaged down (A8), finest first.  Time and clipped water carry
    over; the next step is recomputed from the new states.
 A12 Boxes from flags (Sec. 6.3: refine where the surface jump between
    neighbouring cells exceeds a threshold): level by level from the coarsest,
    a wet cell (h > dry_tol) is flagged where |eta - eta_n| > tol for a wet
    neighbour n in the same patch interior (a dry cell has no free surface:
    its eta is the bathymetry, and its jumps to land or to the shore are not
    waves); where the level has no patch the cell takes its parent
    cell's flag; flags are widened by `buffer` cells (a square); the part of
    each new box of the level that may hold finer patches (two cells inside
    its edges except along the domain boundary) is cut into tile x tile
    squares from its low corner (tile >= 2), the last ones clipped and a
    one-cell remainder merged into the square before it, and every square
    holding a widened flag becomes a box of the next level.
"""
import numpy as np

from . import oracle as O

NG = 2


def block_mean(a, r):
    """Mean of each r x r block, summed in row order then divided by r^2 (A2)."""
    ny, nx = a.shape
    s = np.zeros((ny // r, nx // r))
    for dj in range(r):
        for di in range(r):
            s = s + a[dj::r, di::r]
    return s / (r * r)


def bc_map(X, N, lo, hi):
    """Boundary-condition map of a level index (wall: mirror and flip; extrapolation: clamp)."""
    if X < 0:
        return (-X - 1, True) if lo == O.WALL else (0, False)
    if X >= N:
        return (2 * N - 1 - X, True) if hi == O.WALL else (N - 1, False)
    return X, False


def _cuts(a0, a1, tile):
    """A12: [a0, a1) cut into pieces of `tile` cells from a0; a last piece of one
    cell is merged into the one before it, so that no piece ends one cell short
    of a1 (a box one parent cell from its parent's edge breaks A1 when that edge
    is the domain boundary)."""
    out, x = [], a0
    while x < a1:
        w = min(tile, a1 - x)
        if a1 - (x + w) == 1:
            w += 1
        out.append((x, w))
        x += w
    return out


def minmod(a, b):
    if a * b <= 0.0:
        return 0.0
    return a if abs(a) < abs(b) else b


class AmrOracle:
    """boxes: for levels 1..L-1, lists of (i0, j0, nx, ny) in that level's cells.
    b_fine: bathymetry of the finest level, (ny0 r^(L-1), nx0 r^(L-1))."""

    def __init__(self, b_fine, nx0, ny0, dx0, r, boxes, model=O.HSGN, bc=(O.WALL,) * 4, **cfg):
        if any(v == O.PERIODIC for v in bc):
            raise ValueError("periodic boundaries are not supported with refinement")
        self.L = len(boxes) + 1
        self.r, self.model, self.bc = r, model, tuple(bc)
        self.nv = O.NVAR[model]
        self.cfg = dict(cfg)
        self.cfl = cfg.get("cfl", 0.9)
        self.dry_tol = cfg.get("dry_tol", 1e-3)
        self.alpha = cfg.get("alpha", 3.0)
        self.g = cfg.get("g", 9.81)
        L = self.L
        self.dims = [(nx0 * r ** l, ny0 * r ** l) for l in range(L)]
        self.dx = [dx0 / r ** l for l in range(L)]
        b_fine = np.asarray(b_fine, dtype=np.float64)
        assert b_fine.shape == (self.dims[-1][1], self.dims[-1][0])
        self.b = [None] * L
        self.b[L - 1] = b_fine.copy()
        for l in range(L - 2, -1, -1):
            self.b[l] = block_mean(self.b[l + 1], r)
        self.phi = []
        for l in range(L):
            o = O.Oracle(self.b[l], dx=self.dx[l], bc=bc, model=model, **cfg)
            self.phi.append(o.aux()[1])
            del o
        allboxes = [[(0, 0, nx0, ny0)]] + [list(map(tuple, bl)) for bl in boxes]
        self.boxes = allboxes
        self._validate()
        self.levels = []
        for l, bl in enumerate(allboxes):
            pats = []
            for (i0, j0, nx, ny) in bl:
                bfr, pfr = self._frame_aux(l, i0, j0, nx, ny)
                P = O.Patch(bfr, pfr, dx=self.dx[l], model=model, **cfg)
                H = np.maximum(-bfr, 0.0)
                c2 = self.alpha * self.alpha * self.g * H * pfr
                q = np.zeros((self.nv, ny + 2 * NG, nx + 2 * NG))
                q[0] = np.maximum(bfr, 0.0)
                pats.append(dict(box=(i0, j0, nx, ny), P=P, b=bfr, c2=c2, q=q, q_old=None,
                                 parent=self._parent(l, i0, j0, nx, ny) if l else None))
            self.levels.append(pats)
        self._build_ghosts()
        self._build_registers()
        self.t = 0.0
        self.status = 0
        self.smax = [0.0] * L
        self.dt_next = 0.0

    # ---- structure -------------------------------------------------------
    def _parent(self, l, i0, j0, nx, ny):
        r = self.r
        for pi, (pi0, pj0, pnx, pny) in enumerate(self.boxes[l - 1]):
            if pi0 <= i0 // r and (i0 + nx) // r <= pi0 + pnx and pj0 <= j0 // r and (j0 + ny) // r <= pj0 + pny:
                return pi
        return None

    def _validate(self):
        r = self.r
        for l in range(1, self.L):
            NXp, NYp = self.dims[l - 1]
            for bi, (i0, j0, nx, ny) in enumerate(self.boxes[l]):
                if min(i0, j0) < 0 or i0 + nx > self.dims[l][0] or j0 + ny > self.dims[l][1]:
                    raise ValueError("box outside the domain")
                if i0 % r or j0 % r or nx % r or ny % r or nx < 2 or ny < 2:
                    raise ValueError("box not aligned to parent cells")
                pi = self._parent(l, i0, j0, nx, ny)
                if pi is None:
                    raise ValueError("box not inside a single parent patch")
                pi0, pj0, pnx, pny = self.boxes[l - 1][pi]
                c0, c1, d0, d1 = i0 // r, (i0 + nx) // r, j0 // r, (j0 + ny) // r
                for gap, edge in ((c0 - pi0, c0 == 0), (pi0 + pnx - c1, c1 == NXp),
                                  (d0 - pj0, d0 == 0), (pj0 + pny - d1, d1 == NYp)):
                    if gap < 2 and not edge:
                        raise ValueError("box closer than two parent cells to its parent's edge")
                for bj, (k0, m0, kx, ky) in enumerate(self.boxes[l]):
                    if bj != bi and i0 < k0 + kx and k0 < i0 + nx and j0 < m0 + ky and m0 < j0 + ny:
                        raise ValueError("overlapping boxes")

    def _frame_aux(self, l, i0, j0, nx, ny):
        NX, NY = self.dims[l]
        bfr = np.empty((ny + 2 * NG, nx + 2 * NG))
        pfr = np.empty((ny + 2 * NG, nx + 2 * NG), dtype=np.uint8)
        for J in range(ny + 2 * NG):
            Ys, _ = bc_map(j0 - NG + J, NY, self.bc[2], self.bc[3])
            for I in range(nx + 2 * NG):
                Xs, _ = bc_map(i0 - NG + I, NX, self.bc[0], self.bc[1])
                bfr[J, I] = self.b[l][Ys, Xs]
                pfr[J, I] = self.phi[l][Ys, Xs]
        return bfr, pfr

    def _owner(self, l, X, Y, skip):
        for k, (i0, j0, nx, ny) in enumerate(self.boxes[l]):
            if k != skip and i0 <= X < i0 + nx and j0 <= Y < j0 + ny:
                return k
        return None

    def _build_ghosts(self):
        r = self.r
        for l, pats in enumerate(self.levels):
            NX, NY = self.dims[l]
            for pi, p in enumerate(pats):
                i0, j0, nx, ny = p["box"]
                sib, par, bcs = [], [], []
                for J in range(ny + 2 * NG):
                    for I in range(nx + 2 * NG):
                        if NG <= I < nx + NG and NG <= J < ny + NG:
                            continue
                        X, Y = i0 - NG + I, j0 - NG + J
                        if not (0 <= X < NX and 0 <= Y < NY):
                            Xs, fx = bc_map(X, NX, self.bc[0], self.bc[1])
                            Ys, fy = bc_map(Y, NY, self.bc[2], self.bc[3])
                            Is, Js = Xs - i0 + NG, Ys - j0 + NG
                            assert 0 <= Is < nx + 2 * NG and 0 <= Js < ny + 2 * NG
                            bcs.append((J, I, Js, Is, fx, fy))
                            continue
                        k = self._owner(l, X, Y, pi)
                        if k is not None:
                            k0, m0 = self.boxes[l][k][:2]
                            sib.append((J, I, k, Y - m0 + NG, X - k0 + NG))
                            continue
                        assert l > 0
                        P = self.boxes[l - 1][p["parent"]]
                        ic, jc = X // r, Y // r
                        nb = (ic - 1 >= 0, ic + 1 < self.dims[l - 1][0], jc - 1 >= 0, jc + 1 < self.dims[l - 1][1])
                        Ip, Jp = ic - P[0] + NG, jc - P[1] + NG
                        for ok, (a, b) in zip(nb, ((-1, 0), (1, 0), (0, -1), (0, 1))):
                            if ok:
                                assert NG <= Ip + a < P[2] + NG and NG <= Jp + b < P[3] + NG
                        par.append((J, I, Jp, Ip, X % r, Y % r, nb))
                p["sib"], p["par"], p["bc"] = sib, par, bcs

    def _build_registers(self):
        """Reflux registers (A7): one per coarse face between a covered and an
        uncovered coarse cell."""
        r = self.r
        self.regs = [[] for _ in range(self.L)]
        self.cover = []
        for l, pats in enumerate(self.levels):
            cov = []
            for p in pats:
                i0, j0, nx, ny = p["box"]
                m = np.zeros((ny, nx), dtype=bool)
                if l + 1 < self.L:
                    for (k0, m0, kx, ky) in self.boxes[l + 1]:
                        a0, a1 = max(k0 // r, i0), min((k0 + kx) // r, i0 + nx)
                        b0, b1 = max(m0 // r, j0), min((m0 + ky) // r, j0 + ny)
                        if a0 < a1 and b0 < b1:
                            m[b0 - j0:b1 - j0, a0 - i0:a1 - i0] = True
                cov.append(m)
            self.cover.append(cov)
        for l in range(self.L - 1):
            NX, NY = self.dims[l]

            def covered(X, Y):
                return any(k0 // r <= X < (k0 + kx) // r and m0 // r <= Y < (m0 + ky) // r
                           for (k0, m0, kx, ky) in self.boxes[l + 1])

            for ci, c in enumerate(self.levels[l + 1]):
                k0, m0, kx, ky = c["box"]
                pi = c["parent"]
                P0, P1 = self.boxes[l][pi][:2]
                c0, d0, cw, ch = k0 // r, m0 // r, kx // r, ky // r
                cand = []
                for jc in range(d0, d0 + ch):
                    cand.append((0, c0 - 1, jc, c0, jc, +1, 0, (jc - d0) * r))      # left edge
                    cand.append((0, c0 + cw, jc, c0 + cw, jc, -1, kx, (jc - d0) * r))  # right edge
                for ic in range(c0, c0 + cw):
                    cand.append((1, ic, d0 - 1, ic, d0, +1, 0, (ic - c0) * r))      # bottom edge
                    cand.append((1, ic, d0 + ch, ic, d0 + ch, -1, ky, (ic - c0) * r))  # top edge
                for (d, ux, uy, fx, fy, s, fpos, f0) in cand:
                    if not (0 <= ux < NX and 0 <= uy < NY) or covered(ux, uy):
                        continue
                    # coarse face (fx, fy) in the parent's face_mass indexing, the
                    # uncovered cell in its frame, the r fine faces of the child
                    self.regs[l].append(dict(parent=pi, dir=d, face=(fy - P1, fx - P0), cell=(uy - P1 + NG, ux - P0 + NG),
                                             sign=s, child=ci, fine=(fpos, f0), val=0.0))

    # ---- state ----------------------------------------------------------
    def _switch(self, p, q):
        """SWE / dry switch of Sec. 3.3 on the interior of a patch frame."""
        h = np.maximum(q[0] - p["b"], 0.0)
        wet = h > self.dry_tol
        sl = (slice(NG, -NG), slice(NG, -NG))
        for k in range(1, self.nv):
            q[k][sl] = np.where(wet[sl], q[k][sl], 0.0)
        for k in range(3, self.nv):
            q[k][sl] = np.where(p["c2"][sl] > 0.0, q[k][sl], 0.0)

    def set_state(self, qs, t=0.0):
        """qs[l]: dense (nvar, NY_l, NX_l) state of level l (only the patch
        interiors are read); the switch is applied."""
        for l, pats in enumerate(self.levels):
            for p in pats:
                i0, j0, nx, ny = p["box"]
                p["q"][:, NG:NG + ny, NG:NG + nx] = qs[l][:, j0:j0 + ny, i0:i0 + nx]
                self._switch(p, p["q"])
        self.t = t
        self.status = 0
        self.clipped = 0.0
        self.smax = [0.0] * self.L
        for l, pats in enumerate(self.levels):
            for p in pats:
                p["P"].set_frame(p["q"], t)
                self.smax[l] = max(self.smax[l], p["P"].max_speed())
        self.dt_next = self._dt_from_smax()

    def patch_state(self, l, k):
        i0, j0, nx, ny = self.levels[l][k]["box"]
        return self.levels[l][k]["q"][:, NG:NG + ny, NG:NG + nx].copy()

    def _dt_from_smax(self):
        best = None
        for l in range(self.L):
            if self.smax[l] > 0.0:
                d = self.cfl * float(self.r ** l) / self.smax[l]
                best = d if best is None or d < best else best
        return 0.0 if best is None else best

    def mass(self):
        m = 0.0
        for l, pats in enumerate(self.levels):
            for k, p in enumerate(pats):
                i0, j0, nx, ny = p["box"]
                h = np.maximum(p["q"][0, NG:NG + ny, NG:NG + nx] - p["b"][NG:NG + ny, NG:NG + nx], 0.0)
                m += float(np.sum(h[~self.cover[l][k]])) * self.dx[l] * self.dx[l]
        return m

    # ---- ghost cells (A3, A4) ----------------------------------------------
    def _interp(self, bf, qo, qn, bp, Jp, Ip, sx, sy, nb, a):
        """A4: value of the fine cell (bathymetry bf, sub-cell offsets sx, sy)
        in coarse cell (Jp, Ip) of a parent frame with old / new states qo /
        qn and bathymetry bp, at time weight a; nb: in-domain flags W E S N."""
        r = self.r

        def prim(dj, di):
            vv = (1.0 - a) * qo[:, Jp + dj, Ip + di] + a * qn[:, Jp + dj, Ip + di]
            h = vv[0] - bp[Jp + dj, Ip + di]
            if not h > self.dry_tol:
                return None
            out = vv / h
            out[0] = vv[0]
            return out
        c = prim(0, 0)
        out = np.zeros(self.nv)
        if c is None:
            out[0] = max(bf, 0.0)
            return out
        side = {}
        for key, ok, (dj, di) in zip("WESN", nb, ((0, -1), (0, 1), (-1, 0), (1, 0))):
            side[key] = prim(dj, di) if ok else None
        xi, yi = (sx + 0.5) / r - 0.5, (sy + 0.5) / r - 0.5
        for f in range(self.nv):
            sxl = minmod(c[f] - side["W"][f], side["E"][f] - c[f]) \
                if side["W"] is not None and side["E"] is not None else 0.0
            syl = minmod(c[f] - side["S"][f], side["N"][f] - c[f]) \
                if side["S"] is not None and side["N"] is not None else 0.0
            out[f] = c[f] + xi * sxl + yi * syl
        out[0] = max(out[0], bf)
        hf = out[0] - bf
        cc = (1.0 - a) * qo[:, Jp, Ip] + a * qn[:, Jp, Ip]
        for f in range(1, self.nv):
            v = hf * out[f] if hf > self.dry_tol else 0.0
            # no larger than the coarse cell's own conserved value (A4)
            out[f] = (v if abs(v) <= abs(cc[f]) else cc[f]) if v * cc[f] > 0.0 else 0.0
        return out

    def _fill(self, l, a):
        pats = self.levels[l]
        r = self.r
        for p in pats:
            q = p["q"]
            for (J, I, k, Js, Is) in p["sib"]:
                q[:, J, I] = pats[k]["q"][:, Js, Is]
            if p["par"]:
                P = self.levels[l - 1][p["parent"]]
                for (J, I, Jp, Ip, sx, sy, nb) in p["par"]:
                    q[:, J, I] = self._interp(p["b"][J, I], P["q_old"], P["q"], P["b"], Jp, Ip, sx, sy, nb, a)
        for p in pats:
            q = p["q"]
            for (J, I, Js, Is, fx, fy) in p["bc"]:
                v = q[:, Js, Is].copy()
                if fx:
                    v[1] = -v[1]
                if fy:
                    v[2] = -v[2]
                q[:, J, I] = v

    # ---- stepping (A5-A9) ------------------------------------------------
    def _advance(self, l, dt, a):
        pats = self.levels[l]
        self._fill(l, a)
        for p in pats:
            p["q_old"] = p["q"].copy()
            p["P"].set_frame(p["q"], self.t)
            p["P"].step_begin(dt)
        th = [p["P"].get_theta() for p in pats]
        for k, p in enumerate(pats):
            tn = th[k].copy()
            for (J, I, s, Js, Is) in p["sib"]:
                tn[J, I] = th[s][Js, Is]
            p["P"].set_theta(tn)
        fm = [(p["P"].face_mass(0), p["P"].face_mass(1)) for p in pats]
        if l + 1 < self.L:
            for g in self.regs[l]:
                lam = dt / self.dx[l]
                g["val"] = g["sign"] * lam * fm[g["parent"]][g["dir"]][g["face"]]
        if l > 0:
            coef = (dt / self.dx[l]) / float(self.r * self.r)
            for g in self.regs[l - 1]:
                F = fm[g["child"]][g["dir"]]
                fpos, f0 = g["fine"]
                s = 0.0
                for m in range(self.r):
                    s += F[f0 + m, fpos] if g["dir"] == 0 else F[fpos, f0 + m]
                g["val"] -= g["sign"] * coef * s
        for p in pats:
            if p["P"].step_end(dt):
                self.status |= p["P"].status
            p["q"] = p["P"].get_frame()
            self.smax[l] = max(self.smax[l], p["P"].max_speed())
        if l + 1 < self.L:
            for k in range(self.r):
                self._advance(l + 1, dt / self.r, k / self.r)
            self._average_down(l)
            corr = {}
            for g in self.regs[l]:
                key = (g["parent"], g["cell"])
                corr[key] = corr.get(key, 0.0) + g["val"]
            for (pi, cell), v in corr.items():
                P = self.levels[l][pi]
                e = P["q"][0][cell] + v
                if e < P["b"][cell]:
                    self.clipped += (P["b"][cell] - e) * self.dx[l] * self.dx[l]
                    e = P["b"][cell]
                P["q"][0][cell] = e

    def _average_down(self, l):
        r = self.r
        for c in self.levels[l + 1]:
            k0, m0, kx, ky = c["box"]
            P = self.levels[l][c["parent"]]
            P0, P1 = P["box"][:2]
            fine = c["q"][:, NG:NG + ky, NG:NG + kx]
            for f in range(self.nv):
                P["q"][f, m0 // r - P1 + NG:(m0 + ky) // r - P1 + NG,
                       k0 // r - P0 + NG:(k0 + kx) // r - P0 + NG] = block_mean(fine[f], r)

    # ---- regridding (A11) --------------------------------------------------
    def regrid(self, boxes):
        """Replace the patches of levels 1..L-1 by `boxes` (as in the
        constructor) and carry the state over (A11)."""
        r = self.r
        new = AmrOracle(self.b[-1], self.dims[0][0], self.dims[0][1], self.dx[0], r, boxes, model=self.model,
                        bc=self.bc, **self.cfg)
        new.levels[0][0]["q"] = self.levels[0][0]["q"].copy()
        for l in range(1, self.L):
            for p in new.levels[l]:
                i0, j0, nx, ny = p["box"]
                P = new.levels[l - 1][p["parent"]]
                P0, P1 = P["box"][:2]
                for j in range(ny):
                    for i in range(nx):
                        X, Y = i0 + i, j0 + j
                        k = self._owner(l, X, Y, None)
                        if k is not None:
                            o = self.levels[l][k]
                            p["q"][:, NG + j, NG + i] = o["q"][:, Y - o["box"][1] + NG, X - o["box"][0] + NG]
                            continue
                        ic, jc = X // r, Y // r
                        nb = (ic - 1 >= 0, ic + 1 < new.dims[l - 1][0], jc - 1 >= 0, jc + 1 < new.dims[l - 1][1])
                        p["q"][:, NG + j, NG + i] = new._interp(p["b"][NG + j, NG + i], P["q"], P["q"], P["b"],
                                                                jc - P1 + NG, ic - P0 + NG, X % r, Y % r, nb, 0.0)
        for l in range(self.L - 2, -1, -1):
            new._average_down(l)
        new.t, new.clipped, new.status = self.t, self.clipped, 0
        new.smax = [0.0] * self.L
        for l, pats in enumerate(new.levels):
            for p in pats:
                p["P"].set_frame(p["q"], new.t)
                new.smax[l] = max(new.smax[l], p["P"].max_speed())
        new.dt_next = new._dt_from_smax()
        self.__dict__.update(new.__dict__)

    def flag_boxes(self, tol, tile, buffer):
        """A12: box lists of levels 1..L-1 from refinement flags of the
        current state."""
        if tile < 2:
            raise ValueError("tile must be at least 2 cells")
        r, out, prev = self.r, [], None
        parents = [self.boxes[0][0]]
        for l in range(self.L - 1):
            NX, NY = self.dims[l]
            f = np.zeros((NY, NX), dtype=bool)
            have = np.zeros((NY, NX), dtype=bool)
            for p in self.levels[l]:
                i0, j0, nx, ny = p["box"]
                e = p["q"][0, NG:NG + ny, NG:NG + nx]
                wt = (e - p["b"][NG:NG + ny, NG:NG + nx]) > self.dry_tol
                g = np.zeros((ny, nx), dtype=bool)
                jx = (np.abs(e[:, 1:] - e[:, :-1]) > tol) & wt[:, 1:] & wt[:, :-1]
                jy = (np.abs(e[1:, :] - e[:-1, :]) > tol) & wt[1:, :] & wt[:-1, :]
                g[:, 1:] |= jx
                g[:, :-1] |= jx
                g[1:, :] |= jy
                g[:-1, :] |= jy
                f[j0:j0 + ny, i0:i0 + nx] = g
                have[j0:j0 + ny, i0:i0 + nx] = True
            if l > 0:
                pro = np.repeat(np.repeat(prev, r, axis=0), r, axis=1)
                f = np.where(have, f, pro)
            w = np.zeros_like(f)
            for Y, X in zip(*np.nonzero(f)):
                w[max(0, Y - buffer):Y + buffer + 1, max(0, X - buffer):X + buffer + 1] = True
            bl = []
            for (i0, j0, nx, ny) in parents:
                x0, x1 = i0 + (0 if i0 == 0 else 2), i0 + nx - (0 if i0 + nx == NX else 2)
                y0, y1 = j0 + (0 if j0 == 0 else 2), j0 + ny - (0 if j0 + ny == NY else 2)
                for ty, th in _cuts(y0, y1, tile):
                    for tx, tw in _cuts(x0, x1, tile):
                        if w[ty:ty + th, tx:tx + tw].any():
                            bl.append((tx * r, ty * r, tw * r, th * r))
            out.append(bl)
            parents, prev = bl, f
        return out

    def step_dt(self, dt0):
        """One level-0 step of dt0 with all finer substeps; returns 0 or the status bits."""
        self.smax = [0.0] * self.L
        self._advance(0, dt0, 0.0)
        self.t += dt0
        self.dt_next = self._dt_from_smax()
        return self.status

    def step(self, n=1):
        for _ in range(n):
            if not self.dt_next > 0.0:
                self.status |= O.ST_ALLDRY
                return self.status
            if self.step_dt(self.dt_next):
                return self.status
        return self.status
