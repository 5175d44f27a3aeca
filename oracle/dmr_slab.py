"""Slab decomposition of the time step over several ranks: the uniform mesh
(SlabSim, local arrays) and the DMR step (DmrSlabSim, ghost zones).

TEST INFRASTRUCTURE ONLY (like dmr_oracle.py): the CPU reference of how the
method shards over processes, checked against the unsplit oracle.  Nothing on
the product path imports it.

The mesh (nx x ny cells, Sec. II.B) is cut along x into slabs of node
columns, one per rank of a torch.distributed process group (gloo on CPU).
Every element is updated by its owning rank with the oracle's own
arithmetic (Eqs. 1-4, Mur outer boundary), so the fields equal the unsplit
run's bit for bit.  Exchanged per EM step (Eqs. 1-3, Yee leapfrog):
  * after the H half-step: the Hz cell column next to the boundary, to the
    rank on the right (its Ey update reads Hz of the cell on its left);
  * after the E half-step: the Ey node column at the boundary, to the rank on
    the left (its last H cell reads Ey on its right), and the Ex cell column,
    to the rank on the right (the E^2 sum at its first node reads Ex on its
    left).
Per period (the continuity step, Eq. 4): the D_eff and density node columns
next to each boundary, both ways; the FP64 electron and absorbed-power
partial sums all-reduced (SUM; the order of the additions differs from the
unsplit sum, so totals agree within rounding); the refinement flags' bounding
box all-reduced (MIN / MAX) and their count (SUM) (Sec. III.A-III.B).
Ownership: rank k holds node columns [a_k, b_k) and cell columns [a_k, b_k)
clipped to the mesh; its arrays carry one halo column on each side.
"""
from __future__ import annotations

import numpy as np

from . import dmr_oracle as O


def slab_bounds(nx, world):
    """Node-column ranges [a, b) of the ranks; each holds at least two."""
    nodes = nx + 1
    if world < 1 or nodes < 2 * world:
        raise ValueError("too many ranks for %d node columns" % nodes)
    cuts = [(nodes * k) // world for k in range(world + 1)]
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


class SlabSim:
    """One rank's slab of a uniform (r = 1) run with a Mur outer boundary."""

    def __init__(self, cfg: dict, rank: int, world: int, comm):
        self.P = P = O.Params(cfg)
        if P.r != 1 or P.boundary != 0:
            raise ValueError("the slab reference covers uniform runs with the Mur boundary")
        self.rank, self.world, self.comm = rank, world, comm
        self.a, self.b = slab_bounds(P.nx, world)[rank]
        self.ga = max(self.a - 1, 0)                 # first local node column (halo)
        self.gb = min(self.b + 1, P.nx + 1)          # end of the local node columns
        # the global mesh's geometry, for the incident wave and weights
        self.full = O.Mesh(P, P.nx, P.ny, 1)
        self.dx, self.dt, self.N = self.full.dx, self.full.dt, self.full.N
        nn = self.gb - self.ga                       # local node columns
        nc = min(self.gb, P.nx) - self.ga            # local cell columns
        z = lambda a, c: np.zeros((a, c))
        self.Ex, self.vx = z(nc, P.ny + 1), z(nc, P.ny + 1)
        self.Ey, self.vy = z(nn, P.ny), z(nn, P.ny)
        self.Hz = z(nc, P.ny)
        self.n, self.S2 = z(nn, P.ny + 1), z(nn, P.ny + 1)
        self.erms_last = z(nn, P.ny + 1)
        self.m = 0
        self.N_e = self.P_abs = self.W_abs = 0.0
        self.bbox, self.nflag = None, 0

    # -- local index helpers: global column -> local index
    def c(self, i):
        return i - self.ga

    def seed_from(self, nmap):
        """Take the density of the global node map (x-major [i, j])."""
        self.n[...] = nmap[self.ga:self.gb, :]

    # -- halo exchange of one column ------------------------------------------
    def _send_recv(self, send_right, send_left):
        """Send a column to the right and/or left neighbour and receive the
        columns they send; returns (from_left, from_right)."""
        import torch
        import torch.distributed as dist
        ops, got = [], {}
        left, right = self.rank - 1, self.rank + 1
        if send_right is not None and right < self.world:
            ops.append(dist.P2POp(dist.isend, torch.from_numpy(np.ascontiguousarray(send_right)), right))
        if send_left is not None and left >= 0:
            ops.append(dist.P2POp(dist.isend, torch.from_numpy(np.ascontiguousarray(send_left)), left))
        if send_right is not None and left >= 0:
            got["left"] = torch.empty(send_right.shape, dtype=torch.float64)
            ops.append(dist.P2POp(dist.irecv, got["left"], left))
        if send_left is not None and right < self.world:
            got["right"] = torch.empty(send_left.shape, dtype=torch.float64)
            ops.append(dist.P2POp(dist.irecv, got["right"], right))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        return (got["left"].numpy() if "left" in got else None,
                got["right"].numpy() if "right" in got else None)

    # -- EM step (Eqs. 1-3) ----------------------------------------------------
    def em_step(self):
        P, dx, dt = self.P, self.dx, self.dt
        a, b, ga = self.a, self.b, self.ga
        Ex, Ey, Hz, vx, vy, n = self.Ex, self.Ey, self.Hz, self.vx, self.vy, self.n
        ca0, ca1 = a, min(b, P.nx)                   # owned cells
        s = slice(self.c(ca0), self.c(ca1))
        # Eq. 2 on the owned cells (Ey of the node on the right: local or halo)
        Hz[s] -= (dt / O.MU0) * ((Ey[self.c(ca0) + 1:self.c(ca1) + 1, :] - Ey[s, :]) / dx
                                 - (Ex[s, 1:] - Ex[s, :-1]) / dx)
        # the cell left of the slab (for the Ey update of node a)
        from_left, _ = self._send_recv(Hz[self.c(ca1) - 1, :] if ca1 > ca0 else None, None)
        if from_left is not None:
            Hz[self.c(a - 1), :] = from_left
        # Eq. 3 on the owned edges (total field)
        einc = P.E0 * np.sin(2.0 * np.pi * (self.m % self.N) / self.N - P.k * self.full.node_x())
        half = 0.5 * P.nu_m * dt
        vx[s] = ((1.0 - half) * vx[s] - (O.QE * dt / O.ME) * Ex[s]) / (1.0 + half)
        sn = slice(self.c(a), self.c(b))
        vy[sn] = ((1.0 - half) * vy[sn] - (O.QE * dt / O.ME) * (Ey[sn] + einc[a:b, None])) / (1.0 + half)
        Jx = -O.QE * (0.5 * (n[self.c(ca0):self.c(ca1), :] + n[self.c(ca0) + 1:self.c(ca1) + 1, :])) * vx[s]
        Jy = -O.QE * (0.5 * (n[sn, :-1] + n[sn, 1:])) * vy[sn]
        Ex_old, Ey_old = Ex.copy(), Ey.copy()
        # Eq. 1 on the owned interior edges
        Ex[s, 1:-1] += (dt / O.EPS0) * ((Hz[s, 1:] - Hz[s, :-1]) / dx - Jx[:, 1:-1])
        i0, i1 = max(a, 1), min(b, P.nx)             # owned interior Ey columns
        if i1 > i0:
            li = slice(self.c(i0), self.c(i1))
            Ey[li, :] += (dt / O.EPS0) * (-(Hz[li, :] - Hz[self.c(i0) - 1:self.c(i1) - 1, :]) / dx
                                          - Jy[i0 - a:i1 - a, :])
        # first-order Mur on the domain sides the slab touches
        coef = (O.C0 * dt - dx) / (O.C0 * dt + dx)
        if a == 0:
            Ey[0, :] = Ey_old[1, :] + coef * (Ey[1, :] - Ey_old[0, :])
        if b == P.nx + 1:
            Ey[self.c(P.nx), :] = Ey_old[self.c(P.nx) - 1, :] + coef * (Ey[self.c(P.nx) - 1, :] - Ey_old[self.c(P.nx), :])
        Ex[s, 0] = Ex_old[s, 1] + coef * (Ex[s, 1] - Ex_old[s, 0])
        Ex[s, -1] = Ex_old[s, -2] + coef * (Ex[s, -2] - Ex_old[s, -1])
        # Ey of the first owned node to the left, Ex of the last owned cell to the right
        _, ey_right = self._send_recv(None, Ey[self.c(a), :])
        if ey_right is not None:
            Ey[self.c(b), :] = ey_right
        ex_left, _ = self._send_recv(Ex[self.c(ca1) - 1, :] if ca1 > ca0 else None, None)
        if ex_left is not None:
            Ex[self.c(a - 1), :] = ex_left
        self.m += 1

    def accumulate_e2(self):
        """The E^2 sample of the present level at the owned nodes (the
        oracle's node average, total field)."""
        P = self.P
        a, b = self.a, self.b
        ex2 = self.Ex * self.Ex
        einc = P.E0 * np.sin(2.0 * np.pi * (self.m % self.N) / self.N - P.k * self.full.node_x())
        eyt = self.Ey + einc[self.ga:self.gb, None]
        ey2 = eyt * eyt
        for i in range(a, b):
            li = self.c(i)
            if 0 < i < P.nx:
                sx = 0.5 * (ex2[li - 1, :] + ex2[li, :])
            elif i == 0:
                sx = ex2[li, :]
            else:
                sx = ex2[li - 1, :]
            sy = np.zeros(P.ny + 1)
            sy[1:P.ny] = 0.5 * (ey2[li, :-1] + ey2[li, 1:])
            sy[0] = ey2[li, 0]
            sy[P.ny] = ey2[li, P.ny - 1]
            self.S2[li, :] += sx + sy

    # -- period end (Eq. 4) ----------------------------------------------------
    def period_end(self):
        import torch
        import torch.distributed as dist
        P, a, b = self.P, self.a, self.b
        dx = self.dx
        self.erms_last = np.sqrt(self.S2 / self.N)
        eeff, nu_net, D = O.density_rates(P, self.full_view(self.S2), self.n)
        wx = np.ones(P.nx + 1)
        wx[[0, -1]] = 0.5
        wy = np.ones(P.ny + 1)
        wy[[0, -1]] = 0.5
        w = wx[self.ga:self.gb, None] * wy[None, :]
        own = slice(self.c(a), self.c(b))
        heat = O.QE * O.QE / (O.ME * P.nu_m)
        p_part = float(np.sum(w[own] * self.n[own] * heat * eeff[own] * eeff[own]))
        # D_eff next to each boundary (the n halos are current)
        dl, dr = self._send_recv(D[self.c(b) - 1, :], D[self.c(a), :])
        if dl is not None:
            D[self.c(a - 1), :] = dl
        if dr is not None:
            D[self.c(b), :] = dr
        # continuity step on the local columns, the oracle's flux order
        n = self.n
        lap = np.zeros_like(n)
        fx = (0.5 * (D[:-1, :] + D[1:, :])) * (n[1:, :] - n[:-1, :])
        lap[:-1, :] += fx
        lap[1:, :] -= fx
        fy = (0.5 * (D[:, :-1] + D[:, 1:])) * (n[:, 1:] - n[:, :-1])
        lap[:, :-1] += fy
        lap[:, 1:] -= fy
        n_new = n + P.T * (lap / (dx * dx) + nu_net * n - P.r_ei * n * n)
        self.n[own] = n_new[own]
        nl, nr = self._send_recv(self.n[self.c(b) - 1, :], self.n[self.c(a), :])
        if nl is not None:
            self.n[self.c(a - 1), :] = nl
        if nr is not None:
            self.n[self.c(b), :] = nr
        self.S2[...] = 0.0
        # FP64 totals: all-reduced partial sums
        parts = torch.tensor([float(np.sum(w[own] * self.n[own])), p_part], dtype=torch.float64)
        dist.all_reduce(parts, op=dist.ReduceOp.SUM)
        self.N_e = dx * dx * float(parts[0])
        self.P_abs = dx * dx * float(parts[1])
        self.W_abs = self.W_abs + self.P_abs * P.T
        # refinement flags (Sec. III.A-III.B): bounding box MIN / MAX, count SUM
        full_cols = self.n                       # local columns incl. halos
        mask = O.flag_mask(full_cols, P.n_th, P.g_th, dx)
        lo = 1 if self.ga < a else 0             # a halo column holds no owned node
        hi = mask.shape[0] - (1 if self.gb > b else 0)
        own_mask = mask[lo:hi].copy()
        # the gradient test at the slab's first/last owned node used the halo
        # columns, like the unsplit mask; the mesh edge columns have no test
        ii, jj = np.nonzero(own_mask)
        big = 1 << 30
        box = torch.tensor([ii.min() + a if len(ii) else big, jj.min() if len(jj) else big,
                            -(ii.max() + a) if len(ii) else big, -jj.max() if len(jj) else big],
                           dtype=torch.int64)
        dist.all_reduce(box, op=dist.ReduceOp.MIN)
        cnt = torch.tensor([len(ii)], dtype=torch.int64)
        dist.all_reduce(cnt, op=dist.ReduceOp.SUM)
        self.nflag = int(cnt[0])
        self.bbox = None if self.nflag == 0 else (int(box[0]), int(box[1]), int(-box[2]), int(-box[3]))

    def full_view(self, S2):
        """A stand-in mesh for density_rates (it reads S2 and N only)."""
        class _V:
            pass
        v = _V()
        v.S2, v.N = S2, self.N
        return v

    def step(self):
        self.em_step()
        self.accumulate_e2()
        if self.m % self.P.N_T == 0:
            self.period_end()

    def advance(self, n_steps):
        for _ in range(int(n_steps)):
            self.step()

    def owned(self, name):
        """The owned columns of a field (x-major), global column offset a."""
        arr = getattr(self, name)
        a, b = self.a, self.b
        if name in ("Ex", "vx", "Hz"):
            return arr[self.c(a):self.c(min(b, self.P.nx))]
        return arr[self.c(a):self.c(b)]


# ----------------------------------------------------------------------------
# The DMR step (coarse mesh and fine rectangle) over the same slabs
# ----------------------------------------------------------------------------
_CELL = ("Ex", "vx", "Hz")
_ARRAYS = ("Ex", "vx", "Hz", "Ey", "vy", "n", "S2", "erms_last")


class DmrSlabSim(O.Sim):
    """One rank's share of a DMR run (Sec. III.C-III.D): the coarse mesh and the
    fine rectangle are cut at the same x positions (rank k owns coarse node
    columns [a_k, b_k) and the fine node columns at x in [a_k, b_k) dx_c;
    cell columns go with their left node).

    Ghost-zone form: the rank keeps arrays of the full size, but only its own
    columns and a halo of HALO coarse columns (r HALO fine columns) on each
    side hold data; everything beyond is set to NaN before every coarse step,
    so a read outside the halo would reach an owned value and show.  Before
    each coarse step every array of both meshes exchanges HALO columns with
    the neighbouring ranks; the step itself (Eqs. 1-3 on both meshes, Eq. 5b
    on the rectangle's sides, the fine->coarse transfer) is the oracle's own
    code.  At a period end (Eq. 4) the FP64 totals are all-reduced from the
    owned nodes' partial sums (SUM), the flags' bounding box (MIN / MAX) and
    the threshold-line hits (MAX) likewise, so every rank takes the same
    growth decision; the expansion (Eq. 5a) is again the oracle's own code.
    One coarse step with its period end reads at most 4 coarse columns
    beyond a slab (a halo of 3 lets NaN reach owned values in the tests);
    HALO keeps a margin."""

    HALO = 6

    def __init__(self, cfg: dict, rect, rank: int, world: int):
        super().__init__(cfg, rect=rect)
        if self.P.boundary != 0 or self.P.r < 2:
            raise ValueError("the DMR slab reference covers DMR runs with the Mur boundary")
        self.rank, self.world = rank, world
        self.bounds = slab_bounds(self.P.nx, world)
        if min(hi - lo for lo, hi in self.bounds) < self.HALO + 1:
            raise ValueError("slabs narrower than the halo")
        self.a, self.b = self.bounds[rank]

    def cols(self, k, level, name):
        """[lo, hi) of the columns rank k owns in array `name` of a level."""
        a, b = self.bounds[k]
        P = self.P
        if level == 0:
            lo, hi, ncell = a, b, P.nx
        else:
            r, i0, fnx = P.r, self.rect[0], self.fine.nx
            lo = min(max(r * (a - i0), 0), fnx + 1)
            hi = min(max(r * (b - i0), 0), fnx + 1)
            ncell = fnx
        if name in _CELL:
            lo, hi = min(lo, ncell), min(hi, ncell)
        return lo, hi

    def exchange(self):
        """Halo exchange of every array of both meshes, then the NaN fill."""
        import torch
        import torch.distributed as dist
        ops, into, fills = [], [], []
        meshes = [(0, self.coarse)] + ([(1, self.fine)] if self.fine is not None else [])
        for level, mesh in meshes:
            w = self.HALO * (1 if level == 0 else self.P.r)
            for name in _ARRAYS:
                arr = getattr(mesh, name)
                lo, hi = self.cols(self.rank, level, name)
                got_l = got_r = 0
                for nb in (self.rank - 1, self.rank + 1):
                    if nb < 0 or nb >= self.world:
                        continue
                    nlo, nhi = self.cols(nb, level, name)
                    ws, wr = min(w, hi - lo), min(w, nhi - nlo)
                    if ws > 0:
                        part = arr[lo:lo + ws] if nb < self.rank else arr[hi - ws:hi]
                        ops.append(dist.P2POp(dist.isend, torch.from_numpy(np.ascontiguousarray(part)), nb))
                    if wr > 0:
                        t = torch.empty((wr,) + arr.shape[1:], dtype=torch.float64)
                        ops.append(dist.P2POp(dist.irecv, t, nb))
                        at = lo - wr if nb < self.rank else hi
                        into.append((arr, at, t))
                        if nb < self.rank:
                            got_l = wr
                        else:
                            got_r = wr
                fills.append((arr, lo - got_l, hi + got_r))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for arr, at, t in into:
            arr[at:at + t.shape[0]] = t.numpy()
        for arr, keep_lo, keep_hi in fills:
            arr[:max(keep_lo, 0)] = np.nan
            arr[keep_hi:] = np.nan

    def advance(self, n_steps):
        with np.errstate(all="ignore"):
            for _ in range(int(n_steps)):
                self.exchange()
                self.coarse_step()

    def _owned_sum(self, level, values):
        lo, hi = self.cols(self.rank, level, "n")
        return float(np.sum(values[lo:hi]))

    def _period_end(self):
        """The oracle's period end with its sums, flags and hits taken over the
        owned nodes and all-reduced."""
        import torch
        import torch.distributed as dist
        P = self.P
        c, f = self.coarse, self.fine
        wc, wf = self._weights()
        heat = O.QE * O.QE / (O.ME * P.nu_m)
        c.erms_last = np.sqrt(c.S2 / c.N)
        f.erms_last = np.sqrt(f.S2 / f.N)
        eeff_c, nu_c, D_c = O.density_rates(P, c, c.n)
        pc = self._owned_sum(0, wc * c.n * heat * eeff_c * eeff_c)
        n_c_new = O.continuity_update(P, c.n, D_c, nu_c, c.dx)
        c.S2[...] = 0.0
        c.n = n_c_new
        eeff_f, nu_f, D_f = O.density_rates(P, f, f.n)
        pf = self._owned_sum(1, wf * f.n * heat * eeff_f * eeff_f)
        n_f_new = O.continuity_update(P, f.n, D_f, nu_f, f.dx)
        r = P.r
        i0, j0, i1, j1 = self.rect
        on_edge = self._sides()
        pa = i0 + np.arange(f.nx + 1) / r
        pb = j0 + np.arange(f.ny + 1) / r
        if not on_edge["bottom"]:
            n_f_new[:, 0] = O.linear_cfb(n_c_new[:, j0], n_c_new[:, j0], 1.0, pa)
        if not on_edge["top"]:
            n_f_new[:, -1] = O.linear_cfb(n_c_new[:, j1], n_c_new[:, j1], 1.0, pa)
        if not on_edge["left"]:
            n_f_new[0, :] = O.linear_cfb(n_c_new[i0, :], n_c_new[i0, :], 1.0, pb)
        if not on_edge["right"]:
            n_f_new[-1, :] = O.linear_cfb(n_c_new[i1, :], n_c_new[i1, :], 1.0, pb)
        f.S2[...] = 0.0
        f.n = n_f_new
        self._inject()
        parts = torch.tensor([pc, pf, self._owned_sum(0, wc * c.n), self._owned_sum(1, wf * f.n)],
                             dtype=torch.float64)
        dist.all_reduce(parts, op=dist.ReduceOp.SUM)
        p_abs = c.dx * c.dx * float(parts[0]) + f.dx * f.dx * float(parts[1])
        self.N_e = c.dx * c.dx * float(parts[2]) + f.dx * f.dx * float(parts[3])
        self.P_abs = p_abs
        self.W_abs = self.W_abs + p_abs * P.T
        self.period += 1
        # flags and growth (Sec. III.D) from the owned coarse nodes
        lo, hi = self.cols(self.rank, 0, "n")
        mask = O.flag_mask(c.n, P.n_th, P.g_th, c.dx)
        own = np.zeros_like(mask)
        own[lo:hi] = mask[lo:hi]
        self.masks.append(own)
        if self.replay is not None:
            new_rect = tuple(self.replay[self.period - 1])
        elif P.growth == 2:
            n_own = np.full(c.n.shape, -np.inf)
            n_own[lo:hi] = c.n[lo:hi]
            hits = torch.tensor([int(h) for h in O.line_hits(n_own, self.rect, P.n_th)],
                                dtype=torch.int64)
            dist.all_reduce(hits, op=dist.ReduceOp.MAX)
            new_rect = O.grow_lines(self.rect, tuple(bool(h) for h in hits.tolist()),
                                    P.m_ex, P.m_ey, P.nx, P.ny, P.rect_margin)
        elif P.growth:
            bb = O.mask_bbox(own)
            big = 1 << 30
            box = torch.tensor([big] * 4 if bb is None else [bb[0], bb[1], -bb[2], -bb[3]],
                               dtype=torch.int64)
            dist.all_reduce(box, op=dist.ReduceOp.MIN)
            bbox = None if int(box[0]) == big else (int(box[0]), int(box[1]), -int(box[2]), -int(box[3]))
            new_rect = O.grow_rect(self.rect, bbox, P.buffer, P.nx, P.ny, P.rect_margin)
        else:
            new_rect = self.rect
        if new_rect != self.rect:
            self._expand(new_rect)
        self.log.append(self.rect)
        self.stats_hist.append(self.stats())

    def owned(self, level, name):
        """The owned columns of a field of a level (x-major)."""
        mesh = self.coarse if level == 0 else self.fine
        lo, hi = self.cols(self.rank, level, name)
        return getattr(mesh, name)[lo:hi]


def dmr_slab_from_workload(w, rank, world):
    """A rank's DmrSlabSim seeded as the oracle seeds a workload (every rank
    evaluates the seed over the whole domain; the first exchange keeps its
    own columns and halo)."""
    sim = DmrSlabSim(w["cfg"], w["rect"], rank, world)
    P = sim.P
    Lx, Ly = P.nx * P.dxc, P.ny * P.dxc
    for q, (n0, fx, fy, sxl, syl) in enumerate(w["seeds"]):
        sim.seed_gaussian(n0, fx * Lx, fy * Ly, sxl * P.lam, syl * P.lam, add=q > 0)
    return sim
