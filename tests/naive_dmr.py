"""A second, deliberately naive implementation of the DMR time step with one
element per loop iteration and no shared helpers with the oracle.  It exists
only to cross-check the oracle's index arithmetic on tiny meshes (P11).

Every formula is written out per element from the method statement:
Eqs. 1-4 (Sec. II.A), Yee scattered-field FDTD with first-order Mur
(Sec. II.B), sub-cycling and Eq. 5a/5b transfers (Sec. III.C), flagging and
growth (Sec. III.D).
"""
import math

C = 299792458.0
MU = 1.25663706212e-6
EPS = 8.8541878128e-12
Q = 1.602176634e-19
M = 9.1093837015e-31


def grid(a, b, v=0.0):
    return [[v for _ in range(b)] for _ in range(a)]


class NMesh:
    def __init__(self, nx, ny, dx, dt, steps, gi0, gj0):
        self.nx, self.ny, self.dx, self.dt, self.N = nx, ny, dx, dt, steps
        self.gi0, self.gj0 = gi0, gj0
        self.Ex = grid(nx, ny + 1)
        self.vx = grid(nx, ny + 1)
        self.Ey = grid(nx + 1, ny)
        self.vy = grid(nx + 1, ny)
        self.Hz = grid(nx, ny)
        self.n = grid(nx + 1, ny + 1)
        self.S2 = grid(nx + 1, ny + 1)
        self.m = 0


class Naive:
    def __init__(self, cfg, rect):
        self.nx, self.ny, self.r = cfg["nx"], cfg["ny"], cfg["r"]
        self.f = cfg["freq"]
        self.E0 = cfg["E0"]
        self.p = cfg["p_torr"]
        self.NT = cfg["steps_per_period"]
        lam = C / self.f
        self.lam = lam
        self.w = 2 * math.pi * self.f
        self.k = self.w / C
        self.num = 5.3e9 * self.p
        self.De = 0.1 * 760.0 / self.p if cfg.get("De") is None else cfg["De"]
        self.Da = self.De / 100.0 if cfg.get("Da") is None else cfg["Da"]
        beta = 1.0 if cfg.get("beta_rec") is None else cfg["beta_rec"]
        Te = 300.0 if cfg.get("Te") is None else cfg["Te"]
        self.rei = beta * 1e-13 * math.sqrt(300.0 / Te)
        self.snu = 1.0 if cfg.get("nu_scale") is None else cfg["nu_scale"]
        nl = cfg["n_lambda"]
        dxc = lam / nl
        ncrit = M * EPS * self.w * self.w / (Q * Q)
        self.nth = 1e-3 * ncrit if cfg.get("n_th") is None else cfg["n_th"]
        self.gth = self.nth / (4 * dxc) if cfg.get("g_th") is None else cfg["g_th"]
        self.buf = cfg.get("buffer_cells", 4)
        self.mode = 1 if cfg.get("growth") is None else int(cfg["growth"])
        self.mex = 2 * self.buf if cfg.get("m_ex") is None else cfg["m_ex"]
        self.mey = self.buf if cfg.get("m_ey") is None else cfg["m_ey"]
        self.coupling = int(cfg.get("coupling") or 0)   # 1: no fine -> coarse E
        self.nl = nl
        self.c = NMesh(self.nx, self.ny, lam / nl, 1.0 / (self.f * self.NT), self.NT, 0, 0)
        self.rect = tuple(rect)
        self.fm = self._new_fine(self.rect)
        self.log = []

    def _new_fine(self, rect):
        r = self.r
        i0, j0, i1, j1 = rect
        return NMesh(r * (i1 - i0), r * (j1 - j0), self.lam / (r * self.nl),
                     1.0 / (self.f * (r * self.NT)), r * self.NT, r * i0, r * j0)

    def seed(self, n0, x0, y0, sx, sy):
        for mesh in (self.c, self.fm):
            for i in range(mesh.nx + 1):
                for j in range(mesh.ny + 1):
                    x = (mesh.gi0 + i) * mesh.dx
                    y = (mesh.gj0 + j) * mesh.dx
                    a = (x - x0) ** 2 / sx ** 2 + (y - y0) ** 2 / sy ** 2
                    mesh.n[i][j] = n0 * math.exp(-a) if a <= 60.0 else 0.0
        self.inject()

    def inject(self):
        r = self.r
        i0, j0, i1, j1 = self.rect
        for i in range(i0, i1 + 1):
            for j in range(j0, j1 + 1):
                self.c.n[i][j] = self.fm.n[r * (i - i0)][r * (j - j0)]

    def einc(self, mesh, i, m):
        x = (mesh.gi0 + i) * mesh.dx
        return self.E0 * math.sin(2 * math.pi * (m % mesh.N) / mesh.N - self.k * x)

    def step_mesh(self, mesh, boundary):
        """boundary(side, idx, Eold_boundary, Eold_inner, Enew_inner) -> value"""
        dt, dx = mesh.dt, mesh.dx
        nx, ny = mesh.nx, mesh.ny
        for i in range(nx):
            for j in range(ny):
                curl = (mesh.Ey[i + 1][j] - mesh.Ey[i][j]) / dx - (mesh.Ex[i][j + 1] - mesh.Ex[i][j]) / dx
                mesh.Hz[i][j] = mesh.Hz[i][j] - dt / MU * curl
        h = self.num * dt / 2
        for i in range(nx):
            for j in range(ny + 1):
                mesh.vx[i][j] = ((1 - h) * mesh.vx[i][j] - Q * dt / M * mesh.Ex[i][j]) / (1 + h)
        for i in range(nx + 1):
            e_in = self.einc(mesh, i, mesh.m)
            for j in range(ny):
                mesh.vy[i][j] = ((1 - h) * mesh.vy[i][j] - Q * dt / M * (mesh.Ey[i][j] + e_in)) / (1 + h)
        oldEx = [row[:] for row in mesh.Ex]
        oldEy = [row[:] for row in mesh.Ey]
        for i in range(nx):
            for j in range(1, ny):
                J = -Q * 0.5 * (mesh.n[i][j] + mesh.n[i + 1][j]) * mesh.vx[i][j]
                mesh.Ex[i][j] = oldEx[i][j] + dt / EPS * ((mesh.Hz[i][j] - mesh.Hz[i][j - 1]) / dx - J)
        for i in range(1, nx):
            for j in range(ny):
                J = -Q * 0.5 * (mesh.n[i][j] + mesh.n[i][j + 1]) * mesh.vy[i][j]
                mesh.Ey[i][j] = oldEy[i][j] + dt / EPS * (-(mesh.Hz[i][j] - mesh.Hz[i - 1][j]) / dx - J)
        for j in range(ny):
            mesh.Ey[0][j] = boundary("left", j, oldEy[0][j], oldEy[1][j], mesh.Ey[1][j])
            mesh.Ey[nx][j] = boundary("right", j, oldEy[nx][j], oldEy[nx - 1][j], mesh.Ey[nx - 1][j])
        for i in range(nx):
            mesh.Ex[i][0] = boundary("bottom", i, oldEx[i][0], oldEx[i][1], mesh.Ex[i][1])
            mesh.Ex[i][ny] = boundary("top", i, oldEx[i][ny], oldEx[i][ny - 1], mesh.Ex[i][ny - 1])
        mesh.m += 1

    def mur(self, mesh):
        co = (C * mesh.dt - mesh.dx) / (C * mesh.dt + mesh.dx)
        return lambda side, idx, eb, e1o, e1n: e1o + co * (e1n - eb)

    def acc(self, mesh):
        for i in range(mesh.nx + 1):
            e_in = self.einc(mesh, i, mesh.m)
            for j in range(mesh.ny + 1):
                xs = []
                if i - 1 >= 0:
                    xs.append(mesh.Ex[i - 1][j] ** 2)
                if i <= mesh.nx - 1:
                    xs.append(mesh.Ex[i][j] ** 2)
                ys = []
                if j - 1 >= 0:
                    ys.append((mesh.Ey[i][j - 1] + e_in) ** 2)
                if j <= mesh.ny - 1:
                    ys.append((mesh.Ey[i][j] + e_in) ** 2)
                mesh.S2[i][j] += sum(xs) / len(xs) + sum(ys) / len(ys)

    @staticmethod
    def lin(line, pos):
        L = len(line)
        i = math.floor(pos)
        w = pos - i
        if i < 0:
            i, w = 0, 0.0
        if i > L - 2:
            i, w = L - 2, 1.0
        return line[i] * (1 - w) + line[i + 1] * w

    def coarse_step(self):
        c, fm, r = self.c, self.fm, self.r
        i0, j0, i1, j1 = self.rect
        old_b = [c.Ex[i][j0] for i in range(c.nx)]
        old_t = [c.Ex[i][j1] for i in range(c.nx)]
        old_l = [c.Ey[i0][j] for j in range(c.ny)]
        old_r = [c.Ey[i1][j] for j in range(c.ny)]
        self.step_mesh(c, self.mur(c))
        new_b = [c.Ex[i][j0] for i in range(c.nx)]
        new_t = [c.Ex[i][j1] for i in range(c.nx)]
        new_l = [c.Ey[i0][j] for j in range(c.ny)]
        new_r = [c.Ey[i1][j] for j in range(c.ny)]
        edge = {"left": i0 == 0, "right": i1 == self.nx, "bottom": j0 == 0, "top": j1 == self.ny}
        lines = {"bottom": (old_b, new_b, i0), "top": (old_t, new_t, i0),
                 "left": (old_l, new_l, j0), "right": (old_r, new_r, j0)}
        murf = self.mur(fm)
        for k in range(1, r + 1):
            frac = k / r

            def bnd(side, idx, eb, e1o, e1n):
                if edge[side]:
                    return murf(side, idx, eb, e1o, e1n)
                old, new, start = lines[side]
                pos = start + (idx + 0.5) / r - 0.5
                return (1 - frac) * self.lin(old, pos) + frac * self.lin(new, pos)

            self.step_mesh(fm, bnd)
            self.acc(fm)
        # fine -> coarse
        for i in (range(i0, i1) if self.coupling == 0 else ()):
            for j in range(j0, j1 + 1):
                if (j == j0 and not edge["bottom"]) or (j == j1 and not edge["top"]):
                    continue
                s = 0.0
                for q in range(r):
                    s = s + fm.Ex[r * (i - i0) + q][r * (j - j0)]
                c.Ex[i][j] = s / r
        for i in (range(i0, i1 + 1) if self.coupling == 0 else ()):
            if (i == i0 and not edge["left"]) or (i == i1 and not edge["right"]):
                continue
            for j in range(j0, j1):
                s = 0.0
                for q in range(r):
                    s = s + fm.Ey[r * (i - i0)][r * (j - j0) + q]
                c.Ey[i][j] = s / r
        self.acc(c)
        if c.m % self.NT == 0:
            self.period_end()

    def rates(self, mesh, i, j):
        erms2 = mesh.S2[i][j] / mesh.N
        eeff = math.sqrt(erms2 / (1 + (self.w / self.num) ** 2))
        x = eeff / (100 * self.p)
        nu = self.snu * 5.14e11 * self.p * math.exp(-73 * x ** -0.44) if x > 0 else 0.0
        wp2 = mesh.n[i][j] * Q * Q / (M * EPS)
        den = nu * self.num + wp2
        D = self.De if den == 0 else (nu * self.num * self.De + wp2 * self.Da) / den
        return nu, D

    def density(self, mesh):
        nx, ny = mesh.nx, mesh.ny
        nu = grid(nx + 1, ny + 1)
        D = grid(nx + 1, ny + 1)
        for i in range(nx + 1):
            for j in range(ny + 1):
                nu[i][j], D[i][j] = self.rates(mesh, i, j)
        out = grid(nx + 1, ny + 1)
        for i in range(nx + 1):
            for j in range(ny + 1):
                n = mesh.n[i][j]
                lap = 0.0
                for a, b in ((i - 1, j), (i + 1, j), (i, j - 1), (i, j + 1)):
                    if 0 <= a <= nx and 0 <= b <= ny:
                        lap += 0.5 * (D[i][j] + D[a][b]) * (mesh.n[a][b] - n)
                out[i][j] = n + (1.0 / self.f) * (lap / mesh.dx ** 2 + nu[i][j] * n - self.rei * n * n)
        return out

    def flags(self):
        c = self.c
        s = 1.0 / (2 * c.dx * self.gth)
        hits = []
        for i in range(c.nx + 1):
            for j in range(c.ny + 1):
                fl = c.n[i][j] > self.nth
                if 0 < i < c.nx and 0 < j < c.ny:
                    gx = (c.n[i + 1][j] - c.n[i - 1][j]) * s
                    gy = (c.n[i][j + 1] - c.n[i][j - 1]) * s
                    fl = fl or (gx * gx + gy * gy > 1.0)
                if fl:
                    hits.append((i, j))
        return hits

    def period_end(self):
        c, fm, r = self.c, self.fm, self.r
        i0, j0, i1, j1 = self.rect
        nc = self.density(c)
        nf = self.density(fm)
        edge = {"left": i0 == 0, "right": i1 == self.nx, "bottom": j0 == 0, "top": j1 == self.ny}
        for a in range(fm.nx + 1):
            if not edge["bottom"]:
                nf[a][0] = self.lin([nc[i][j0] for i in range(c.nx + 1)], i0 + a / r)
            if not edge["top"]:
                nf[a][fm.ny] = self.lin([nc[i][j1] for i in range(c.nx + 1)], i0 + a / r)
        for b in range(fm.ny + 1):
            if not edge["left"]:
                nf[0][b] = self.lin([nc[i0][j] for j in range(c.ny + 1)], j0 + b / r)
            if not edge["right"]:
                nf[fm.nx][b] = self.lin([nc[i1][j] for j in range(c.ny + 1)], j0 + b / r)
        c.n, fm.n = nc, nf
        c.S2 = grid(c.nx + 1, c.ny + 1)
        fm.S2 = grid(fm.nx + 1, fm.ny + 1)
        self.inject()
        hits = self.flags()
        self.last_hits = hits
        if self.mode == 2:
            # threshold lines = the rectangle's sides, node by node
            th = self.nth
            left = right = bottom = top = False
            for j in range(j0, j1 + 1):
                left = left or c.n[i0][j] > th
                right = right or c.n[i1][j] > th
            for i in range(i0, i1 + 1):
                bottom = bottom or c.n[i][j0] > th
                top = top or c.n[i][j1] > th
            new = (i0, j0, i1, j1)
            if left:
                new = (max(i0 - self.mex, 0), new[1], new[2], new[3])
            if right:
                new = (new[0], new[1], min(i1 + self.mex, self.nx), new[3])
            if bottom:
                new = (new[0], max(j0 - self.mey, 0), new[2], new[3])
            if top:
                new = (new[0], new[1], new[2], min(j1 + self.mey, self.ny))
            if new != self.rect:
                self.expand(new)
        elif hits and self.mode == 1:
            bi0 = max(min(h[0] for h in hits) - self.buf, 0)
            bj0 = max(min(h[1] for h in hits) - self.buf, 0)
            bi1 = min(max(h[0] for h in hits) + self.buf, self.nx)
            bj1 = min(max(h[1] for h in hits) + self.buf, self.ny)
            new = (min(i0, bi0), min(j0, bj0), max(i1, bi1), max(j1, bj1))
            if new != self.rect:
                self.expand(new)
        self.log.append(self.rect)

    def sample(self, F, ox, oy, x, y):
        Lx, Ly = len(F), len(F[0])
        u, v = x - ox, y - oy
        i = math.floor(u)
        fu = u - i
        if i < 0:
            i, fu = 0, 0.0
        if i > Lx - 2:
            i, fu = Lx - 2, 1.0
        j = math.floor(v)
        fv = v - j
        if j < 0:
            j, fv = 0, 0.0
        if j > Ly - 2:
            j, fv = Ly - 2, 1.0
        return (F[i][j] * (1 - fu) * (1 - fv) + F[i + 1][j] * fu * (1 - fv)
                + F[i][j + 1] * (1 - fu) * fv + F[i + 1][j + 1] * fu * fv)

    def expand(self, new):
        r = self.r
        old, orect = self.fm, self.rect
        nf = self._new_fine(new)
        nf.m = old.m
        oi, oj = r * (orect[0] - new[0]), r * (orect[1] - new[1])
        spec = (("Ex", 0.5, 0.0), ("vx", 0.5, 0.0), ("Ey", 0.0, 0.5), ("vy", 0.0, 0.5),
                ("Hz", 0.5, 0.5), ("n", 0.0, 0.0))
        for name, ox, oy in spec:
            dst = getattr(nf, name)
            src = getattr(old, name)
            cF = getattr(self.c, name)
            for a in range(len(dst)):
                for b in range(len(dst[0])):
                    sa, sb = a - oi, b - oj
                    if 0 <= sa < len(src) and 0 <= sb < len(src[0]):
                        dst[a][b] = src[sa][sb]
                    else:
                        x = new[0] + (a + ox) / r
                        y = new[1] + (b + oy) / r
                        dst[a][b] = self.sample(cF, ox, oy, x, y)
        self.fm = nf
        self.rect = new
