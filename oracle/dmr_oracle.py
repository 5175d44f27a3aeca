"""Plain FP64 CPU oracle of the DMR EM-plasma time step.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline
and reference legs) may use it.  It shares no code with the CUDA library.

What it computes (paper: Ghosh & Chaudhury, "Dynamic mesh refinement for
HPM breakdown", arXiv 2105.13276):

* Eqs. 1-3 (Sec. II.A) on a 2D TE_z Yee mesh in scattered-field form with a
  first-order Mur outer boundary (Sec. II.B, Fig. 1 caption);
* Eq. 4 (Sec. II.A), the electron continuity equation with ionization,
  effective diffusion and recombination, advanced once per EM period
  (Sec. II.B, Sec. III.C);
* one coarse mesh plus one fine rectangle with refinement factor r and r
  fine sub-steps per coarse step (Sec. III.C);
* coarse -> fine transfer by Eq. 5b (linear, on the coarse-fine boundary)
  and Eq. 5a (bilinear, into newly refined area), fine -> coarse transfer
  (Sec. III.C);
* threshold / gradient flagging and rectangle growth (Sec. III.A-III.D).

Arrays are indexed ``[i, j]`` with i along x and j along y:
  Ex, vx : (nx, ny+1)   at ((i+1/2)d, j d)
  Ey, vy : (nx+1, ny)   at (i d, (j+1/2)d)
  Hz     : (nx, ny)     at ((i+1/2)d, (j+1/2)d)
  n, S2  : (nx+1, ny+1) at nodes (i d, j d)
E lives on integer time levels, H and v on half levels.

All arithmetic is written so that it also runs on complex128 arrays
(complex-step derivatives): comparisons use the real part.

Readings of passages the paper leaves open are stated where they are used.
Parity unpinned: the spatio-temporal physics magnitudes (filament spacing,
front speed), whose figures are missing from the paper.
"""
from __future__ import annotations

import math

import numpy as np

# CODATA 2018 constants (SI).
C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 8.8541878128e-12
QE = 1.602176634e-19
ME = 9.1093837015e-31


class CapacityError(RuntimeError):
    """The patch would exceed the configured fine-cell capacity."""


# ----------------------------------------------------------------------------
# Parameters
# ----------------------------------------------------------------------------
class Params:
    """Physical and numerical parameters (Sec. II, Sec. III.C).

    ``cfg`` is a plain dict with keys nx, ny, r, n_lambda, steps_per_period,
    freq, E0, p_torr and optional De, Da, beta_rec, Te, nu_scale, nu_a, n_th,
    g_th, buffer_cells, growth, m_ex, m_ey, nu_model, town_A, town_B,
    boundary, pml_cells, patch_cap_cells, coupling.  A value of None (or a
    missing key) selects the default reading.
    """

    def __init__(self, cfg: dict):
        g = cfg.get
        self.nx = int(cfg["nx"])
        self.ny = int(cfg["ny"])
        self.r = int(g("r", 1))
        self.n_lambda = int(cfg["n_lambda"])
        self.N_T = int(cfg["steps_per_period"])
        self.freq = float(cfg["freq"])
        self.E0 = cfg["E0"]                      # may be complex (complex step)
        self.p = float(cfg["p_torr"])
        # Sec. II.A: nu_m = 5.3e9 p[Torr] s^-1.
        self.nu_m = 5.3e9 * self.p
        self.omega = 2.0 * math.pi * self.freq
        self.lam = C0 / self.freq
        self.k = self.omega / C0
        # Reading: D_e = 0.1 (760/p) m^2/s, D_a = D_e/100 (D_eff deferred to
        # cited works, Sec. II.A).
        self.De = float(g("De") if g("De") is not None else 0.1 * 760.0 / self.p)
        self.Da = float(g("Da") if g("Da") is not None else self.De / 100.0)
        self.beta_rec = float(g("beta_rec") if g("beta_rec") is not None else 1.0)
        self.Te = float(g("Te") if g("Te") is not None else 300.0)
        self.nu_scale = g("nu_scale") if g("nu_scale") is not None else 1.0
        self.nu_a = float(g("nu_a") if g("nu_a") is not None else 0.0)
        # ionization coefficient set: 0 the air fit, 1 the Townsend form with
        # A = 15 /(cm Torr), B = 365 V/(cm Torr) by default (reading; SI here)
        self.nu_model = int(g("nu_model") if g("nu_model") is not None else 0)
        # outer boundary: 0 first-order Mur (Fig. 1 caption), 1 CPML of
        # pml_cells coarse cells backed by PEC (the benchmark set-up names
        # "Mur/PML"); the fine rectangle then stays pml_cells + 2 cells inside
        self.boundary = int(g("boundary") if g("boundary") is not None else 0)
        self.pml_cells = int(g("pml_cells") if g("pml_cells") is not None else 8)
        self.rect_margin = self.pml_cells + 2 if self.boundary == 1 else 0
        self.town_A = float(g("town_A") if g("town_A") is not None else 1500.0)
        self.town_B = float(g("town_B") if g("town_B") is not None else 36500.0)
        # Sec. III.A: critical density n_c = m eps0 w^2 / e^2 (the square is
        # fixed by the quoted cutoff density ~9e20 m^-3, Sec. IV.D).
        self.n_crit = ME * EPS0 * self.omega ** 2 / QE ** 2
        self.dxc = self.lam / self.n_lambda
        self.n_th = float(g("n_th") if g("n_th") is not None else 1e-3 * self.n_crit)
        self.g_th = float(g("g_th") if g("g_th") is not None else self.n_th / (4.0 * self.dxc))
        self.buffer = int(g("buffer_cells") if g("buffer_cells") is not None else 4)
        # growth: 0 fixed rectangle, 1 flag bounding box + buffer, 2 threshold
        # lines with jumps m_ex, m_ey (Sec. III.D; reading: 2 and 1 buffers)
        gr = g("growth")
        self.growth = 1 if gr is None else int(gr)
        self.m_ex = int(g("m_ex") if g("m_ex") is not None else 2 * self.buffer)
        self.m_ey = int(g("m_ey") if g("m_ey") is not None else self.buffer)
        self.cap = int(g("patch_cap_cells") if g("patch_cap_cells") is not None
                       else (self.r * self.nx) * (self.r * self.ny))
        # Sec. III.C: the fine mesh's updated quantities go back to the coarse
        # mesh.  coupling 0 (default reading): the E means every coarse step and
        # the density every period; 1: the density only (the coarse E under
        # the rectangle stays the coarse mesh's own)
        self.coupling = int(g("coupling") or 0)
        if self.coupling not in (0, 1):
            raise ValueError("coupling must be 0 or 1")
        # Sec. II.A: r_ei = beta 1e-13 (300/T_e)^(1/2), read in m^3/s.
        self.r_ei = self.beta_rec * 1e-13 * math.sqrt(300.0 / self.Te)
        # Plasma step: forward Euler over one EM period (Sec. III.C).
        self.T = 1.0 / self.freq
        # 2D Yee stability: Courant number c dt/dx = n_lambda/N_T <= 1/sqrt(2)
        self.courant = self.n_lambda / self.N_T
        if self.courant > 1.0 / math.sqrt(2.0):
            raise ValueError("Courant number %.3f exceeds 1/sqrt(2)" % self.courant)

    def mesh_dx(self, rr):
        """Cell size of a mesh refined rr times relative to the coarse one."""
        return self.lam / (rr * self.n_lambda)

    def mesh_dt(self, rr):
        """EM time step: an integer number rr*N_T of steps fills one period."""
        return 1.0 / (self.freq * (rr * self.N_T))


# ----------------------------------------------------------------------------
# One Yee mesh
# ----------------------------------------------------------------------------
class Mesh:
    """Field arrays of one mesh (the coarse mesh or the fine rectangle).

    ``gi0, gj0`` are the global node indices of its lower-left node in its own
    resolution (the fine rectangle starting at coarse node I0 has gi0 = r*I0).
    """

    def __init__(self, P: Params, nx, ny, rr, gi0=0, gj0=0, dtype=np.float64):
        self.nx, self.ny, self.rr = nx, ny, rr
        self.gi0, self.gj0 = gi0, gj0
        self.dx = P.mesh_dx(rr)
        self.dt = P.mesh_dt(rr)
        self.N = rr * P.N_T                 # EM steps per period on this mesh
        z = lambda a, b: np.zeros((a, b), dtype=dtype)
        self.Ex, self.vx = z(nx, ny + 1), z(nx, ny + 1)
        self.Ey, self.vy = z(nx + 1, ny), z(nx + 1, ny)
        self.Hz = z(nx, ny)
        self.n = z(nx + 1, ny + 1)
        self.S2 = z(nx + 1, ny + 1)
        # E_rms of the last completed period at the nodes (Sec. II.B output
        # E_rms(x, y, t)), kept when the period end resets S2
        self.erms_last = np.zeros((nx + 1, ny + 1))
        self.m = 0                           # time level of E (steps done)

    def node_x(self):
        return (self.gi0 + np.arange(self.nx + 1)) * self.dx

    def node_y(self):
        return (self.gj0 + np.arange(self.ny + 1)) * self.dx


def incident_ey(P: Params, mesh: Mesh, m):
    """Incident plane wave on the Ey columns at time level m (Sec. II.B).

    Reading: E_inc,y = E0 sin(w t - k x), k = w/c, x from the left edge,
    present in the whole domain from t = 0.  Because N steps fill one period
    exactly, w t is taken as 2 pi (m mod N)/N.
    """
    phase = 2.0 * math.pi * (m % mesh.N) / mesh.N
    return P.E0 * np.sin(phase - P.k * mesh.node_x())


# ----------------------------------------------------------------------------
# EM step: Eqs. 1-3 with Mur / coarse-fine boundaries
# ----------------------------------------------------------------------------
class CPML:
    """Convolutional PML (Roden and Gedney's recursive form, kappa = 1,
    alpha = 0) on the outer L cells of a mesh, backed by PEC.  sigma grows as
    sigma_max (d/L)^3 with the depth d into the layer, sigma_max =
    0.8 (m + 1) / (eta0 dx), m = 3; per step psi <- b psi + c D with
    b = exp(-sigma dt / eps0), c = b - 1, D the difference the curl uses at
    the point where psi lives (cell centres for Hz, nodes for Ex, Ey).
    Outside the layer b = 1, c = 0, so psi stays exactly 0 there."""

    def __init__(self, mesh, L, dtype=np.float64):
        nx, ny, dx, dt = mesh.nx, mesh.ny, mesh.dx, mesh.dt
        eta0 = math.sqrt(MU0 / EPS0)
        smax = 0.8 * 4.0 / (eta0 * dx)

        def coef(pos, n):
            d = np.maximum(np.maximum(L - pos, pos - (n - L)), 0.0) / L
            b = np.exp(-smax * d ** 3 * dt / EPS0)
            return b, b - 1.0

        self.bxh, self.cxh = coef(np.arange(nx) + 0.5, nx)      # Hz cells, x
        self.byh, self.cyh = coef(np.arange(ny) + 0.5, ny)      # Hz cells, y
        self.bxn, self.cxn = coef(np.arange(nx + 1.0), nx)      # nodes, x (Ey)
        self.byn, self.cyn = coef(np.arange(ny + 1.0), ny)      # nodes, y (Ex)
        z = lambda a, b: np.zeros((a, b), dtype=dtype)
        self.hx, self.hy = z(nx, ny), z(nx, ny)                 # psi of Hz (x, y)
        self.exy = z(nx, ny + 1)                                 # psi of Ex (y)
        self.eyx = z(nx + 1, ny)                                 # psi of Ey (x)


def em_step(P: Params, mesh: Mesh, sides=None, bc="mur"):
    """Advance one EM step on ``mesh`` (Eqs. 1-3, Yee leapfrog, Sec. II.B).

    Order: H^{n+1/2} from E^n (Eq. 2); v^{n+1/2} from v^{n-1/2} and the total
    field E^n (Eq. 3, Crank-Nicolson on the collision term -- a reading);
    E^{n+1} on interior edges from curl H and J = -e n v (Eq. 1, J with the
    mean density of the edge's two end nodes); then the four sides.

    ``sides`` maps 'left','right','bottom','top' to either 'mur' (first-order
    Mur on the scattered tangential E, Fig. 1 caption) or an array holding
    the tangential E of that side at level n+1 (coarse-fine boundary values
    from Eq. 5b).  ``bc='pec'`` zeroes the tangential E instead (the cavity
    invariants); ``bc='cpml'`` applies the mesh's CPML layer (``mesh.pml``)
    and PEC behind it.
    """
    dt, dx = mesh.dt, mesh.dx
    Ex, Ey, Hz, vx, vy, n = mesh.Ex, mesh.Ey, mesh.Hz, mesh.vx, mesh.vy, mesh.n
    pml = mesh.pml if bc == "cpml" else None

    # Eq. 2: dHz/dt = -(1/mu0) (dEy/dx - dEx/dy)
    if pml is None:
        Hz -= (dt / MU0) * ((Ey[1:, :] - Ey[:-1, :]) / dx - (Ex[:, 1:] - Ex[:, :-1]) / dx)
    else:
        dey, dex = Ey[1:, :] - Ey[:-1, :], Ex[:, 1:] - Ex[:, :-1]
        pml.hx[...] = pml.bxh[:, None] * pml.hx + pml.cxh[:, None] * dey
        pml.hy[...] = pml.byh[None, :] * pml.hy + pml.cyh[None, :] * dex
        Hz -= (dt / MU0) * ((dey + pml.hx) / dx - (dex + pml.hy) / dx)

    # Eq. 3: dv/dt = -e E/m - nu_m v, E = scattered + incident (total field)
    einc = incident_ey(P, mesh, mesh.m)
    half = 0.5 * P.nu_m * dt
    vx[...] = ((1.0 - half) * vx - (QE * dt / ME) * Ex) / (1.0 + half)
    vy[...] = ((1.0 - half) * vy - (QE * dt / ME) * (Ey + einc[:, None])) / (1.0 + half)

    # J = -e n v with n averaged over the two end nodes of each edge
    Jx = -QE * (0.5 * (n[:-1, :] + n[1:, :])) * vx
    Jy = -QE * (0.5 * (n[:, :-1] + n[:, 1:])) * vy

    Ex_old, Ey_old = Ex.copy(), Ey.copy()
    # Eq. 1 on interior edges: dEx/dt = (dHz/dy - Jx)/eps0, dEy/dt = (-dHz/dx - Jy)/eps0
    if pml is None:
        Ex[:, 1:-1] += (dt / EPS0) * ((Hz[:, 1:] - Hz[:, :-1]) / dx - Jx[:, 1:-1])
        Ey[1:-1, :] += (dt / EPS0) * (-(Hz[1:, :] - Hz[:-1, :]) / dx - Jy[1:-1, :])
    else:
        dhy, dhx = Hz[:, 1:] - Hz[:, :-1], Hz[1:, :] - Hz[:-1, :]
        pml.exy[:, 1:-1] = pml.byn[None, 1:-1] * pml.exy[:, 1:-1] + pml.cyn[None, 1:-1] * dhy
        pml.eyx[1:-1, :] = pml.bxn[1:-1, None] * pml.eyx[1:-1, :] + pml.cxn[1:-1, None] * dhx
        Ex[:, 1:-1] += (dt / EPS0) * ((dhy + pml.exy[:, 1:-1]) / dx - Jx[:, 1:-1])
        Ey[1:-1, :] += (dt / EPS0) * (-(dhx + pml.eyx[1:-1, :]) / dx - Jy[1:-1, :])
        bc = "pec"                               # the layer is backed by PEC

    if sides is None:
        sides = {s: bc for s in ("left", "right", "bottom", "top")}
    coef = (C0 * dt - dx) / (C0 * dt + dx)
    for side, how in sides.items():
        if isinstance(how, str) and how == "pec":
            if side == "left":
                Ey[0, :] = 0.0
            elif side == "right":
                Ey[-1, :] = 0.0
            elif side == "bottom":
                Ex[:, 0] = 0.0
            else:
                Ex[:, -1] = 0.0
        elif isinstance(how, str) and how == "mur":
            # first-order Mur: E_b^{n+1} = E_1^n + coef (E_1^{n+1} - E_b^n)
            if side == "left":
                Ey[0, :] = Ey_old[1, :] + coef * (Ey[1, :] - Ey_old[0, :])
            elif side == "right":
                Ey[-1, :] = Ey_old[-2, :] + coef * (Ey[-2, :] - Ey_old[-1, :])
            elif side == "bottom":
                Ex[:, 0] = Ex_old[:, 1] + coef * (Ex[:, 1] - Ex_old[:, 0])
            else:
                Ex[:, -1] = Ex_old[:, -2] + coef * (Ex[:, -2] - Ex_old[:, -1])
        else:
            vals = how
            if side == "left":
                Ey[0, :] = vals
            elif side == "right":
                Ey[-1, :] = vals
            elif side == "bottom":
                Ex[:, 0] = vals
            else:
                Ex[:, -1] = vals
    mesh.m += 1


def accumulate_e2(P: Params, mesh: Mesh):
    """Add the squared total field at the current level to S2 (nodes).

    Reading of the E_eff time average (Sec. II.A local-field approximation):
    at node (i,j) the Ex^2 term is the mean over the existing Ex edges
    (i-1,j),(i,j) and the Ey^2 term the mean over the existing Ey edges
    (i,j-1),(i,j), with Ey total = scattered + incident at this level.
    """
    ex2 = mesh.Ex * mesh.Ex
    eyt = mesh.Ey + incident_ey(P, mesh, mesh.m)[:, None]
    ey2 = eyt * eyt
    nx, ny = mesh.nx, mesh.ny
    sx = np.zeros_like(mesh.S2)
    sx[1:nx, :] = 0.5 * (ex2[:-1, :] + ex2[1:, :])
    sx[0, :] = ex2[0, :]
    sx[nx, :] = ex2[nx - 1, :]
    sy = np.zeros_like(mesh.S2)
    sy[:, 1:ny] = 0.5 * (ey2[:, :-1] + ey2[:, 1:])
    sy[:, 0] = ey2[:, 0]
    sy[:, ny] = ey2[:, ny - 1]
    mesh.S2 += sx + sy


# ----------------------------------------------------------------------------
# Eq. 4: electron continuity, once per period
# ----------------------------------------------------------------------------
def ionization_frequency(P: Params, eeff):
    """nu_i(E_eff/p) (Sec. II.A gives nu_i - nu_a = gamma v_d with A, B, v_d
    deferred to cited work); nu_i = 0 where E_eff = 0.

    nu_model 0 (default reading): the air fit
      nu_i = s_nu 5.14e11 p exp(-73 (E_eff/p)^-0.44), E_eff/p in V/(cm Torr),
      p in Torr.
    nu_model 1 (the paper's Townsend form): nu_i = s_nu gamma v_d with
      gamma = A p exp(-B p / E_eff) (1/m), A in 1/(m Torr), B in V/(m Torr),
      and the drift velocity v_d = mu_e E_eff, mu_e = e / (m_e nu_m) (the
      mobility of the model's collision frequency)."""
    pos = np.real(eeff) > 0
    es = np.where(pos, eeff, 1.0)
    if P.nu_model == 1:
        mu_e = QE / (ME * P.nu_m)
        nu = P.nu_scale * P.town_A * P.p * np.exp(-P.town_B * P.p / es) * mu_e * es
        return np.where(pos, nu, 0.0)
    xs = es / (100.0 * P.p)
    return np.where(pos, P.nu_scale * 5.14e11 * P.p * np.exp(-73.0 * xs ** -0.44), 0.0)


def density_rates(P: Params, mesh: Mesh, n):
    """E_eff, nu_net and D_eff at the nodes from the period's S2 (Sec. II.A).

    E_rms^2 = S2/N (N samples over one period); E_eff = E_rms/sqrt(1+w^2/nu_m^2)
    (local-field approximation, pinned by the worked example in Sec. IV.D);
    D_eff = (alpha D_e + D_a)/(1 + alpha), alpha = nu_i nu_m / w_p^2 (reading of
    the effective diffusion of the cited work), D_eff = D_e where nu_i nu_m and
    w_p^2 are both zero.
    """
    erms2 = mesh.S2 / mesh.N
    eeff = np.sqrt(erms2 / (1.0 + (P.omega / P.nu_m) ** 2))
    nu_i = ionization_frequency(P, eeff)
    nu_net = nu_i - P.nu_a
    wp2 = n * (QE * QE / (ME * EPS0))
    num = nu_i * P.nu_m * P.De + wp2 * P.Da
    den = nu_i * P.nu_m + wp2
    zero = np.real(den) == 0
    D = np.where(zero, P.De, num / np.where(zero, 1.0, den))
    return eeff, nu_net, D


def continuity_update(P: Params, n, D, nu_net, dx):
    """One forward-Euler step of Eq. 4 over one EM period T.

    n' = n + T [ div(D_eff grad n) + nu_net n - r_ei n^2 ] with the flux on
    each face D_face (n_nb - n)/dx^2, D_face the mean of the face's two nodes,
    and no flux through the domain edges (reading).
    """
    lap = np.zeros_like(n)
    fx = (0.5 * (D[:-1, :] + D[1:, :])) * (n[1:, :] - n[:-1, :])
    lap[:-1, :] += fx
    lap[1:, :] -= fx
    fy = (0.5 * (D[:, :-1] + D[:, 1:])) * (n[:, 1:] - n[:, :-1])
    lap[:, :-1] += fy
    lap[:, 1:] -= fy
    return n + P.T * (lap / (dx * dx) + nu_net * n - P.r_ei * n * n)


# ----------------------------------------------------------------------------
# Coarse <-> fine transfers (Sec. III.C, Eq. 5a/5b)
# ----------------------------------------------------------------------------
def _lin_index(pos, length):
    """Index and weight of position ``pos`` (in sample units) on a line of
    ``length`` samples, clamped to the line (constant beyond its ends)."""
    i0 = np.floor(pos).astype(np.int64)
    w = pos - i0
    lo = i0 < 0
    hi = i0 > length - 2
    i0 = np.where(lo, 0, np.where(hi, length - 2, i0))
    w = np.where(lo, 0.0, np.where(hi, 1.0, w))
    return i0, w


def linear_cfb(old_line, new_line, frac, pos):
    """Eq. 5b: L = (1-frac)[O1 (1-xp) + O2 xp]_old + frac[O1 (1-xp) + O2 xp]_new.

    ``pos`` are the fine sample positions in units of the coarse samples of
    the line (sample s sits at position s)."""
    i0, xp = _lin_index(np.asarray(pos, dtype=np.float64), len(old_line))
    lo = old_line[i0] * (1.0 - xp) + old_line[i0 + 1] * xp
    ln = new_line[i0] * (1.0 - xp) + new_line[i0 + 1] * xp
    return (1.0 - frac) * lo + frac * ln


def bilinear(F, px, py):
    """Eq. 5a at frac = 1: opposite-area weights of the four surrounding
    coarse samples.  ``px, py`` are the query positions (1-D, separable) in
    units of F's sample grid; the result has shape (len(px), len(py))."""
    i0, fu = _lin_index(np.asarray(px, dtype=np.float64), F.shape[0])
    j0, fv = _lin_index(np.asarray(py, dtype=np.float64), F.shape[1])
    fu = fu[:, None]
    fv = fv[None, :]
    return (F[np.ix_(i0, j0)] * ((1.0 - fu) * (1.0 - fv))
            + F[np.ix_(i0 + 1, j0)] * (fu * (1.0 - fv))
            + F[np.ix_(i0, j0 + 1)] * ((1.0 - fu) * fv)
            + F[np.ix_(i0 + 1, j0 + 1)] * (fu * fv))


# ----------------------------------------------------------------------------
# Flags (Sec. III.A, III.B, III.D)
# ----------------------------------------------------------------------------
def flag_mask(n, n_th, g_th, dx, dtype=None):
    """Refinement flags on the coarse nodes.

    flag = n > n_th (threshold density, Sec. III.A/III.D) OR the central
    gradient magnitude |grad n| > g_th (gradient length scale, Sec. III.B),
    the latter on interior nodes only.  The gradient test is written as
    (dn_x s)^2 + (dn_y s)^2 > 1 with s = 1/(2 dx g_th), which is the same
    test without overflowing FP32.  ``dtype`` selects the precision the
    decision is taken in.
    """
    a = np.real(n)
    if dtype is not None:
        a = a.astype(dtype)
        cast = lambda v: dtype(v)
    else:
        cast = lambda v: v
    th = a > cast(n_th)
    s = cast(1.0 / (2.0 * dx * g_th))
    gx = (a[2:, 1:-1] - a[:-2, 1:-1]) * s
    gy = (a[1:-1, 2:] - a[1:-1, :-2]) * s
    g = np.zeros_like(th)
    g[1:-1, 1:-1] = (gx * gx + gy * gy) > cast(1.0)
    return th | g


def mask_bbox(mask):
    """(i0, j0, i1, j1) of the flagged nodes, or None."""
    ii, jj = np.nonzero(mask)
    if len(ii) == 0:
        return None
    return (int(ii.min()), int(jj.min()), int(ii.max()), int(jj.max()))


def grow_rect(rect, bbox, buffer, nx, ny, lo=0):
    """Growth policy: bbox of the flags widened by ``buffer`` coarse cells,
    united with the current rectangle and clipped to the domain less a
    margin ``lo`` (the CPML layer).  The rectangle only grows (Sec. III.D)."""
    if bbox is None:
        return tuple(rect)
    c = (max(bbox[0] - buffer, lo), max(bbox[1] - buffer, lo),
         min(bbox[2] + buffer, nx - lo), min(bbox[3] + buffer, ny - lo))
    return (min(rect[0], c[0]), min(rect[1], c[1]), max(rect[2], c[2]), max(rect[3], c[3]))


def line_hits(n, rect, n_th):
    """Threshold-line test of Sec. III.D: the threshold lines are the sides
    of the fine rectangle (the coarse-fine boundary); a side is hit when the
    density exceeds the threshold density at a coarse node on it (corners
    included).  The fine boundary values are linear interpolations of these
    nodes, so the coarse nodes hold the line's maximum.  Returns
    (left, bottom, right, top) booleans, with the strict comparison n > n_th.
    ``n`` is indexed [i, j]."""
    i0, j0, i1, j1 = rect
    a = np.real(n)
    return (bool(np.any(a[i0, j0:j1 + 1] > n_th)), bool(np.any(a[i0:i1 + 1, j0] > n_th)),
            bool(np.any(a[i1, j0:j1 + 1] > n_th)), bool(np.any(a[i0:i1 + 1, j1] > n_th)))


def grow_lines(rect, hits, m_ex, m_ey, nx, ny, lo=0):
    """Expansion of Sec. III.D by threshold lines: a hit on the backward or
    forward line (left, right side) moves that side outwards by m_ex coarse
    cells along x, a hit on the lower or upper line (bottom, top) by m_ey
    along y (the paper takes m_ex > m_ey); clipped to the domain, so the
    rectangle only grows."""
    left, bottom, right, top = hits
    return (max(rect[0] - m_ex, lo) if left else rect[0],
            max(rect[1] - m_ey, lo) if bottom else rect[1],
            min(rect[2] + m_ex, nx - lo) if right else rect[2],
            min(rect[3] + m_ey, ny - lo) if top else rect[3])


# ----------------------------------------------------------------------------
# Simulation driver: coarse mesh + one growing fine rectangle
# ----------------------------------------------------------------------------
class Sim:
    """DMR run (Sec. III.C-III.D); r = 1 is the uniform mesh.

    Per coarse step (Sec. III.C):
      1. keep the coarse tangential E of the coarse-fine boundary lines (old);
      2. coarse EM step (Mur on the domain edges);
      3. r fine EM steps; fine tangential E on interior rectangle sides from
         Eq. 5b with frac = k/r, Mur on sides lying on the domain edge;
         fine S2 accumulated after each sub-step;
      4. fine -> coarse: every coarse E edge in the closed rectangle except the
         tangential edges of interior sides becomes the mean of its r
         collinear fine edges (reading of "transferred back");
      5. coarse S2 accumulated.
    After every N_T coarse steps (one period): coarse continuity step, fine
    continuity step with the fine nodes of interior sides set from the new
    coarse density by Eq. 5b (frac = 1), injection of the fine density into
    the coarse nodes of the closed rectangle, FP64 totals, flags and growth.
    """

    def __init__(self, cfg: dict, rect=None, dtype=np.float64):
        P = Params(cfg)
        self.P = P
        self.dtype = dtype
        self.coarse = Mesh(P, P.nx, P.ny, 1, dtype=dtype)
        self.coarse.pml = CPML(self.coarse, P.pml_cells, dtype) if P.boundary == 1 else None
        self.cbc = "cpml" if P.boundary == 1 else "mur"
        self.fine = None
        self.rect = None
        self.period = 0
        self.log = []            # rect after each period
        self.masks = []          # flag mask after each period
        self.replay = None
        self.stats_hist = []
        self.N_e = 0.0
        self.P_abs = 0.0
        self.W_abs = 0.0
        if P.r > 1:
            if rect is None:
                raise ValueError("a DMR run (r > 1) needs an initial rectangle")
            self._make_fine(tuple(rect))

    # -- set-up --------------------------------------------------------------
    def _make_fine(self, rect):
        P = self.P
        i0, j0, i1, j1 = rect
        k = P.rect_margin
        if not (k <= i0 < i1 <= P.nx - k and k <= j0 < j1 <= P.ny - k):
            raise ValueError("bad rectangle %r (margin %d)" % (rect, k))
        if P.r * P.r * (i1 - i0) * (j1 - j0) > P.cap:
            raise CapacityError("patch %r exceeds the capacity" % (rect,))
        self.rect = rect
        self.fine = Mesh(P, P.r * (i1 - i0), P.r * (j1 - j0), P.r,
                         gi0=P.r * i0, gj0=P.r * j0, dtype=self.dtype)

    def seed_gaussian(self, n0, x0, y0, sx, sy, add=False):
        """Gaussian seed n0 exp(-((x-x0)^2/sx^2 + (y-y0)^2/sy^2)) at the nodes
        (Sec. IV); zero where the exponent is below -60 (reading).  With
        ``add`` the Gaussian is added to the present density (several seeds)."""
        for mesh in (self.coarse, self.fine):
            if mesh is None:
                continue
            ax = (mesh.node_x() - x0) ** 2 / sx ** 2
            ay = (mesh.node_y() - y0) ** 2 / sy ** 2
            arg = ax[:, None] + ay[None, :]
            g = np.where(arg <= 60.0, n0 * np.exp(-np.minimum(arg, 60.0)), 0.0)
            if add:
                mesh.n[...] = mesh.n + g
            else:
                mesh.n[...] = g
        self._inject()

    def seed_map(self, nmap, a0, b0):
        """Set the fine nodes [a0, a0+mx) x [b0, b0+my) of the rectangle to the
        given density map (a seed given as a node map), then inject into the
        coarse nodes."""
        nmap = np.asarray(nmap)
        mx, my = nmap.shape
        self.fine.n[a0:a0 + mx, b0:b0 + my] = nmap
        self._inject()

    def _inject(self):
        """Fine density -> coarse nodes of the closed rectangle (direct copy
        where nodes coincide, Sec. III.C)."""
        if self.fine is None:
            return
        r = self.P.r
        i0, j0, i1, j1 = self.rect
        self.coarse.n[i0:i1 + 1, j0:j1 + 1] = self.fine.n[::r, ::r]

    def _sides(self):
        P = self.P
        i0, j0, i1, j1 = self.rect
        return {"left": i0 == 0, "right": i1 == P.nx, "bottom": j0 == 0, "top": j1 == P.ny}

    # -- EM ------------------------------------------------------------------
    def coarse_step(self):
        P = self.P
        c = self.coarse
        if self.fine is None:
            em_step(P, c, bc=self.cbc)
            accumulate_e2(P, c)
        else:
            f = self.fine
            r = P.r
            i0, j0, i1, j1 = self.rect
            old = {"bottom": c.Ex[:, j0].copy(), "top": c.Ex[:, j1].copy(),
                   "left": c.Ey[i0, :].copy(), "right": c.Ey[i1, :].copy()}
            em_step(P, c, bc=self.cbc)
            new = {"bottom": c.Ex[:, j0], "top": c.Ex[:, j1],
                   "left": c.Ey[i0, :], "right": c.Ey[i1, :]}
            on_edge = self._sides()
            # fine tangential sample b sits at coarse position start + (b+1/2)/r;
            # coarse tangential sample s sits at s + 1/2.
            px = i0 + (np.arange(f.nx) + 0.5) / r - 0.5
            py = j0 + (np.arange(f.ny) + 0.5) / r - 0.5
            for k in range(1, r + 1):
                frac = k / r
                sides = {}
                for side, pos in (("bottom", px), ("top", px), ("left", py), ("right", py)):
                    sides[side] = "mur" if on_edge[side] else linear_cfb(old[side], new[side], frac, pos)
                em_step(P, f, sides)
                accumulate_e2(P, f)
            if P.coupling == 0:
                self._restrict_e()
            accumulate_e2(P, c)
        if c.m % P.N_T == 0:
            self._period_end()

    def _restrict_e(self):
        """Coarse E edges of the closed rectangle (except tangential edges of
        interior sides) = mean of the r collinear fine edges (Sec. III.C)."""
        P = self.P
        c, f, r = self.coarse, self.fine, P.r
        i0, j0, i1, j1 = self.rect
        on_edge = self._sides()
        jlo = j0 if on_edge["bottom"] else j0 + 1
        jhi = j1 if on_edge["top"] else j1 - 1
        if jhi >= jlo:
            acc = f.Ex[0::r, r * (jlo - j0):r * (jhi - j0) + 1:r].copy()
            for q in range(1, r):
                acc = acc + f.Ex[q::r, r * (jlo - j0):r * (jhi - j0) + 1:r]
            c.Ex[i0:i1, jlo:jhi + 1] = acc / r
        ilo = i0 if on_edge["left"] else i0 + 1
        ihi = i1 if on_edge["right"] else i1 - 1
        if ihi >= ilo:
            acc = f.Ey[r * (ilo - i0):r * (ihi - i0) + 1:r, 0::r].copy()
            for q in range(1, r):
                acc = acc + f.Ey[r * (ilo - i0):r * (ihi - i0) + 1:r, q::r]
            c.Ey[ilo:ihi + 1, j0:j1] = acc / r

    def advance(self, n_steps):
        for _ in range(int(n_steps)):
            self.coarse_step()

    # -- period end ------------------------------------------------------------
    def _weights(self):
        """Composite trapezoid weights: the coarse mesh outside the rectangle
        and the fine mesh inside it (used by the FP64 totals)."""
        P = self.P
        wx = np.ones(P.nx + 1)
        wx[[0, -1]] = 0.5
        wy = np.ones(P.ny + 1)
        wy[[0, -1]] = 0.5
        wc = wx[:, None] * wy[None, :]
        wf = None
        if self.fine is not None:
            i0, j0, i1, j1 = self.rect
            px = np.zeros(P.nx + 1)
            px[i0:i1 + 1] = 1.0
            px[[i0, i1]] = 0.5
            py = np.zeros(P.ny + 1)
            py[j0:j1 + 1] = 1.0
            py[[j0, j1]] = 0.5
            wc = wc - px[:, None] * py[None, :]
            qx = np.ones(self.fine.nx + 1)
            qx[[0, -1]] = 0.5
            qy = np.ones(self.fine.ny + 1)
            qy[[0, -1]] = 0.5
            wf = qx[:, None] * qy[None, :]
        return wc, wf

    def _period_end(self):
        P = self.P
        c, f = self.coarse, self.fine
        wc, wf = self._weights()
        heat = QE * QE / (ME * P.nu_m)
        # E_rms of the completed period, E_rms^2 = S2 / N (the mean over the
        # period's N samples, the same quantity E_eff is taken from)
        c.erms_last = np.sqrt(c.S2 / c.N)
        if f is not None:
            f.erms_last = np.sqrt(f.S2 / f.N)
        # coarse continuity step
        eeff_c, nu_c, D_c = density_rates(P, c, c.n)
        p_abs = c.dx * c.dx * np.sum(wc * c.n * heat * eeff_c * eeff_c)
        n_c_new = continuity_update(P, c.n, D_c, nu_c, c.dx)
        c.S2[...] = 0.0
        c.n = n_c_new
        if f is not None:
            eeff_f, nu_f, D_f = density_rates(P, f, f.n)
            p_abs = p_abs + f.dx * f.dx * np.sum(wf * f.n * heat * eeff_f * eeff_f)
            n_f_new = continuity_update(P, f.n, D_f, nu_f, f.dx)
            # fine nodes on interior sides take the new coarse density (Eq. 5b, frac = 1)
            r = P.r
            i0, j0, i1, j1 = self.rect
            on_edge = self._sides()
            pa = i0 + np.arange(f.nx + 1) / r
            pb = j0 + np.arange(f.ny + 1) / r
            if not on_edge["bottom"]:
                n_f_new[:, 0] = linear_cfb(n_c_new[:, j0], n_c_new[:, j0], 1.0, pa)
            if not on_edge["top"]:
                n_f_new[:, -1] = linear_cfb(n_c_new[:, j1], n_c_new[:, j1], 1.0, pa)
            if not on_edge["left"]:
                n_f_new[0, :] = linear_cfb(n_c_new[i0, :], n_c_new[i0, :], 1.0, pb)
            if not on_edge["right"]:
                n_f_new[-1, :] = linear_cfb(n_c_new[i1, :], n_c_new[i1, :], 1.0, pb)
            f.S2[...] = 0.0
            f.n = n_f_new
            self._inject()
        # FP64 totals: electrons per unit depth and period-mean absorbed power
        n_e = c.dx * c.dx * np.sum(wc * c.n)
        if f is not None:
            n_e = n_e + f.dx * f.dx * np.sum(wf * f.n)
        self.N_e = n_e
        self.P_abs = p_abs
        self.W_abs = self.W_abs + p_abs * P.T
        self.period += 1
        # flags and growth (Sec. III.D)
        if f is not None:
            mask = flag_mask(c.n, P.n_th, P.g_th, c.dx)
            self.masks.append(mask)
            if self.replay is not None:
                new_rect = tuple(self.replay[self.period - 1])
            elif P.growth == 2:
                new_rect = grow_lines(self.rect, line_hits(c.n, self.rect, P.n_th),
                                      P.m_ex, P.m_ey, P.nx, P.ny, P.rect_margin)
            elif P.growth:
                new_rect = grow_rect(self.rect, mask_bbox(mask), P.buffer, P.nx, P.ny,
                                     P.rect_margin)
            else:
                new_rect = self.rect
            if new_rect != self.rect:
                self._expand(new_rect)
            self.log.append(self.rect)
        self.stats_hist.append(self.stats())

    def _expand(self, new_rect):
        """Grow the rectangle (Sec. III.D): fine data of the old rectangle are
        copied to the same places, the rest of the new rectangle is filled by
        bilinear interpolation of the coarse data (Eq. 5a, frac = 1); S2 is
        zero (growth happens right after the period's reset)."""
        P = self.P
        r = P.r
        old, orect = self.fine, self.rect
        self._make_fine(tuple(new_rect))
        f, c = self.fine, self.coarse
        i0, j0, _, _ = new_rect
        oi = r * (orect[0] - i0)
        oj = r * (orect[1] - j0)
        fa = np.arange(f.nx + 1)
        fb = np.arange(f.ny + 1)
        ax_node = i0 + fa / r
        ax_half = i0 + (fa[:-1] + 0.5) / r
        by_node = j0 + fb / r
        by_half = j0 + (fb[:-1] + 0.5) / r
        # coarse sample grids: Ex (i+1/2, j), Ey (i, j+1/2), Hz (i+1/2, j+1/2), n (i, j)
        f.Ex[...] = bilinear(c.Ex, ax_half - 0.5, by_node)
        f.vx[...] = bilinear(c.vx, ax_half - 0.5, by_node)
        f.Ey[...] = bilinear(c.Ey, ax_node, by_half - 0.5)
        f.vy[...] = bilinear(c.vy, ax_node, by_half - 0.5)
        f.Hz[...] = bilinear(c.Hz, ax_half - 0.5, by_half - 0.5)
        f.n[...] = bilinear(c.n, ax_node, by_node)
        f.erms_last = bilinear(c.erms_last, ax_node, by_node)
        for name in ("Ex", "vx", "Ey", "vy", "Hz", "n", "erms_last"):
            src = getattr(old, name)
            getattr(f, name)[oi:oi + src.shape[0], oj:oj + src.shape[1]] = src
        f.m = old.m

    # -- outputs -----------------------------------------------------------------
    def stats(self):
        P = self.P
        c = self.coarse
        fine_cells = 0 if self.fine is None else self.fine.nx * self.fine.ny
        R = fine_cells / float(P.r * P.r * P.nx * P.ny) if self.fine is not None else 0.0
        return {"t": c.m * c.dt, "R": R, "fine_cells": fine_cells, "N_e": self.N_e,
                "P_abs": self.P_abs, "W_abs": self.W_abs, "periods": self.period,
                "coarse_steps": c.m}

    def erms(self, level=0):
        """E_rms at the nodes (the output E_rms(x, y, t), Sec. II.B, Sec. IV).

        Reading: within a period, the RMS of the total field over the samples
        taken since the period began (levels after the period's first, through
        the present E level: E_rms^2 = S2 / q for q samples); at a period
        boundary, where S2 has just been reset, the E_rms of the period just
        completed, E_rms^2 = S2 / N over its N samples.  Area that the
        rectangle gained at that boundary takes the coarse values by the
        bilinear fill of Eq. 5a, like every other fine quantity."""
        mesh = self.coarse if level == 0 else self.fine
        q = mesh.m % mesh.N
        if q == 0:
            return mesh.erms_last.copy()
        return np.sqrt(mesh.S2 / q)


def default_patch(nx, ny, ic, jc, m):
    """An m x m coarse-cell rectangle centred on coarse node (ic, jc), shifted
    inward so that it stays inside the domain."""
    i0 = min(max(ic - m // 2, 0), nx - m)
    j0 = min(max(jc - m // 2, 0), ny - m)
    return (i0, j0, i0 + m, j0 + m)


def sim_from_workload(w, dtype=np.float64, cfg_overrides=None, rect=None):
    """Build and seed a Sim from a workload dict (parameters + seeds given as
    domain fractions and widths in wavelengths)."""
    cfg = dict(w["cfg"])
    if cfg_overrides:
        cfg.update(cfg_overrides)
    sim = Sim(cfg, rect=rect if rect is not None else w.get("rect"), dtype=dtype)
    P = sim.P
    Lx, Ly = P.nx * P.dxc, P.ny * P.dxc
    for q, (n0, fx, fy, sxl, syl) in enumerate(w["seeds"]):
        sim.seed_gaussian(n0, fx * Lx, fy * Ly, sxl * P.lam, syl * P.lam, add=q > 0)
    return sim
