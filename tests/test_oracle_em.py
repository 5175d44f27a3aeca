"""Pins of the oracle's EM update (Eqs. 1-3) against closed forms and
invariants that do not come from the oracle itself."""
import math

import numpy as np
import pytest

from oracle import dmr_oracle as O
from paper_2105_13276_gb300 import workloads as W

# CODATA 2018, typed independently of the oracle module.
c_light = 299792458.0
mu0 = 1.25663706212e-6
eps0 = 8.8541878128e-12
q_e = 1.602176634e-19
m_e = 9.1093837015e-31


def vacuum_cfg(nx, ny, **kw):
    return W.base_cfg(nx=nx, ny=ny, r=1, n_lambda=32, steps_per_period=64, E0=0.0, **kw)


def test_p1_vacuum_scattered_field_stays_zero():
    """P1: with n = 0 the plasma current vanishes, so the scattered field of
    the scattered-field formulation stays identically zero (the incident wave
    is analytic), on the uniform mesh and on a DMR mesh."""
    for r, rect in ((1, None), (2, (4, 3, 12, 10))):
        cfg = W.base_cfg(nx=16, ny=14, r=r, n_lambda=16, steps_per_period=32, E0=5e6)
        sim = O.Sim(cfg, rect=rect)
        sim.advance(70)
        for mesh in (sim.coarse, sim.fine):
            if mesh is None:
                continue
            for a in (mesh.Ex, mesh.Ey, mesh.Hz):
                assert np.all(a == 0.0)


def _te_mode(nx, ny, m, n, dx, dt, H0=1.0):
    Lx, Ly = nx * dx, ny * dx
    kx, ky = m * math.pi / Lx, n * math.pi / Ly
    Kx = 2.0 * math.sin(kx * dx / 2) / dx
    Ky = 2.0 * math.sin(ky * dx / 2) / dx
    # discrete Yee dispersion: (2/dt sin(w dt/2))^2 = (Kx^2 + Ky^2)/(mu0 eps0)
    Wd = math.sqrt((Kx * Kx + Ky * Ky) / (mu0 * eps0))
    w = 2.0 / dt * math.asin(Wd * dt / 2.0)
    A = -H0 * Ky / (eps0 * Wd)
    B = H0 * Kx / (eps0 * Wd)
    xc = (np.arange(nx) + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * dx
    xn = np.arange(nx + 1) * dx
    yn = np.arange(ny + 1) * dx

    def fields(level):
        t_e = level * dt
        t_h = (level - 0.5) * dt
        Hz = H0 * math.cos(w * t_h) * np.outer(np.cos(kx * xc), np.cos(ky * yc))
        Ex = A * math.sin(w * t_e) * np.outer(np.cos(kx * xc), np.sin(ky * yn))
        Ey = B * math.sin(w * t_e) * np.outer(np.sin(kx * xn), np.cos(ky * yc))
        return Ex, Ey, Hz

    return fields, w


@pytest.mark.parametrize("mode", [(1, 1), (3, 2), (5, 7)])
def test_p3_yee_dispersion_pec_eigenmode(mode):
    """P3: a discrete TE_mn eigenmode of a PEC box oscillates at the Yee
    numerical frequency sin^2(w dt/2)/(c dt)^2 = sum sin^2(k d/2)/d^2."""
    nx, ny = 24, 18
    P = O.Params(vacuum_cfg(nx, ny))
    mesh = O.Mesh(P, nx, ny, 1)
    fields, w = _te_mode(nx, ny, *mode, mesh.dx, mesh.dt)
    Ex, Ey, Hz = fields(0)
    mesh.Ex[...], mesh.Ey[...], mesh.Hz[...] = Ex, Ey, Hz
    steps = 1000
    for _ in range(steps):
        O.em_step(P, mesh, bc="pec")
    Ex, Ey, Hz = fields(steps)
    # amplitudes: H0 = 1 A/m, E ~ eta H0
    scaleE = math.sqrt(mu0 / eps0)
    assert np.abs(mesh.Hz - Hz).max() < 1e-10
    assert np.abs(mesh.Ex - Ex).max() / scaleE < 1e-10
    assert np.abs(mesh.Ey - Ey).max() / scaleE < 1e-10
    # the numerical frequency approaches the continuum one as d -> 0
    kx = mode[0] * math.pi / (nx * mesh.dx)
    ky = mode[1] * math.pi / (ny * mesh.dx)
    kd = math.hypot(kx, ky) * mesh.dx
    assert abs(w / (c_light * math.hypot(kx, ky)) - 1.0) < kd * kd / 12.0


def test_p4_pec_cavity_energy_invariant():
    """P4: for Yee in a PEC box, eps0 sum E^n.E^n + mu0 sum H^{n-1/2} H^{n+1/2}
    is exactly conserved (up to rounding)."""
    nx, ny = 20, 16
    P = O.Params(vacuum_cfg(nx, ny))
    mesh = O.Mesh(P, nx, ny, 1)
    mesh.Ex[...] = W.random_fields(mesh.Ex.shape, 1, 1e3)
    mesh.Ey[...] = W.random_fields(mesh.Ey.shape, 2, 1e3)
    mesh.Hz[...] = W.random_fields(mesh.Hz.shape, 3, 1e3 / 377.0)
    mesh.Ex[:, 0] = mesh.Ex[:, -1] = 0.0
    mesh.Ey[0, :] = mesh.Ey[-1, :] = 0.0
    energies = []
    for _ in range(300):
        e2 = np.sum(mesh.Ex ** 2) + np.sum(mesh.Ey ** 2)
        h_old = mesh.Hz.copy()
        O.em_step(P, mesh, bc="pec")
        energies.append(eps0 * e2 + mu0 * np.sum(h_old * mesh.Hz))
    energies = np.array(energies)
    assert np.abs(energies - energies[0]).max() / energies[0] < 1e-12


def _plasma_closed_form(Einit, steps, dt, n, nu_m):
    a = (1 - nu_m * dt / 2) / (1 + nu_m * dt / 2)
    b = (q_e * dt / m_e) / (1 + nu_m * dt / 2)
    c = dt * q_e * n / eps0
    # x_{k+1} = M x_k with x = (v_{k-1/2}, E_k), M = [[a, -b], [c a, 1 - c b]]
    tr = a + 1 - c * b
    disc = complex(tr * tr - 4 * a) ** 0.5
    l1, l2 = (tr + disc) / 2, (tr - disc) / 2
    E1 = (1 - c * b) * Einit
    alpha = (E1 - l2 * Einit) / (l1 - l2)
    beta = Einit - alpha
    k = np.arange(steps + 1)
    return np.real(alpha * l1 ** k + beta * l2 ** k), l1


@pytest.mark.parametrize("p_torr", [1.0, 700.0])
def test_p5_uniform_plasma_oscillation(p_torr):
    """P5: uniform plasma, uniform Ex, no incident field.  Far from the walls
    the (v, E) pair follows the 2x2 recurrence whose eigenvalues are closed
    form; with nu_m -> 0 the discrete frequency obeys sin(th/2) = w_p dt/2."""
    nx, ny = 8, 200
    cfg = W.base_cfg(nx=nx, ny=ny, r=1, n_lambda=32, steps_per_period=64, E0=0.0, p_torr=p_torr)
    P = O.Params(cfg)
    mesh = O.Mesh(P, nx, ny, 1)
    wp_dt = 0.3
    n_p = (wp_dt / mesh.dt) ** 2 * m_e * eps0 / q_e ** 2
    mesh.n[...] = n_p
    mesh.Ex[...] = 1e5
    steps = 90
    hist = [mesh.Ex[3, ny // 2]]
    for _ in range(steps):
        O.em_step(P, mesh)
        hist.append(mesh.Ex[3, ny // 2])
    ref, l1 = _plasma_closed_form(1e5, steps, mesh.dt, n_p, 5.3e9 * p_torr)
    assert np.abs(np.array(hist) - ref).max() < 1e-9 * 1e5
    if p_torr == 1.0:
        theta = abs(np.angle(l1))
        assert abs(math.sin(theta / 2) - wp_dt / 2) < 1e-3 * wp_dt


def test_mur_absorbs_normal_plane_wave():
    """First-order Mur at normal incidence: a y-uniform scattered pulse
    leaving through the right edge is absorbed to well below 1% in energy."""
    nx, ny = 200, 6
    P = O.Params(vacuum_cfg(nx, ny))
    mesh = O.Mesh(P, nx, ny, 1)
    xn = np.arange(nx + 1) * mesh.dx
    xc = (np.arange(nx) + 0.5) * mesh.dx
    x0, s = 100 * mesh.dx, 8 * mesh.dx
    # right-going pulse Ey = f(x - ct), Hz = f(x - ct)/eta (Faraday), H half a step back
    eta = math.sqrt(mu0 / eps0)
    mesh.Ey[...] = np.exp(-((xn - x0) / s) ** 2)[:, None]
    mesh.Hz[...] = (np.exp(-((xc + 0.5 * c_light * mesh.dt - x0) / s) ** 2) / eta)[:, None]
    e0 = np.sum(mesh.Ey ** 2)
    for _ in range(600):
        O.em_step(P, mesh)
    assert np.sum(mesh.Ey ** 2) < 1e-2 * e0


def _pulse_run(nx, boundary, steps, L=8):
    cfg = W.base_cfg(nx=nx, ny=nx, r=1, n_lambda=16, steps_per_period=32, E0=0.0,
                     boundary=boundary, pml_cells=L)
    sim = O.Sim(cfg)
    c = sim.coarse
    xc = (np.arange(nx) + 0.5 - nx / 2.0)
    c.Hz[...] = np.exp(-(xc[:, None] ** 2 + xc[None, :] ** 2) / (2 * 2.0 ** 2))
    for _ in range(steps):
        sim.coarse_step()
    return c.Hz


def test_cpml_absorbs_far_better_than_mur():
    """Outer boundary (§8(f) next 3): a divergence-free Hz pulse leaves a
    64x64 domain; after the reflections would have come back, the interior
    (outside the 8-cell layer) is compared with the same region of a 320x320
    run whose edges are too far to matter.  CPML leaves a small fraction of
    Mur's error, and a small error in absolute terms."""
    nx, big, steps, L = 64, 320, 130, 8
    ref = _pulse_run(big, 0, steps)
    o = (big - nx) // 2
    ref = ref[o:o + nx, o:o + nx]
    err = {}
    for b in (0, 1):
        hz = _pulse_run(nx, b, steps, L)
        err[b] = np.abs(hz - ref)[L:nx - L, L:nx - L].max()
    assert err[1] < 0.05 * err[0], err
    assert err[1] < 2e-3, err


def test_cpml_late_time_stays_bounded():
    """A long CPML run empties the domain and stays empty (no growing mode)."""
    hz = _pulse_run(48, 1, 1500)
    assert np.abs(hz).max() < 1e-3
