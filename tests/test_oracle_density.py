"""Pins of the oracle's E_eff / continuity step (Eq. 4) against numbers the
paper prints and closed forms of the discrete scheme."""
import json
import math
import os

import numpy as np
import pytest

from oracle import dmr_oracle as O
from paper_2105_13276_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))

q_e = 1.602176634e-19
m_e = 9.1093837015e-31
eps0 = 8.8541878128e-12


def _mesh_with_uniform_s2(cfg, erms, nx=12, ny=10):
    P = O.Params(cfg)
    mesh = O.Mesh(P, nx, ny, 1)
    mesh.S2[...] = erms * erms * mesh.N
    return P, mesh


def test_paper_e_eff_worked_example():
    """Sec. IV.D: w ~ 6e11, nu_m ~ 4e12 and E_rms = 3.5 MV/m give
    E_eff ~ 3.46 MV/m (local-field approximation reading)."""
    g = GOLD["e_eff_worked_example"]
    cfg = W.base_cfg(freq=g["omega"] / (2 * math.pi), p_torr=g["nu_m"] / 5.3e9)
    P, mesh = _mesh_with_uniform_s2(cfg, g["E_rms"])
    eeff, _, _ = O.density_rates(P, mesh, mesh.n)
    assert np.allclose(eeff, g["E_eff"], rtol=g["rel_tol"])


def test_p2_incident_rms_and_e_eff():
    """P2: with n = 0, one period of N equispaced samples of the incident
    field gives E_rms^2 = E0^2/2 exactly (sum of sin^2 over a full period), so
    E_rms = E0/sqrt(2) (Sec. IV.D: 5 MV/m -> 3.5 MV/m rms)."""
    g = GOLD["incident_rms"]
    cfg = W.base_cfg(nx=10, ny=6, r=1, n_lambda=16, steps_per_period=32, E0=g["E0"], p_torr=760.0)
    P = O.Params(cfg)
    mesh = O.Mesh(P, 10, 6, 1)
    for _ in range(mesh.N):
        O.em_step(P, mesh)
        O.accumulate_e2(P, mesh)
    erms = np.sqrt(mesh.S2 / mesh.N)
    assert np.abs(erms - g["E0"] / math.sqrt(2)).max() < 1e-9 * g["E0"]
    assert abs(erms.mean() - g["E_rms"]) / g["E_rms"] < g["rel_tol"]
    eeff, _, _ = O.density_rates(P, mesh, mesh.n)
    expect = g["E0"] / math.sqrt(2) / math.sqrt(1 + (2 * math.pi * 110e9 / (5.3e9 * 760)) ** 2)
    assert np.allclose(eeff, expect, rtol=1e-12)
    assert abs(expect - 3.4846e6) < 1e2


def test_cutoff_density_and_nu_m():
    """Sec. III.A / IV.D: n_cutoff = n_crit nu_m / w ~ 9e20 m^-3 at 110 GHz,
    1 atm, which fixes n_crit = m eps0 w^2/e^2; Sec. II.A nu_m = 5.3e9 p."""
    g = GOLD["cutoff_density"]
    P = O.Params(W.base_cfg(freq=g["freq"], p_torr=g["p_torr"]))
    assert abs(P.nu_m - GOLD["nu_m_air"]["nu_m"]) / P.nu_m < GOLD["nu_m_air"]["rel_tol"]
    n_cut = P.n_crit * P.nu_m / P.omega
    assert abs(n_cut - g["n_cutoff"]) / g["n_cutoff"] < g["rel_tol"]
    # default refinement threshold is 1e-3 n_crit
    assert abs(P.n_th - 1.5009e17) / 1.5009e17 < 1e-3


def test_ionization_magnitudes_match_paper_range():
    """Sec. IV.D: nu_i of order 0.18e9 - 1.3e9 s^-1 at E_eff ~ 3.46 MV/m and
    above, 1 atm; small near the breakdown field E_cr ~ 2.5 MV/m rms.  This
    pins the chosen nu_i fit only to order of magnitude."""
    g = GOLD["ionization_range"]
    P = O.Params(W.base_cfg(p_torr=g["p_torr"]))
    nu = O.ionization_frequency(P, np.array([g["E_eff_example"], 4.0e6]))
    assert g["nu_low"] <= nu[0] <= g["nu_high"]
    assert nu[1] > nu[0]
    e_cr_eff = g["E_cr_rms"] / math.sqrt(1 + (P.omega / P.nu_m) ** 2)
    nu_cr = O.ionization_frequency(P, np.array([e_cr_eff]))[0]
    assert nu_cr < 0.2 * nu[0]
    assert O.ionization_frequency(P, np.array([0.0]))[0] == 0.0


def test_townsend_form_stoletov_point_and_saturation():
    """Townsend coefficient set (Sec. II.A, gamma = A p exp(-B p/E_eff),
    v_d = mu_e E_eff): properties of the form, not a retyped formula.
    - ionization per volt gamma/E = nu_i/(mu_e E^2) peaks at E = B p (the
      Stoletov point) with value A/(B e);
    - at high field gamma saturates to A p;
    - nu_i scales with s_nu and vanishes at E_eff = 0."""
    cfg = W.base_cfg(nu_model=1, town_A=1500.0, town_B=36500.0, p_torr=300.0)
    P = O.Params(cfg)
    mu = O.QE / (O.ME * P.nu_m)
    E = np.linspace(0.2, 5.0, 200001) * P.town_B * P.p
    eta = O.ionization_frequency(P, E) / (mu * E * E)
    k = int(np.argmax(eta))
    assert abs(E[k] / (P.town_B * P.p) - 1.0) < 1e-4
    assert abs(eta[k] / (P.town_A / (P.town_B * math.e)) - 1.0) < 1e-9
    big = 1e6 * P.town_B * P.p
    assert abs(O.ionization_frequency(P, np.array([big]))[0] / (mu * big) / (P.town_A * P.p) - 1) < 2e-6
    assert O.ionization_frequency(P, np.array([0.0]))[0] == 0.0
    P2 = O.Params(dict(cfg, nu_scale=2.5))
    e = np.array([3e6])
    assert abs(O.ionization_frequency(P2, e)[0] / O.ionization_frequency(P, e)[0] - 2.5) < 1e-15
    # the default fit is unchanged by the new switch
    Pf = O.Params(W.base_cfg(p_torr=300.0))
    assert Pf.nu_model == 0


def test_effective_diffusion_limits():
    """D_eff = (alpha D_e + D_a)/(1 + alpha), alpha = nu_i nu_m / w_p^2:
    free diffusion where there are no electrons, ambipolar in dense plasma,
    and D_e where both rates vanish."""
    cfg = W.base_cfg(p_torr=760.0)
    P, mesh = _mesh_with_uniform_s2(cfg, 3.5e6)
    n = np.zeros_like(mesh.n)
    n[0, 0] = 1e24
    n[1, 1] = 1e10
    _, nu, D = O.density_rates(P, mesh, n)
    assert D[2, 2] == P.De
    assert abs(D[0, 0] - P.Da) / P.Da < 1e-3
    assert abs(D[1, 1] - P.De) / P.De < 1e-6
    mesh.S2[...] = 0.0
    _, _, D0 = O.density_rates(P, mesh, np.zeros_like(mesh.n))
    assert np.all(D0 == P.De)
    # front value of the paper (~0.087 m^2/s) lies between the two limits
    assert P.Da < GOLD["front_diffusion"]["D_eff"] < P.De * 1.2


def test_p7_growth_euler_recurrence_and_exponential():
    """P7: no diffusion, no recombination, uniform E_eff: n_k = n0 (1 + nu T)^k
    exactly, and n0 exp(nu t) within the Euler bound k (nu T)^2 / 2."""
    cfg = W.base_cfg(De=0.0, Da=0.0, beta_rec=0.0, p_torr=760.0)
    P, mesh = _mesh_with_uniform_s2(cfg, 3.5e6)
    n = np.full_like(mesh.n, 1e15)
    _, nu, D = O.density_rates(P, mesh, n)
    nu0 = float(nu[0, 0])
    assert np.all(nu == nu0) and np.all(D == 0.0)
    for _ in range(200):
        n = O.continuity_update(P, n, D, nu, mesh.dx)
    expect = 1e15 * (1 + nu0 * P.T) ** 200
    assert np.abs(n / expect - 1).max() < 1e-12
    x = nu0 * P.T
    assert abs(n[0, 0] / (1e15 * math.exp(200 * x)) - 1) < 200 * x * x / 2 * 1.01


def test_p7_growth_full_system_small_density():
    """P7 through the whole time step: a density too small to perturb the
    field (scattered field ~1e-14 of E0) grows by (1 + nu(E_eff) T) per period
    at every node, with E_eff that of the incident wave."""
    cfg = W.base_cfg(nx=12, ny=10, r=1, n_lambda=16, steps_per_period=32, p_torr=760.0,
                     De=0.0, Da=0.0, beta_rec=0.0)
    sim = O.Sim(cfg)
    sim.coarse.n[...] = 1e8
    sim.advance(3 * 32)
    P = sim.P
    e_eff = 5e6 / math.sqrt(2) / math.sqrt(1 + (P.omega / P.nu_m) ** 2)
    nu = 5.14e11 * 760.0 * math.exp(-73.0 * (e_eff / (100 * 760.0)) ** -0.44)
    assert np.abs(sim.coarse.n / (1e8 * (1 + nu * P.T) ** 3) - 1).max() < 1e-9


@pytest.mark.parametrize("m", [1, 3, 7])
def test_p8_diffusion_fourier_mode(m):
    """P8: constant D, no reactions: the zero-flux discrete cosine mode
    cos(pi m (i+1/2)/(N+1)) decays by exactly 1 - 4 D T/d^2 sin^2(pi m/(2(N+1)))
    per step."""
    D = 0.1
    cfg = W.base_cfg(De=D, Da=D, beta_rec=0.0, nu_scale=0.0)
    P = O.Params(cfg)
    nx, ny = 30, 4
    mesh = O.Mesh(P, nx, ny, 1)
    i = np.arange(nx + 1)
    mode = np.cos(math.pi * m * (i + 0.5) / (nx + 1))
    n = (1e16 + 1e15 * mode)[:, None] * np.ones((1, ny + 1))
    Dm = np.full_like(n, D)
    nu = np.zeros_like(n)
    g = 1 - 4 * D * P.T / mesh.dx ** 2 * math.sin(math.pi * m / (2 * (nx + 1))) ** 2
    for _ in range(50):
        n = O.continuity_update(P, n, Dm, nu, mesh.dx)
    expect = (1e16 + 1e15 * g ** 50 * mode)[:, None]
    assert np.abs(n - expect).max() < 1e-12 * 1e16


def test_p8_gaussian_spreading_second_order():
    """P8: a 1-D Gaussian under constant D spreads as sigma^2 -> sigma^2 + 4 D t
    (for exp(-x^2/sigma^2)), amplitude sigma0/sigma; the discrete error falls
    by ~4x when the mesh is halved."""
    errs = []
    for nl in (64, 128):
        D = 0.1
        cfg = W.base_cfg(n_lambda=nl, steps_per_period=2 * nl, De=D, Da=D, beta_rec=0.0,
                         nu_scale=0.0)
        P = O.Params(cfg)
        L = 4 * P.lam
        nx = int(round(L / P.dxc))
        x = np.arange(nx + 1) * P.dxc - L / 2
        s0 = 0.2 * P.lam
        n = np.exp(-x ** 2 / s0 ** 2)[:, None] * np.ones((1, 3))
        steps = 4000
        for _ in range(steps):
            n = O.continuity_update(P, n, np.full_like(n, D), np.zeros_like(n), P.dxc)
        t = steps * P.T
        s2 = s0 ** 2 + 4 * D * t
        exact = math.sqrt(s0 ** 2 / s2) * np.exp(-x ** 2 / s2)
        errs.append(np.abs(n[:, 1] - exact).max())
    assert errs[0] < 1e-3
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_p10_recombination_only():
    """P10: recombination alone follows dn/dt = -r n^2, solution
    1/(1/n0 + r t); forward Euler stays within its first-order bound."""
    cfg = W.base_cfg(nu_scale=0.0, De=0.0, Da=0.0, beta_rec=1.0, Te=300.0)
    P = O.Params(cfg)
    n0 = 1e21
    n = np.full((4, 4), n0)
    zero = np.zeros_like(n)
    steps = 300
    for _ in range(steps):
        n = O.continuity_update(P, n, zero, zero, 1e-4)
    exact = 1.0 / (1.0 / n0 + 1e-13 * steps * P.T)
    h = 1e-13 * n0 * P.T
    assert abs(n[0, 0] / exact - 1) < 2 * h
    assert n[0, 0] < n0


def test_absorbed_power_matches_harmonic_conductivity():
    """The period-mean absorbed power equals Re(sigma) E_rms^2 integrated over
    the domain, sigma = n e^2/(m (nu_m + i w)) for a cold collisional plasma
    in a harmonic field; checked with a density too small to perturb E."""
    cfg = W.base_cfg(nx=12, ny=10, r=1, n_lambda=16, steps_per_period=32, p_torr=760.0)
    sim = O.Sim(cfg)
    n_p = 1e8
    sim.coarse.n[...] = n_p
    sim.advance(32)
    P = sim.P
    sigma = n_p * q_e ** 2 / (m_e * complex(P.nu_m, P.omega))
    area = (12 * P.dxc) * (10 * P.dxc)
    expect = sigma.real * (5e6 ** 2 / 2) * area
    assert abs(sim.P_abs / expect - 1) < 1e-10
    assert abs(sim.W_abs - sim.P_abs * P.T) <= 1e-15 * abs(sim.W_abs)


def _incident_rms_closed_form(E0, N, k, x, levels):
    """RMS over the given consecutive E levels of E0 sin(2 pi l / N - k x),
    from the Dirichlet-kernel sum of cos(a + l d):
    sum_l sin^2 = q/2 - (1/2) sin(q d/2)/sin(d/2) cos(a + (l_0 + l_1) d/2)
    with d = 4 pi / N and a = -2 k x."""
    l0, l1 = levels[0], levels[-1]
    q = l1 - l0 + 1
    d = 4.0 * math.pi / N
    a = -2.0 * k * x
    s = 0.5 * q - 0.5 * math.sin(q * d / 2) / math.sin(d / 2) * np.cos(a + (l0 + l1) * d / 2)
    return E0 * np.sqrt(s / q)


def test_erms_output_in_vacuum_is_the_incident_rms():
    """The E_rms output (Sec. II.B, IV) with n = 0: the total field is the
    incident plane wave, so at every period boundary E_rms = E0/sqrt(2) at
    every node of both meshes (P2), also on area the rectangle gains by
    growth (Eq. 5a fill of the coarse value); within a period it is the RMS
    of the incident samples taken since the period began, whose sum has a
    closed form."""
    w = dict(W.small_dmr(), seeds=[(0.0, 0.5, 0.5, 0.1, 0.1)])
    sim = O.sim_from_workload(w)
    P = sim.P
    NT = P.N_T
    E0 = P.E0
    grown = (8, 6, 30, 26)
    sim.replay = [grown, grown]
    for period in range(2):
        for q in range(1, NT + 1):
            sim.coarse_step()
            if q in (1, 5, NT - 1):
                m = sim.coarse.m
                lv = list(range(m - q + 1, m + 1))
                xc = sim.coarse.node_x()
                ref = _incident_rms_closed_form(E0, NT, P.k, xc, lv)[:, None]
                assert np.abs(sim.erms(0) - ref).max() < 1e-12 * E0, (period, q)
                mf = sim.fine.m
                qf = mf % sim.fine.N
                lvf = list(range(mf - qf + 1, mf + 1))
                xf = sim.fine.node_x()
                reff = _incident_rms_closed_form(E0, sim.fine.N, P.k, xf, lvf)[:, None]
                assert np.abs(sim.erms(1) - reff).max() < 1e-12 * E0, (period, q)
        assert sim.rect == grown
        for level in (0, 1):
            e = sim.erms(level)
            assert np.abs(e - E0 / math.sqrt(2)).max() < 1e-12 * E0, (period, level)
