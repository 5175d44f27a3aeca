"""Pins of the oracle's coarse-fine coupling readings (Sec. III.C: the coarse
mesh hands E, H, v and n to the fine boundaries, and the fine mesh's updated
quantities go back to the coarse mesh).

coupling = 0 (the default reading) sends the fine E means back every coarse
step and the fine density every period; coupling = 1 sends the density only.
Two properties fix the difference without retyping either step:
- with coupling = 1 nothing of the fine fields reaches the coarse mesh before
  the first density transfer, so the coarse mesh steps exactly as a run
  without a rectangle;
- the vacuum coupled step (no plasma, no incident wave) is linear; its matrix
  is block-triangular for coupling = 1 (coarse -> fine only), so its spectral
  radius is that of the two uncoupled meshes, 1, while the two-way loop of
  coupling = 0 has a growing mode."""
import numpy as np
import pytest

from oracle import dmr_oracle as O
from paper_2105_13276_gb300 import workloads as W

FIELDS = ("Ex", "Ey", "Hz", "vx", "vy")


def _pair(coupling):
    w = W.small_dmr(nx=40, ny=32, r=2, rect=(12, 10, 24, 20), precision=0, coupling=coupling)
    dmr = O.sim_from_workload(w)
    coarse_only = O.sim_from_workload(dict(w, rect=None, cfg=dict(w["cfg"], r=1)))
    return w, dmr, coarse_only


def test_one_way_coarse_mesh_steps_as_without_a_rectangle():
    w, dmr, alone = _pair(1)
    steps = w["cfg"]["steps_per_period"]   # the first density transfer ends the period
    dmr.advance(steps)
    alone.advance(steps)
    for name in FIELDS:
        a, b = getattr(dmr.coarse, name), getattr(alone.coarse, name)
        assert np.abs(b).max() > 0, name
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-13 * np.abs(b).max(), err_msg=name)


def test_two_way_coarse_mesh_takes_the_fine_means():
    """The same comparison with coupling = 0 fails by far more than rounding:
    the coarse E under the rectangle is the fine mean."""
    w, dmr, alone = _pair(0)
    steps = w["cfg"]["steps_per_period"]
    dmr.advance(steps)
    alone.advance(steps)
    a, b = dmr.coarse.Ey, alone.coarse.Ey
    assert np.abs(a - b).max() > 1e-6 * np.abs(b).max()


def _vacuum_radius(coupling, nx=12, ny=12, rect=(4, 4, 8, 8), r=2):
    w = W.small_dmr(nx=nx, ny=ny, r=r, rect=rect, precision=0)
    sim = O.Sim(dict(w["cfg"], E0=0.0, growth=0, coupling=coupling), rect=rect)
    c, f = sim.coarse, sim.fine
    state = [c.Ex, c.Ey, c.Hz, f.Ex, f.Ey, f.Hz]
    sizes = [a.size for a in state]
    M = np.zeros((sum(sizes), sum(sizes)))
    for col in range(M.shape[1]):
        for mesh in (c, f):
            for a in (mesh.Ex, mesh.Ey, mesh.Hz, mesh.vx, mesh.vy, mesh.n):
                a[...] = 0.0
        q = col
        for a, s in zip(state, sizes):
            if q < s:
                a.flat[q] = 1.0
                break
            q -= s
        c.m, f.m = 1, r                      # mid-period: no period end in the step
        sim.coarse_step()
        M[:, col] = np.concatenate([a.ravel() for a in state])
    return float(np.abs(np.linalg.eigvals(M)).max())


@pytest.mark.parametrize("coupling", [0, 1])
def test_vacuum_coupled_step_spectral_radius(coupling):
    """12^2 coarse cells, a 4^2 rectangle at r = 2, Mur outside: one coarse
    step as a matrix over the E and H of both meshes (with no plasma the
    velocities do not act on E).  One-way: radius 1 (eigenvalue error of a
    non-normal matrix ~1e-9); two-way: 1.00019."""
    rho = _vacuum_radius(coupling)
    if coupling == 1:
        assert rho <= 1.0 + 1e-8, rho
    else:
        assert rho >= 1.0 + 5e-5, rho
