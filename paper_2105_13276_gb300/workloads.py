"""Seeded synthetic workloads shaped like the paper's HPM-breakdown set-ups.

This module only states parameters and draws seeded random numbers.  It holds
none of the method's arithmetic, so both the CUDA library's tests and the CPU
oracle can take their inputs from it.

A workload is a plain dict:
  cfg   : mesh / physics parameters (keys of ``dmr_config``)
  seeds : list of Gaussian seeds, each (n0, x0_frac, y0_frac, sx_lambda, sy_lambda)
          with the centre as a fraction of the domain and widths in wavelengths
  rect  : initial fine rectangle (i0, j0, i1, j1) in coarse node indices, or None
  steps : coarse steps of the run

Set-up of the paper (Sec. II.B, Sec. IV): 110 GHz plane wave incident from the
left, E along y, air at high pressure, Gaussian seed, Mur outer boundary.
"""
from __future__ import annotations

import numpy as np

FREQ = 110e9


def centred_rect(nx, ny, ic, jc, m):
    """m x m coarse cells centred on node (ic, jc), shifted inside the domain."""
    i0 = min(max(ic - m // 2, 0), nx - m)
    j0 = min(max(jc - m // 2, 0), ny - m)
    return (i0, j0, i0 + m, j0 + m)


def base_cfg(**kw):
    cfg = dict(nx=64, ny=64, r=1, n_lambda=32, steps_per_period=64, freq=FREQ,
               E0=5e6, p_torr=700.0, De=None, Da=None, beta_rec=None, Te=None,
               nu_scale=None, nu_a=None, n_th=None, g_th=None, buffer_cells=4,
               growth=True, m_ex=None, m_ey=None, nu_model=None, town_A=None, town_B=None,
               boundary=None, pml_cells=None, coupling=None,
               patch_cap_cells=None, precision=0)
    cfg.update(kw)
    return cfg


def uniform_256(precision=0):
    """Plain uniform mesh: 256x256 cells at lambda/64, Courant 0.5, 700 Torr,
    E0 = 5 MV/m, Gaussian seed 1e15 m^-3 with sigma = lambda/8 at the centre,
    2048 EM steps (16 periods)."""
    cfg = base_cfg(nx=256, ny=256, r=1, n_lambda=64, steps_per_period=128, precision=precision)
    return dict(name="uniform 256x256 lambda/64", cfg=cfg,
                seeds=[(1e15, 0.5, 0.5, 0.125, 0.125)], rect=None, steps=2048)


def dmr_512_r2(precision=1):
    """DMR r=2: coarse 512x512 at lambda/32 (16 x 16 wavelengths), fine patch
    starting at 64x64 fine cells around the seed, fine sub-cycling 2 steps per
    coarse step, 20 ns simulated (2200 periods of 64 coarse steps)."""
    cfg = base_cfg(nx=512, ny=512, r=2, n_lambda=32, steps_per_period=64, precision=precision)
    return dict(name="DMR r=2 coarse 512x512 lambda/32", cfg=cfg,
                seeds=[(1e15, 0.5, 0.5, 0.125, 0.125)],
                rect=centred_rect(512, 512, 256, 256, 32), steps=2200 * 64)


def uniform_fine_equivalent(w):
    """The uniform fine mesh that a DMR workload refines to (r = 1 at r times
    the resolution), for the DMR-versus-uniform comparison."""
    c = dict(w["cfg"])
    r = c["r"]
    c.update(nx=c["nx"] * r, ny=c["ny"] * r, n_lambda=c["n_lambda"] * r,
             steps_per_period=c["steps_per_period"] * r, r=1)
    return dict(name=w["name"] + " (uniform fine equivalent)", cfg=c, seeds=w["seeds"],
                rect=None, steps=w["steps"])


def large_dmr(r=2, precision=1, seed=2105, lo=0.25):
    """Large DMR: coarse 2048x1024 (64 x 32 wavelengths) at lambda/32, eight
    Gaussian seeds with n0 log-uniform in [1e14, 1e16] m^-3, centres uniform in
    [lo, 1 - lo] along each axis (the central half by default), sigma =
    lambda/8.  The rectangle starts at the seeds' bounding box plus 16 coarse
    cells: 15 % of the domain for the central half, 25 % for lo = 0.17."""
    rng = np.random.default_rng(seed)
    n0 = 10.0 ** rng.uniform(14.0, 16.0, size=8)
    xc = rng.uniform(lo, 1.0 - lo, size=8)
    yc = rng.uniform(lo, 1.0 - lo, size=8)
    seeds = [(float(n0[q]), float(xc[q]), float(yc[q]), 0.125, 0.125) for q in range(8)]
    cfg = base_cfg(nx=2048, ny=1024, r=r, n_lambda=32, steps_per_period=64, precision=precision)
    i = [int(round(s[1] * 2048)) for s in seeds]
    j = [int(round(s[2] * 1024)) for s in seeds]
    rect = (max(min(i) - 16, 0), max(min(j) - 16, 0), min(max(i) + 16, 2048), min(max(j) + 16, 1024))
    name = "large DMR coarse 2048x1024 r=%d" % r
    if lo != 0.25:
        name += ", seed centres in [%.2f, %.2f]^2" % (lo, 1.0 - lo)
    return dict(name=name, cfg=cfg, seeds=seeds,
                rect=rect, steps=None)


def batch_runs(count=64, seed=13276):
    """Batched set: coarse sizes uniform in {128,256,512,1024}^2, E0 ~ U[3,8]
    MV/m, p ~ U[100,760] Torr, seed centre ~ U(central half), r = 2, FP32."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice([128, 256, 512, 1024], size=count)
    E0 = rng.uniform(3e6, 8e6, size=count)
    p = rng.uniform(100.0, 760.0, size=count)
    xc = rng.uniform(0.25, 0.75, size=count)
    yc = rng.uniform(0.25, 0.75, size=count)
    runs = []
    for q in range(count):
        nx = int(sizes[q])
        cfg = base_cfg(nx=nx, ny=nx, r=2, n_lambda=32, steps_per_period=64,
                       E0=float(E0[q]), p_torr=float(p[q]), precision=1)
        ic, jc = int(round(xc[q] * nx)), int(round(yc[q] * nx))
        runs.append(dict(name="batch run %d" % q, cfg=cfg,
                         seeds=[(1e15, float(xc[q]), float(yc[q]), 0.125, 0.125)],
                         rect=centred_rect(nx, nx, ic, jc, 32), steps=None))
    return runs


def adjoint_target_map(shape=(65, 65), seed=7):
    """Multiplicative perturbation 1 + 0.05 N(0,1) of the seed map that makes
    the target density of the adjoint workload."""
    rng = np.random.default_rng(seed)
    return 1.0 + 0.05 * rng.standard_normal(shape)


def small_dmr(nx=40, ny=32, r=2, rect=(12, 10, 24, 20), precision=0, **kw):
    """A small DMR case the oracle finishes in seconds: a dense seed near the
    patch so that flags fire and the patch grows within a few periods."""
    cfg = base_cfg(nx=nx, ny=ny, r=r, n_lambda=16, steps_per_period=32, precision=precision,
                   **kw)
    return dict(name="small DMR %dx%d r=%d" % (nx, ny, r), cfg=cfg,
                seeds=[(3e17, 0.45, 0.5, 0.1, 0.1)], rect=rect, steps=None)


def front_1p5(n_lambda, r, growth=1, precision=1):
    """Front-velocity set-up of Sec. IV.B: a 1.5 x 1.5 wavelength domain,
    air at 760 Torr, E0 = 5.5 MV/m at 110 GHz, Gaussian n0 = 1e16 m^-3 at
    (0.85 Lx, 0.5 Ly) (sigma = lambda/8 here; the paper does not give it).
    n_lambda is the coarse resolution, r the refinement factor (1: uniform);
    the initial rectangle is lambda/4 wide around the seed."""
    nx = int(round(1.5 * n_lambda))
    cfg = base_cfg(nx=nx, ny=nx, r=r, n_lambda=n_lambda, steps_per_period=2 * n_lambda, E0=5.5e6,
                   p_torr=760.0, growth=growth, precision=precision)
    m = max(2, n_lambda // 4)
    rect = centred_rect(nx, nx, int(0.85 * nx), nx // 2, m) if r > 1 else None
    return dict(name="front 1.5 lambda, lambda/%d, r=%d" % (n_lambda, r), cfg=cfg,
                seeds=[(1e16, 0.85, 0.5, 0.125, 0.125)], rect=rect, steps=None)


def random_fields(shape, seed, scale=1.0):
    """Seeded standard-normal field values (for invariants and parity of the
    EM update with arbitrary states)."""
    return scale * np.random.default_rng(seed).standard_normal(shape)
