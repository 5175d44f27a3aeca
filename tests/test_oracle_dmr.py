"""Pins of the oracle's coarse/fine machinery (Sec. III.C-III.D): the patch
covering the whole domain equals the uniform fine mesh, Eq. 5a/5b reproduce
linear data, composite totals integrate constants exactly, flags and growth
match brute force, and a naive per-element implementation agrees."""
import math

import numpy as np
import pytest

from oracle import dmr_oracle as O
from paper_2105_13276_gb300 import workloads as W
from tests.naive_dmr import Naive


def _seeded(w, **kw):
    return O.sim_from_workload(w, **kw)


def test_p6_full_patch_equals_uniform_fine_bitwise():
    """P6: with the rectangle covering the whole domain, every fine side is on
    the domain edge, so the fine mesh is a uniform fine run: bit-identical."""
    w = W.small_dmr(nx=12, ny=10, r=2, rect=(0, 0, 12, 10))
    dmr = _seeded(w)
    uni = _seeded(W.uniform_fine_equivalent(w))
    steps = 3 * w["cfg"]["steps_per_period"]
    dmr.advance(steps)
    uni.advance(2 * steps)          # the uniform fine mesh steps at dt/r
    f, u = dmr.fine, uni.coarse
    for name in ("Ex", "Ey", "Hz", "vx", "vy", "n"):
        assert np.array_equal(getattr(f, name), getattr(u, name)), name
    assert dmr.N_e == uni.N_e
    assert dmr.P_abs == uni.P_abs
    assert np.any(f.n != 0) and np.any(f.Ex != 0)


def test_p9_interpolation_reproduces_linear_data():
    """P9: Eq. 5b (linear along the line, linear blend in time) and Eq. 5a
    (bilinear) are exact for data linear in space and time."""
    line_old = 3.0 + 0.5 * np.arange(20)
    line_new = -1.0 + 0.25 * np.arange(20)
    pos = np.linspace(0.0, 19.0, 77)
    for frac in (0.0, 0.25, 0.5, 1.0):
        got = O.linear_cfb(line_old, line_new, frac, pos)
        want = (1 - frac) * (3.0 + 0.5 * pos) + frac * (-1.0 + 0.25 * pos)
        assert np.allclose(got, want, rtol=0, atol=1e-12)
    i = np.arange(15)[:, None]
    j = np.arange(11)[None, :]
    F = 2.0 + 0.3 * i - 0.7 * j + 0.0 * i * j
    px = np.linspace(0, 14, 29)
    py = np.linspace(0, 10, 31)
    got = O.bilinear(F, px, py)
    want = 2.0 + 0.3 * px[:, None] - 0.7 * py[None, :]
    assert np.allclose(got, want, rtol=0, atol=1e-12)
    # a bilinear (not only linear) function is reproduced as well
    G = i * j * 1.0
    assert np.allclose(O.bilinear(G, px, py), px[:, None] * py[None, :], atol=1e-12)


def test_p9_expansion_fill_is_exact_for_linear_coarse_fields():
    """Eq. 5a fill of newly refined area: coarse fields linear in space give
    fine values equal to the same linear function at the fine positions."""
    w = W.small_dmr(nx=20, ny=16, r=2, rect=(6, 5, 10, 9))
    sim = _seeded(w)
    c = sim.coarse
    for name, ox, oy in (("Ex", 0.5, 0.0), ("Ey", 0.0, 0.5), ("Hz", 0.5, 0.5), ("n", 0.0, 0.0)):
        a = getattr(c, name)
        ii = np.arange(a.shape[0])[:, None] + ox
        jj = np.arange(a.shape[1])[None, :] + oy
        a[...] = 1.0 + 2.0 * ii + 3.0 * jj
    sim._expand((3, 2, 14, 12))
    f = sim.fine
    for name, ox, oy in (("Ex", 0.5, 0.0), ("Ey", 0.0, 0.5), ("Hz", 0.5, 0.5)):
        a = getattr(f, name)
        x = 3 + (np.arange(a.shape[0])[:, None] + ox) / 2
        y = 2 + (np.arange(a.shape[1])[None, :] + oy) / 2
        want = 1.0 + 2.0 * x + 3.0 * y
        # the old rectangle's part holds the copied old fine data (zeros here)
        oi, oj = 2 * (6 - 3), 2 * (5 - 2)
        outside = np.ones(a.shape, bool)
        if name == "Ex":
            outside[oi:oi + 8, oj:oj + 9] = False
        elif name == "Ey":
            outside[oi:oi + 9, oj:oj + 8] = False
        else:
            outside[oi:oi + 8, oj:oj + 8] = False
        assert np.allclose(a[outside], want[outside], atol=1e-9)


def test_composite_total_integrates_constant_exactly():
    """The FP64 electron total uses composite trapezoid weights (coarse
    outside the rectangle, fine inside): a constant density integrates to
    n Lx Ly exactly, whatever the rectangle."""
    for r, rect in ((1, None), (2, (3, 2, 9, 7)), (2, (0, 0, 5, 10)), (3, (0, 4, 12, 10))):
        cfg = W.base_cfg(nx=12, ny=10, r=r, n_lambda=16, steps_per_period=32)
        sim = O.Sim(cfg, rect=rect)
        wc, wf = sim._weights()
        P = sim.P
        tot = P.dxc ** 2 * wc.sum()
        if wf is not None:
            tot += (P.dxc / r) ** 2 * wf.sum()
        assert abs(tot - 12 * 10 * P.dxc ** 2) < 1e-12 * tot
        assert np.all(wc >= 0)


def _brute_flags(n, n_th, g_th, dx):
    nx1, ny1 = n.shape
    out = np.zeros(n.shape, bool)
    for i in range(nx1):
        for j in range(ny1):
            f = n[i, j] > n_th
            if 0 < i < nx1 - 1 and 0 < j < ny1 - 1:
                g = math.hypot((n[i + 1, j] - n[i - 1, j]) / (2 * dx), (n[i, j + 1] - n[i, j - 1]) / (2 * dx))
                f = f or g > g_th
            out[i, j] = f
    return out


def test_flags_match_brute_force():
    rng = np.random.default_rng(5)
    dx = 1e-4
    for trial in range(5):
        n = 10.0 ** rng.uniform(12, 18, size=(17, 13))
        got = O.flag_mask(n, 1.5e17, 2e20, dx)
        assert np.array_equal(got, _brute_flags(n, 1.5e17, 2e20, dx))
        got32 = O.flag_mask(n, 1.5e17, 2e20, dx, dtype=np.float32)
        # FP32 decision may differ only on near-ties
        assert (got32 != got).sum() <= 2


def test_growth_policy():
    assert O.grow_rect((5, 5, 9, 9), None, 4, 20, 20) == (5, 5, 9, 9)
    assert O.grow_rect((5, 5, 9, 9), (6, 6, 7, 7), 4, 20, 20) == (2, 2, 11, 11)
    assert O.grow_rect((5, 5, 9, 9), (0, 1, 19, 7), 4, 20, 20) == (0, 0, 20, 11)
    assert O.mask_bbox(np.zeros((4, 4), bool)) is None
    m = np.zeros((6, 5), bool)
    m[1, 3] = m[4, 2] = True
    assert O.mask_bbox(m) == (1, 2, 4, 3)


def test_threshold_line_policy():
    """Sec. III.D threshold lines: a side is hit when n > n_th at a coarse
    node on it (corners included); hit sides jump out by m_ex (x) or m_ey
    (y), clipped to the domain."""
    n = np.zeros((21, 21))
    rect = (5, 6, 12, 14)
    assert O.line_hits(n, rect, 1.0) == (False, False, False, False)
    n[12, 9] = 2.0                                   # on the right side
    assert O.line_hits(n, rect, 1.0) == (False, False, True, False)
    n[12, 9] = 1.0                                   # equal: not a hit (strict)
    assert O.line_hits(n, rect, 1.0) == (False, False, False, False)
    n[5, 14] = 3.0                                   # top-left corner: two sides
    assert O.line_hits(n, rect, 1.0) == (True, False, False, True)
    n[8, 10] = 9.0                                   # interior nodes do not count
    n[13, 10] = 9.0                                  # nor nodes outside
    assert O.line_hits(n, rect, 1.0) == (True, False, False, True)
    assert O.grow_lines(rect, (True, False, False, True), 8, 4, 20, 20) == (0, 6, 12, 18)
    assert O.grow_lines(rect, (False, True, True, False), 8, 4, 20, 20) == (5, 2, 20, 14)
    assert O.grow_lines(rect, (True, True, True, True), 3, 2, 20, 20) == (2, 4, 15, 16)
    assert O.grow_lines(rect, (False,) * 4, 8, 4, 20, 20) == rect


@pytest.mark.parametrize("rect,growth,coupling", [((3, 3, 7, 6), 1, 0), ((0, 2, 5, 8), 1, 0),
                                                  ((4, 0, 10, 8), 1, 0), ((4, 3, 6, 5), 2, 0),
                                                  ((5, 3, 8, 5), 2, 0), ((3, 3, 7, 6), 1, 1)])
def test_p11_naive_per_element_implementation_agrees(rect, growth, coupling):
    """P11: a 10x8 coarse r=2 DMR run, a dense seed so that flags fire and the
    rectangle grows, against an independent per-element implementation (also
    with the density-only transfer back, coupling = 1)."""
    cfg = W.base_cfg(nx=10, ny=8, r=2, n_lambda=8, steps_per_period=16, E0=6e6, p_torr=300.0,
                     n_th=1e16, buffer_cells=1, growth=growth, coupling=coupling)
    sim = O.Sim(cfg, rect=rect)
    nv = Naive(cfg, rect)
    P = sim.P
    seed = (2e16, 5.2 * P.dxc, 4.1 * P.dxc, 1.3 * P.dxc, 1.1 * P.dxc)
    sim.seed_gaussian(*seed)
    nv.seed(*seed)
    for step in range(3 * 16):
        sim.coarse_step()
        nv.coarse_step()
        assert sim.rect == nv.rect
        for level in (0, 1):
            a = sim.coarse if level == 0 else sim.fine
            b = nv.c if level == 0 else nv.fm
            for name in ("Ex", "Ey", "Hz", "vx", "vy", "n", "S2"):
                x = getattr(a, name)
                y = np.array(getattr(b, name))
                scale = max(np.abs(y).max(), 1e-300)
                assert np.abs(x - y).max() <= 1e-12 * scale, (step, level, name)
    assert sim.log == nv.log
    assert sim.log[-1] != tuple(rect), "the rectangle should have grown"


def test_replay_reproduces_log():
    """Replaying the recorded rectangle log gives the same run."""
    w = W.small_dmr()
    a = _seeded(w)
    a.advance(4 * 32)
    b = _seeded(w)
    b.replay = list(a.log)
    b.advance(4 * 32)
    assert b.log == a.log
    assert np.array_equal(a.fine.n, b.fine.n)
    assert a.log[-1] != tuple(w["rect"])


def test_capacity_error():
    w = W.small_dmr()
    cfg = dict(w["cfg"])
    cfg["patch_cap_cells"] = 4 * 12 * 10
    sim = O.Sim(cfg, rect=w["rect"])
    with pytest.raises(O.CapacityError):
        sim._expand((0, 0, 40, 32))


def test_p12_oracle_complex_step_matches_central_differences():
    """P12 reference: the oracle runs on complex128, so a complex step gives
    dL/dE0 exact to rounding; it must agree with central differences (h = 1e-6
    relative) to the FD truncation error, with the schedule replayed."""
    w = W.small_dmr()
    base = O.sim_from_workload(w)
    seed = base.fine.n.copy()
    steps = 2 * w["cfg"]["steps_per_period"]

    def run(E0, log=None, dtype=np.float64):
        sim = O.Sim(dict(w["cfg"], E0=E0), rect=w["rect"], dtype=dtype)
        sim.seed_map(seed.astype(dtype), 0, 0)
        if log is not None:
            sim.replay = list(log)
        sim.advance(steps)
        return sim

    ref = run(5e6)
    target = 0.9 * ref.coarse.n
    L = lambda s: np.sum((s.coarse.n - target) ** 2)
    h = 5e6 * 1e-20
    cs = L(run(complex(5e6, h), ref.log, np.complex128)).imag / h
    hf = 5e6 * 1e-6
    fd = (L(run(5e6 + hf, ref.log)) - L(run(5e6 - hf, ref.log))) / (2 * hf)
    assert abs(cs / fd - 1) < 1e-8
    assert abs(L(run(complex(5e6, h), ref.log, np.complex128)).real / L(ref) - 1) < 1e-14
