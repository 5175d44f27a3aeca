"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Tolerances (the run's precision decides):
  FP64 path : relative L2 <= 1e-12 per field, FP64 totals <= 1e-12, masks and
              rectangle logs bit-exact;
  FP32 path : relative L2 <= 1e-4 per field against the FP64 oracle on a
              bounded horizon with the oracle's rectangle log replayed; the
              FP32 mask equals the oracle's flag rule applied to the GPU's own
              density in FP32 (same precision decides the integer).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import dmr_oracle as O  # noqa: E402
from paper_2105_13276_gb300 import dmr as D  # noqa: E402
from paper_2105_13276_gb300 import workloads as W  # noqa: E402

FIELDS = ("Ex", "Ey", "Hz", "vx", "vy", "n")
TOL64 = 1e-12
TOL32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2105_13276_gb300 import build as B
    B.build()
    D.load()


def rel_l2(g, o):
    no = np.linalg.norm(o)
    if no == 0:
        return float(np.linalg.norm(g))
    return float(np.linalg.norm(g.astype(np.float64) - o) / no)


def ring_mask(shape, level, rect):
    """Elements within one cell of the coarse-fine interface: the outermost
    row and column of every fine array, and on the coarse mesh a band of
    width one around the rectangle's sides (index space of the array, which
    covers every stagger).  A wrong interface value is a thin error that a
    relative L2 over the whole mesh can hide."""
    ii, jj = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
    if level == 1:
        return (ii == 0) | (jj == 0) | (ii == shape[0] - 1) | (jj == shape[1] - 1)
    i0, j0, i1, j1 = rect
    near_x = ((abs(ii - i0) <= 1) | (abs(ii - i1) <= 1)) & (jj >= j0 - 1) & (jj <= j1 + 1)
    near_y = ((abs(jj - j0) <= 1) | (abs(jj - j1) <= 1)) & (ii >= i0 - 1) & (ii <= i1 + 1)
    return near_x | near_y


def compare(run, sim, tol, fields=FIELDS, levels=(0, 1), s2=True, verbose=False):
    """Per-field relative L2 (the parity metric) and, where a fine rectangle
    exists, the element-wise max-abs error on the interface ring relative to
    the field's largest magnitude, both within tol."""
    worst = {}
    for level in levels:
        mesh = sim.coarse if level == 0 else sim.fine
        if mesh is None:
            continue
        for name in fields + (("S2",) if s2 else ()):
            g = run.read(name, level).T
            o = getattr(mesh, name)
            assert g.shape == o.shape, (name, level, g.shape, o.shape)
            e = rel_l2(g, o)
            worst[(level, name)] = e
            assert e <= tol, (level, name, e)
            if sim.fine is not None and np.abs(o).max() > 0:
                ring = ring_mask(o.shape, level, sim.rect)
                er = float(np.abs(g.astype(np.float64) - o)[ring].max() / np.abs(o).max())
                worst[(level, name, "ring")] = er
                assert er <= tol, (level, name, "ring", er)
    if verbose:
        print({"%s" % (k,): "%.2e" % v for k, v in worst.items()})
    return worst


def test_uniform_fp64_matches_oracle():
    w = W.small_dmr(nx=70, ny=50, r=1, rect=None)
    sim = O.sim_from_workload(w)
    run = D.run_from_workload(w)
    steps = 2 * 32 + 7
    sim.advance(steps)
    run.advance(steps)
    compare(run, sim, TOL64)
    st = run.stats()
    assert abs(st["N_e"] / sim.N_e - 1) < TOL64
    assert abs(st["P_abs"] / sim.P_abs - 1) < TOL64
    assert abs(st["W_abs"] / sim.W_abs - 1) < TOL64
    assert st["periods"] == 2 and st["coarse_steps"] == steps


def test_uniform_fp64_several_tiles_ragged():
    """150 x 90 cells: 5 x 12 thread blocks with ragged last tiles."""
    w = W.small_dmr(nx=150, ny=90, r=1, rect=None)
    sim = O.sim_from_workload(w)
    run = D.run_from_workload(w)
    sim.advance(40)
    run.advance(40)
    compare(run, sim, TOL64)


@pytest.mark.parametrize("rect", [(12, 10, 24, 20), (0, 0, 10, 9), (28, 20, 40, 32), (3, 0, 30, 6)])
def test_dmr_fp64_growth_matches_oracle(rect):
    """Free-running growth policy on both sides: identical rectangle after
    every period, bit-exact masks, fields within 1e-12."""
    w = W.small_dmr(rect=rect)
    sim = O.sim_from_workload(w)
    run = D.run_from_workload(w)
    NT = w["cfg"]["steps_per_period"]
    for p in range(4):
        sim.advance(NT)
        run.advance(NT)
        assert run.get_patch() == tuple(sim.rect), (p, run.get_patch(), sim.rect)
        mask = run.read("mask").T.astype(bool)
        assert np.array_equal(mask, sim.masks[-1]), p
    sim.advance(5)
    run.advance(5)
    compare(run, sim, TOL64)
    st = run.stats()
    assert abs(st["N_e"] / sim.N_e - 1) < TOL64
    assert abs(st["P_abs"] / sim.P_abs - 1) < TOL64
    assert sim.log[-1] != tuple(rect) or rect == (0, 0, 10, 9)


@pytest.mark.parametrize("rect,nth,mex,mey", [((16, 14, 21, 18), 3e16, None, None),
                                               ((17, 15, 20, 17), 5e16, 30, 3)])
def test_dmr_fp64_threshold_lines_match_oracle(rect, nth, mex, mey):
    """Growth by threshold lines (Sec. III.D), free-running on both sides:
    identical rectangles after every period (the second case clips at both
    x edges of the domain), bit-exact masks, fields within 1e-12."""
    w = W.small_dmr(rect=rect, growth=2, n_th=nth, m_ex=mex, m_ey=mey)
    sim = O.sim_from_workload(w)
    run = D.run_from_workload(w)
    NT = w["cfg"]["steps_per_period"]
    for p in range(3):
        sim.advance(NT)
        run.advance(NT)
        assert run.get_patch() == tuple(sim.rect), (p, run.get_patch(), sim.rect)
        assert np.array_equal(run.read("mask").T.astype(bool), sim.masks[-1]), p
    sim.advance(5)
    run.advance(5)
    compare(run, sim, TOL64)
    assert sim.log[0] != tuple(rect)
    if mex == 30:
        assert sim.log[0][0] == 0 and sim.log[0][2] == w["cfg"]["nx"]


@pytest.mark.parametrize("r,precision", [(2, 0), (4, 0), (2, 1)])
def test_one_way_coupling_matches_oracle(r, precision):
    """coupling = 1 (the density alone goes back to the coarse mesh):
    free-running growth in FP64 (rectangles and masks exact, fields 1e-12),
    FP32 with the oracle's rectangle log replayed (1e-4)."""
    w = W.small_dmr(r=r, precision=precision, coupling=1)
    sim = O.sim_from_workload(w)
    NT = w["cfg"]["steps_per_period"]
    steps = 3 * NT + 5
    sim.advance(steps)
    run = D.run_from_workload(w)
    if precision == 1:
        run.replay_log(sim.log)
    run.advance(steps)
    assert run.get_patch() == tuple(sim.rect)
    assert sim.log[-1] != tuple(w["rect"]), "the rectangle should grow"
    compare(run, sim, TOL64 if precision == 0 else TOL32)
    st = run.stats()
    assert abs(st["N_e"] / sim.N_e - 1) < (TOL64 if precision == 0 else TOL32)


def test_one_way_coupling_launch_forms_identical():
    """coupling = 1 in every launch form: direct launches, CUDA graphs, the
    persistent period and a batch give the same bits (FP32, growth)."""
    w = W.small_dmr(precision=1, coupling=1)
    steps = 3 * w["cfg"]["steps_per_period"] + 7
    runs = []
    for form in ("direct", "graphs", "persistent"):
        run = D.run_from_workload(w)
        if form == "graphs":
            run.set_graphs(True)
        if form == "persistent":
            run.set_persistent(True)
        run.advance(steps)
        runs.append(run)
    b = D.batch_from_workloads([w, W.small_dmr(precision=1)])
    b.advance(steps)
    for other in runs[1:] + [b.runs[0]]:
        assert other.get_patch() == runs[0].get_patch()
        for level in (0, 1):
            for name in FIELDS + ("S2",):
                assert np.array_equal(other.read(name, level), runs[0].read(name, level)), (level, name)


@pytest.mark.parametrize("precision", [0, 1])
def test_townsend_ionization_matches_oracle(precision):
    """The Townsend coefficient set (nu_model = 1, Sec. II.A) on the GPU
    against the oracle: free-running growth in FP64 (rectangles and masks
    bit-exact, fields within 1e-12); FP32 with the oracle's log replayed."""
    w = W.small_dmr(nu_model=1, town_A=2000.0, town_B=30000.0, precision=precision)
    sim = O.sim_from_workload(w)
    NT = w["cfg"]["steps_per_period"]
    run = D.run_from_workload(w)
    if precision:
        ref = O.sim_from_workload(w)
        ref.advance(3 * NT + 5)
        run.replay_log(ref.log)
    for p in range(3):
        sim.advance(NT)
        run.advance(NT)
        assert run.get_patch() == tuple(sim.rect), p
        if precision == 0:
            assert np.array_equal(run.read("mask").T.astype(bool), sim.masks[-1]), p
    sim.advance(5)
    run.advance(5)
    compare(run, sim, TOL64 if precision == 0 else TOL32)
    st = run.stats()
    assert abs(st["N_e"] / sim.N_e - 1) < (TOL64 if precision == 0 else TOL32)
    # the coefficient set matters: the fit gives another density
    sim_fit = O.sim_from_workload(W.small_dmr(precision=precision))
    sim_fit.advance(3 * NT + 5)
    assert abs(sim_fit.N_e / sim.N_e - 1) > 1e-6


@pytest.mark.parametrize("r,precision", [(1, 0), (2, 0), (2, 1)])
def test_cpml_boundary_matches_oracle(r, precision):
    """CPML outer boundary (boundary = 1): uniform and DMR runs against the
    oracle.  FP64 free-running (rectangle logs equal, growth held pml_cells
    + 2 cells inside), FP32 with the oracle's log replayed."""
    if r == 1:
        w = W.small_dmr(nx=70, ny=50, r=1, rect=None, boundary=1, pml_cells=6, precision=precision)
    else:
        w = W.small_dmr(boundary=1, pml_cells=4, precision=precision)
    sim = O.sim_from_workload(w)
    NT = w["cfg"]["steps_per_period"]
    run = D.run_from_workload(w)
    steps = 4 * NT + 7
    if precision:
        ref = O.sim_from_workload(w)
        ref.advance(steps)
        run.replay_log(ref.log)
    sim.advance(steps)
    run.advance(steps)
    if r > 1:
        assert run.get_patch() == tuple(sim.rect)
        k = 4 + 2
        i0, j0, i1, j1 = sim.rect
        assert k <= i0 and k <= j0 and i1 <= 40 - k and j1 <= 32 - k
    compare(run, sim, TOL64 if precision == 0 else TOL32)
    # the layer is active: the scattered field differs from a Mur run's
    mur = O.sim_from_workload(dict(w, cfg=dict(w["cfg"], boundary=0)))
    mur.advance(steps)
    assert np.abs(mur.coarse.Ey - sim.coarse.Ey).max() > 1e-6 * np.abs(sim.coarse.Ey).max()


def test_cpml_rejections():
    w = W.small_dmr(boundary=1, pml_cells=4)
    run = D.Run(w["cfg"])
    with pytest.raises(D.DMRError) as e:
        run.set_patch((3, 10, 24, 20))          # inside the layer's margin
    assert e.value.code == D.EINVAL
    run.set_patch(w["rect"])
    NT = w["cfg"]["steps_per_period"]
    with pytest.raises(D.DMRError) as e:
        run.adjoint_record(2 * NT, NT)
    assert e.value.code == D.EINVAL
    with pytest.raises(D.DMRError):
        D.batch_from_workloads([w, W.small_dmr()])


@pytest.mark.parametrize("precision", [0, 1])
def test_dmr_many_strips_match_oracle(precision):
    """Meshes several warp strips wide on both levels, with strips inside
    the mesh, at its edges and over the restricted region; growth
    free-running in FP64, the oracle's log replayed in FP32."""
    w = W.small_dmr(nx=128, ny=96, rect=(40, 30, 80, 62), precision=precision)
    sim = O.sim_from_workload(w)
    NT = w["cfg"]["steps_per_period"]
    run = D.run_from_workload(w)
    if precision:
        ref = O.sim_from_workload(w)
        ref.advance(2 * NT + 7)
        run.replay_log(ref.log)
    for _ in range(2):
        sim.advance(NT)
        run.advance(NT)
        assert run.get_patch() == tuple(sim.rect)
    sim.advance(7)
    run.advance(7)
    compare(run, sim, TOL64 if precision == 0 else TOL32)


def test_fp32_against_fp64_oracle_with_replay():
    w = W.small_dmr(precision=1)
    sim = O.sim_from_workload(w)
    NT = w["cfg"]["steps_per_period"]
    sim.advance(3 * NT + 9)
    run = D.run_from_workload(w)
    run.replay_log(sim.log)
    run.advance(3 * NT + 9)
    assert run.get_patch() == tuple(sim.rect)
    worst = compare(run, sim, TOL32)
    assert max(worst.values()) > 1e-9  # it really is FP32
    # FP32 flags: the oracle's rule applied to the GPU's density in FP32
    n32 = run.read("n").T
    ref = O.flag_mask(n32, sim.P.n_th, sim.P.g_th, sim.P.dxc, dtype=np.float32)
    run2 = D.run_from_workload(w)
    run2.replay_log(sim.log)
    run2.advance(3 * NT)
    n32 = run2.read("n").T
    ref = O.flag_mask(n32, sim.P.n_th, sim.P.g_th, sim.P.dxc, dtype=np.float32)
    assert np.array_equal(run2.read("mask").T.astype(bool), ref)


def test_full_patch_equals_uniform_fine_on_gpu():
    """A rectangle covering the whole domain makes the fine mesh a uniform
    fine run: bit-identical on the GPU too."""
    w = W.small_dmr(nx=24, ny=20, r=2, rect=(0, 0, 24, 20))
    dmr = D.run_from_workload(w)
    uni = D.run_from_workload(W.uniform_fine_equivalent(w))
    dmr.advance(2 * 32 + 3)
    uni.advance(2 * (2 * 32 + 3))
    for name in FIELDS:
        assert np.array_equal(dmr.read(name, 1), uni.read(name, 0)), name
    assert dmr.stats()["N_e"] == uni.stats()["N_e"]


@pytest.mark.parametrize("precision", [0, 1])
def test_graphs_equal_direct_launches(precision):
    w = W.small_dmr(precision=precision)
    a = D.run_from_workload(w)
    b = D.run_from_workload(w)
    b.set_graphs(True)
    a.advance(5 * 32 + 4)
    b.advance(5 * 32 + 4)
    assert a.get_patch() == b.get_patch()
    for level in (0, 1):
        for name in FIELDS:
            assert np.array_equal(a.read(name, level), b.read(name, level)), (level, name)
    assert b.launch_count() > 0


@pytest.mark.parametrize("precision", [0, 1])
def test_launch_shapes_give_identical_results(precision):
    """Every strip height the autotuner may pick (and one row per warp) gives
    the same bits, graphs on, through growth."""
    w = W.small_dmr(precision=precision)
    ref = D.run_from_workload(w)
    ref.set_graphs(True)
    ref.advance(3 * 32 + 5)
    for wps in (1, 8, 16, 96, 1024):
        run = D.run_from_workload(w)
        run.set_graphs(True)
        run.set_launch_shape(wps)
        run.advance(3 * 32 + 5)
        assert run.get_patch() == ref.get_patch()
        for level in (0, 1):
            for name in FIELDS + ("S2",):
                assert np.array_equal(run.read(name, level), ref.read(name, level)), (wps, level, name)
    with pytest.raises(D.DMRError) as e:
        ref.set_launch_shape(0)
    assert e.value.code == D.EINVAL


@pytest.mark.parametrize("precision", [0, 1])
def test_launch_shapes_identical_with_interior_blocks(precision):
    """Meshes several strips wide and tall: blocks away from every side take
    the strip path without edge tests, the others the full one, and which
    blocks do depends on the strip height.  Every height gives the same bits,
    so the two paths agree node for node."""
    w = W.small_dmr(nx=130, ny=100, rect=(40, 30, 90, 70), precision=precision)
    NT = w["cfg"]["steps_per_period"]
    ref = D.run_from_workload(w)
    ref.set_graphs(True)
    ref.set_launch_shape(1)
    ref.advance(2 * NT + 5)
    for wps in (16, 96, 1024):
        run = D.run_from_workload(w)
        run.set_graphs(True)
        run.set_launch_shape(wps)
        run.advance(2 * NT + 5)
        assert run.get_patch() == ref.get_patch()
        for level in (0, 1):
            for name in FIELDS + ("S2",):
                assert np.array_equal(run.read(name, level), ref.read(name, level)), (wps, level, name)


def test_vacuum_stays_exactly_zero():
    w = W.small_dmr()
    w = dict(w, seeds=[(0.0, 0.5, 0.5, 0.1, 0.1)])
    run = D.run_from_workload(w)
    run.advance(70)
    for level in (0, 1):
        for name in ("Ex", "Ey", "Hz", "vx", "n"):
            assert not np.any(run.read(name, level)), (level, name)


def test_full_size_uniform_256_fp64_in_the_bench_launch_shape():
    """The uniform workload (256^2 at lambda/64, FP64) in the launch shape the
    benchmark times (autotuned strip height, CUDA graphs) against the FP64
    oracle over two periods and seven steps, with the period totals."""
    w = W.uniform_256(precision=0)
    NT = w["cfg"]["steps_per_period"]
    steps = 2 * NT + 7
    sim = O.sim_from_workload(w)
    sim.advance(steps)
    run = D.run_from_workload(w)
    run.autotune()
    run.set_graphs(True)
    run.advance(steps)
    compare(run, sim, TOL64, levels=(0,), verbose=True)
    st = run.stats()
    for key, ref in (("N_e", sim.N_e), ("P_abs", sim.P_abs), ("W_abs", sim.W_abs)):
        assert abs(st[key] / ref - 1) < TOL64, key


def test_full_size_dmr_512_fp64_in_the_bench_launch_shape():
    """The DMR benchmark geometry (coarse 512^2 at lambda/32, r = 2) in FP64,
    autotuned and in CUDA graphs, free-running (its own period-end decisions)
    against the FP64 oracle over two periods and seven steps."""
    w = W.dmr_512_r2(precision=0)
    NT = w["cfg"]["steps_per_period"]
    steps = 2 * NT + 7
    sim = O.sim_from_workload(w)
    sim.advance(steps)
    run = D.run_from_workload(w)
    run.autotune()
    run.set_graphs(True)
    run.advance(steps)
    assert run.get_patch() == tuple(sim.rect)
    compare(run, sim, TOL64, verbose=True)
    st = run.stats()
    for key, ref in (("N_e", sim.N_e), ("P_abs", sim.P_abs), ("W_abs", sim.W_abs)):
        assert abs(st[key] / ref - 1) < TOL64, key


@pytest.mark.parametrize("periods", [10, 100])
def test_full_size_dmr_512_fp32_graphs(periods):
    """The benchmark workload (coarse 512^2 at lambda/32, r = 2, FP32, CUDA
    graphs and the tuned strip height as timed) against the FP64 oracle over
    10 and 100 periods, read mid-period (S2 holds a partial sum).  The FP32
    relative L2 error of every field is printed: the statement of the FP32
    path's error at a stated horizon."""
    w = W.dmr_512_r2(precision=1)
    sim = O.sim_from_workload(w)
    NT = w["cfg"]["steps_per_period"]
    steps = periods * NT + 17
    sim.advance(steps)
    run = D.run_from_workload(w)
    run.autotune()
    run.set_graphs(True)
    run.replay_log(sim.log)
    run.advance(steps)
    print("\nFP32 vs FP64 oracle, 512^2 r=2, %d periods + 17 steps (level, field): relative L2"
          % periods)
    worst = compare(run, sim, TOL32, verbose=True)
    for level in (0, 1):
        e = rel_l2(run.read("erms", level).T, sim.erms(level))
        worst[(level, "erms")] = e
        assert e <= TOL32, (level, "erms", e)
    print("E_rms:", worst[(0, "erms")], worst[(1, "erms")])
    st = run.stats()
    assert abs(st["N_e"] / sim.N_e - 1) < TOL32
    assert abs(st["P_abs"] / sim.P_abs - 1) < TOL32


def test_full_size_dmr_512_fp32_with_growth():
    """The benchmark geometry with a second, dense seed on the rectangle's
    right side, so that the flags fire and the rectangle grows at the first
    period ends: growth (Eq. 5a fill) and the E^2 sums at 512^2, with its
    many strips and blocks, against the FP64 oracle (its log replayed), read
    mid-period."""
    w = W.dmr_512_r2(precision=1)
    w = dict(w, seeds=list(w["seeds"]) + [(3e17, 272 / 512, 0.5, 0.125, 0.125)])
    sim = O.sim_from_workload(w)
    NT = w["cfg"]["steps_per_period"]
    steps = 4 * NT + 17
    sim.advance(steps)
    assert sim.log[0] != tuple(w["rect"]), "the rectangle should grow at the first period end"
    run = D.run_from_workload(w)
    run.set_graphs(True)
    run.replay_log(sim.log)
    run.advance(steps)
    assert run.get_patch() == tuple(sim.rect)
    compare(run, sim, TOL32, verbose=True)
    for level in (0, 1):
        assert rel_l2(run.read("erms", level).T, sim.erms(level)) <= TOL32


@pytest.mark.parametrize("r", [2, 4])
def test_full_size_large_fp32_in_the_bench_launch_shape(r):
    """The 2048x1024 workloads (eight seeds, the rectangle at 15 % of the
    domain) in the launch shape the benchmark times: the autotuner's strip
    heights and lane width (two node columns per lane in the fine sub-steps
    there), blocks away from every side on the path without edge tests,
    CUDA graphs.  Against the FP64 oracle: at r = 2 one period and three
    steps (the oracle's rectangle log replayed), at r = 4 nine coarse steps
    (36 fine sub-steps), read mid-period."""
    w = W.large_dmr(r=r)
    NT = w["cfg"]["steps_per_period"]
    steps = NT + 3 if r == 2 else 9
    sim = O.sim_from_workload(w)
    sim.advance(steps)
    run = D.run_from_workload(w)
    run.autotune()
    run.set_graphs(True)
    if sim.log:
        run.replay_log(sim.log)
    run.advance(steps)
    assert run.get_patch() == tuple(sim.rect)
    compare(run, sim, TOL32, verbose=True)


def test_capacity_error_and_state_errors():
    w = W.small_dmr()
    cfg = dict(w["cfg"], patch_cap_cells=4 * 12 * 10)
    run = D.Run(cfg)
    run.set_patch(w["rect"])
    run.seed_workload(w["seeds"])
    with pytest.raises(D.DMRError) as e:
        run.advance(3 * 32)
    assert e.value.code == D.ECAPACITY
    uni = D.Run(dict(w["cfg"], r=1))
    with pytest.raises(D.DMRError) as e:
        uni.set_patch((1, 1, 5, 5))
    assert e.value.code == D.ESTATE
    run2 = D.run_from_workload(w)
    run2.advance(3)
    with pytest.raises(D.DMRError) as e:
        run2.set_patch((0, 0, 40, 32))
    assert e.value.code == D.ESTATE
    run3 = D.run_from_workload(w)
    with pytest.raises(D.DMRError) as e:
        run3.set_patch((13, 10, 24, 20))
    assert e.value.code == D.EINVAL


def test_timing_counts_launches():
    w = W.small_dmr(precision=1)
    run = D.run_from_workload(w)
    run.set_timing(True)
    run.advance(32)
    kt = run.kernel_times()
    assert kt["em_step"][1] == 32 and kt["fine_em"][1] == 32
    assert all(v[0] > 0 for k, v in kt.items() if v[1] > 0)
    run.set_graphs(True)
    run.set_timing(True)
    run.advance(64)
    kt = run.kernel_times()
    assert kt["fine_em"][1] == 64 and kt["fine_em"][0] > 0
    # algorithmic bytes: 60 B per fine node per FP32 sub-step (44 B without an
    # E^2 sample), plus the coarse Ex, Ey means the last sub-step writes under
    # the rectangle (8 B per coarse node)
    ms, n, nbytes = kt["fine_em"]
    fr = run.get_patch()
    pts = (2 * (fr[2] - fr[0]) + 1) * (2 * (fr[3] - fr[1]) + 1)
    cpts = (fr[2] - fr[0] + 1) * (fr[3] - fr[1] + 1)
    assert n == 64 and nbytes <= 64 * (pts * 60 + cpts * 8)


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_leaves_run_unchanged(precision):
    w = W.small_dmr(precision=precision)
    a = D.run_from_workload(w)
    b = D.run_from_workload(w)
    a.advance(32)
    b.advance(32)
    wps, ms = b.autotune()
    assert wps in D.TUNE_WPS and len(ms) == len(D.TUNE_WPS) and all(t > 0 for t in ms)
    a.advance(2 * 32 + 7)
    b.advance(2 * 32 + 7)
    for level in (0, 1):
        for name in FIELDS + ("S2",):
            assert np.array_equal(a.read(name, level), b.read(name, level)), (level, name)


@pytest.mark.parametrize("precision", [0, 1])
def test_launch_timing_leaves_run_unchanged(precision):
    """dmr_time_launch (the bench's roofline timings) in all three forms, on
    a run mid-way through: the same bits afterwards as an untimed run."""
    w = W.small_dmr(precision=precision)
    a = D.run_from_workload(w)
    b = D.run_from_workload(w)
    a.advance(64)
    b.advance(64)
    for form in (0, 1, 2):
        ms, nbytes = b.time_launch(form, reps=4)
        assert ms > 0 and nbytes > 0
    # the mid-period form moves 16 B per node more (the FP64 E^2 sums)
    assert b.time_launch(1, 2)[1] > b.time_launch(0, 2)[1]
    a.advance(2 * 32 + 7)
    b.advance(2 * 32 + 7)
    assert a.get_patch() == b.get_patch()
    for level in (0, 1):
        for name in FIELDS + ("S2",):
            assert np.array_equal(a.read(name, level), b.read(name, level)), (level, name)
    with pytest.raises(D.DMRError) as e:
        b.time_launch(1)
    assert e.value.code == D.ESTATE


@pytest.mark.parametrize("graphs", [False, True])
def test_launch_modes_mixed_in_one_run(graphs):
    """Per-kernel timing switches the programmatic dependent launches off;
    switching it on and off between steps, mid-period and across periods,
    and reading state in between, gives the bits of an undisturbed run."""
    w = W.small_dmr(precision=1)
    ref = D.run_from_workload(w)
    run = D.run_from_workload(w)
    ref.set_graphs(graphs)
    run.set_graphs(graphs)
    for q, steps in enumerate((5, 27, 40, 32, 9)):
        run.set_timing(q % 2 == 0)
        run.advance(steps)
        ref.advance(steps)
        run.read("Ex", 0)
    assert run.get_patch() == ref.get_patch()
    for level in (0, 1):
        for name in FIELDS + ("S2",):
            assert np.array_equal(run.read(name, level), ref.read(name, level)), (level, name)
