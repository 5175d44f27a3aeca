"""Two node columns per lane in the fine sub-steps with launches of their own
(dmr_set_strip_columns(2): float2 loads and stores, one lane shuffle for two
nodes).

Every element is computed by the same operations in the same order as with
one column per lane, so FP32 runs give the same bits: all fields, the E^2
sums, the rectangle log and the FP64 totals, with growth, CUDA graphs and
programmatic launches, for r = 2 and 4 (two columns in the last fine
sub-step, which writes the fine->coarse means), r = 3 (sub-step 2 with two
columns, the last one with one), rectangles on the domain edges (fine Mur
sides), the threshold-line growth, several strips with a ragged last one,
odd and even mesh widths (a Mur column at either lane slot) and rectangles
wide enough for strips away from every side (the path without edge tests).
One case is also checked against the FP64 oracle directly.
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

FIELDS = ("Ex", "Ey", "Hz", "vx", "vy", "n", "S2")
TOL32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2105_13276_gb300 import build as B
    B.build()
    D.load()


def _case(name):
    if name == "r2":
        return W.small_dmr(precision=1)
    if name == "r2_edges_low":
        return W.small_dmr(precision=1, rect=(0, 0, 10, 9))
    if name == "r2_edges_high":
        return W.small_dmr(precision=1, rect=(28, 20, 40, 32))
    if name == "r2_odd_nx":
        return W.small_dmr(nx=41, ny=33, precision=1, rect=(13, 9, 41, 21))
    if name == "r4":
        return W.small_dmr(r=4, precision=1)
    if name == "r4_edges":
        return W.small_dmr(r=4, precision=1, rect=(0, 20, 9, 32))
    if name == "r3":
        return W.small_dmr(r=3, precision=1)
    if name == "r2_lines":
        return W.small_dmr(precision=1, growth=2, n_th=3e16)
    if name == "r2_many_strips":
        return W.small_dmr(nx=131, ny=70, rect=(40, 30, 101, 52), precision=1)
    if name == "r2_wide":      # fine strips away from every side (the path without edge tests)
        return W.small_dmr(nx=160, ny=64, rect=(20, 10, 100, 54), precision=1)
    if name == "r4_wide":
        return W.small_dmr(nx=100, ny=64, r=4, rect=(20, 10, 60, 40), precision=1)
    raise KeyError(name)


def _run(w, cols, graphs=True, wps=None, steps=None):
    run = D.run_from_workload(w)
    run.set_graphs(graphs)
    if wps is not None:
        run.set_launch_shape(wps)
    run.set_strip_columns(cols)
    NT = w["cfg"]["steps_per_period"]
    run.advance(steps if steps is not None else 3 * NT + 5)
    return run


def _same(a, b, w, tag):
    levels = (0, 1) if w["cfg"].get("r", 1) > 1 else (0,)
    assert a.get_patch() == b.get_patch(), tag
    for level in levels:
        for name in FIELDS:
            assert np.array_equal(a.read(name, level), b.read(name, level)), (tag, level, name)
    sa, sb = a.stats(), b.stats()
    for k in ("N_e", "P_abs", "W_abs", "fine_cells", "n_max"):
        assert sa[k] == sb[k], (tag, k)


@pytest.mark.parametrize("name", ["r2", "r2_edges_low", "r2_edges_high", "r2_odd_nx", "r4",
                                  "r4_edges", "r3", "r2_lines", "r2_many_strips", "r2_wide",
                                  "r4_wide"])
def test_two_columns_per_lane_give_the_same_bits(name):
    w = _case(name)
    ref = _run(w, 1)
    for wps in (None, 1, 96):
        run = _run(w, 2, wps=wps)
        ref_w = ref if wps is None else _run(w, 1, wps=wps)
        _same(run, ref_w, w, (name, wps))
        assert run.launch_shape()[2] == 2


def test_two_columns_direct_launches_and_switch_mid_run():
    """Direct launches (no graphs), and the width switched between periods."""
    w = _case("r2")
    NT = w["cfg"]["steps_per_period"]
    ref = _run(w, 1, graphs=False)
    run = D.run_from_workload(w)
    run.set_strip_columns(2)
    run.advance(NT + 3)
    run.set_strip_columns(1)
    run.advance(NT)
    run.set_strip_columns(2)
    run.set_graphs(True)
    run.advance(NT + 2)
    _same(run, ref, w, "switch")


def test_two_columns_match_the_fp64_oracle():
    """Several strips on both levels, the oracle's rectangle log replayed."""
    w = W.small_dmr(nx=128, ny=96, rect=(40, 30, 80, 62), precision=1)
    NT = w["cfg"]["steps_per_period"]
    sim = O.sim_from_workload(w)
    ref = O.sim_from_workload(w)
    ref.advance(2 * NT + 7)
    run = D.run_from_workload(w)
    run.set_strip_columns(2)
    run.replay_log(ref.log)
    sim.advance(2 * NT + 7)
    run.advance(2 * NT + 7)
    assert run.get_patch() == tuple(sim.rect)
    for level, mesh in ((0, sim.coarse), (1, sim.fine)):
        for name in ("Ex", "Ey", "Hz", "vx", "vy", "n"):
            g = run.read(name, level).T.astype(np.float64)
            o = getattr(mesh, name)
            rel = np.linalg.norm(g - o) / max(np.linalg.norm(o), 1e-300)
            assert rel <= TOL32, (level, name, rel)


def test_full_size_512_two_columns_same_bits_and_autotune():
    """The 512^2 r = 2 benchmark geometry over two periods and a part, graphs
    and programmatic launches on; the autotuner (which tries both widths)
    leaves the run unchanged."""
    w = W.dmr_512_r2(precision=1)
    NT = w["cfg"]["steps_per_period"]
    ref = _run(w, 1, steps=2 * NT + 9)
    run = _run(w, 2, steps=2 * NT + 9)
    _same(run, ref, w, "512")
    t = D.run_from_workload(w)
    t.advance(NT)
    t.autotune()
    assert t.launch_shape()[2] in (1, 2)
    t.set_graphs(True)
    t.advance(NT + 9)
    _same(t, ref, w, "512 autotuned")


def test_strip_columns_rejections():
    w = _case("r2")
    run = D.run_from_workload(w)
    for bad in (0, 3):
        with pytest.raises(D.DMRError) as e:
            run.set_strip_columns(bad)
        assert e.value.code == D.EINVAL
