"""The persistent period launch (dmr_set_persistent): each full period's EM
steps (Sec. III.C sub-cycling) in one cooperative launch whose units wait
only for the units whose output they read.  It must give the bits of the
per-step launches, which the parity suite ties to the oracle:

* small DMR runs at r = 2, 3, 4, 8 in both precisions, with growth, graphs
  on and off, a partial period at the end (per-step launches mid-period);
* every rows-per-warp choice of its units;
* the CPML outer boundary and the uniform mesh;
* a 2048 x 1024 mesh at one row per warp, where every block takes several
  units of each step;
* directly against the FP64 oracle on one case;
* the bounded waits: a unit that waits for a count nothing reaches gives
  DMR_ETIMEOUT at the period end, the run then refuses to step, a loaded
  state continues with the bits of an undisturbed run, and the CUDA context
  stays usable.  The wait is made to run out on purpose by the test hook
  dmr_test_stall; nothing faults or hangs the GPU.
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

FIELDS = ("Ex", "Ey", "Hz", "vx", "vy", "n", "S2", "erms")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2105_13276_gb300 import build as B
    B.build()
    D.load()


def same_bits(a, b, fields=FIELDS):
    assert a.get_patch() == b.get_patch()
    levels = (0, 1) if a.get_patch()[0] >= 0 else (0,)
    for level in levels:
        for name in fields:
            ga, gb = a.read(name, level), b.read(name, level)
            assert np.array_equal(ga, gb), (level, name, float(np.abs(ga - gb).max()))
    sa, sb = a.stats(), b.stats()
    for k in ("N_e", "P_abs", "W_abs"):
        assert sa[k] == sb[k], k


def pair(w, graphs=False, rows=(0, 0)):
    ref = D.run_from_workload(w)
    run = D.run_from_workload(w)
    ref.set_graphs(graphs)
    run.set_graphs(graphs)
    run.set_persistent(True, *rows)
    return ref, run


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("r", [2, 3, 4, 8])
@pytest.mark.parametrize("graphs", [False, True])
def test_persistent_equals_per_step_launches(precision, r, graphs):
    w = W.small_dmr(r=r, precision=precision)
    NT = w["cfg"]["steps_per_period"]
    ref, run = pair(w, graphs)
    steps = 5 * NT + 7
    ref.advance(steps)
    run.advance(steps)
    assert run.get_patch() != tuple(w["rect"]), "the rectangle should grow"
    same_bits(ref, run)


@pytest.mark.parametrize("rows", [(1, 1), (2, 1), (3, 2), (4, 4), (8, 1), (64, 64)])
def test_persistent_rows_choices_give_identical_results(rows):
    w = W.small_dmr(precision=1)
    NT = w["cfg"]["steps_per_period"]
    ref, run = pair(w, True, rows)
    ref.advance(4 * NT)
    run.advance(4 * NT)
    same_bits(ref, run)


@pytest.mark.parametrize("r,precision", [(1, 0), (2, 0), (2, 1)])
def test_persistent_cpml(r, precision):
    if r == 1:
        w = W.small_dmr(nx=70, ny=50, r=1, rect=None, boundary=1, pml_cells=6, precision=precision)
    else:
        w = W.small_dmr(boundary=1, pml_cells=4, precision=precision)
    NT = w["cfg"]["steps_per_period"]
    ref, run = pair(w, True)
    ref.advance(4 * NT + 3)
    run.advance(4 * NT + 3)
    same_bits(ref, run)


@pytest.mark.parametrize("precision", [0, 1])
def test_persistent_uniform_mesh(precision):
    w = W.small_dmr(nx=70, ny=50, r=1, rect=None, precision=precision)
    NT = w["cfg"]["steps_per_period"]
    ref, run = pair(w, False)
    ref.advance(3 * NT)
    run.advance(3 * NT)
    same_bits(ref, run)


def test_persistent_several_units_per_block():
    """2048 x 1024 coarse, r = 2, one row per warp: ~18,000 coarse units and
    ~20,000 fine units per step, many more than resident blocks."""
    w = W.large_dmr(r=2)
    NT = w["cfg"]["steps_per_period"]
    ref, run = pair(w, True, (1, 1))
    ref.advance(2 * NT + 5)
    run.advance(2 * NT + 5)
    same_bits(ref, run, fields=("Ex", "Ey", "Hz", "vx", "n", "S2"))


def test_persistent_matches_fp64_oracle():
    w = W.small_dmr(precision=0)
    NT = w["cfg"]["steps_per_period"]
    sim = O.sim_from_workload(w)
    run = D.run_from_workload(w)
    run.set_persistent(True)
    run.set_graphs(True)
    sim.advance(4 * NT)
    run.advance(4 * NT)
    assert run.get_patch() == tuple(sim.rect)
    for level, mesh in ((0, sim.coarse), (1, sim.fine)):
        for name in ("Ex", "Ey", "Hz", "vx", "vy", "n"):
            g = run.read(name, level).T
            o = getattr(mesh, name)
            e = float(np.linalg.norm(g - o) / np.linalg.norm(o))
            assert e <= 1e-12, (level, name, e)


def test_bounded_wait_gives_up_and_a_loaded_state_continues():
    w = W.small_dmr(precision=1)
    NT = w["cfg"]["steps_per_period"]
    ref = D.run_from_workload(w)
    run = D.run_from_workload(w)
    run.set_persistent(True)
    ref.advance(2 * NT)
    run.advance(2 * NT)
    saved = run.save_state()
    run.test_stall(True, polls=20000)
    with pytest.raises(D.DMRError) as e:
        run.advance(NT)
    assert e.value.code == D.ETIMEOUT
    with pytest.raises(D.DMRError) as e:
        run.advance(1)
    assert e.value.code == D.ESTATE
    run.test_stall(False, polls=1 << 22)
    run.load_state(saved)
    run.advance(2 * NT + 3)
    ref.advance(2 * NT + 3)
    same_bits(ref, run)
    # the context is still usable: a fresh run steps as before
    fresh = D.run_from_workload(w)
    fresh.set_persistent(True)
    fresh.advance(4 * NT + 3)
    same_bits(ref, fresh)


def test_persistent_setter_rejections():
    w = W.small_dmr()
    run = D.run_from_workload(w)
    with pytest.raises(D.DMRError) as e:
        run.set_persistent(True, 65, 0)
    assert e.value.code == D.EINVAL
    with pytest.raises(D.DMRError) as e:
        run.test_stall(True, polls=0)
    assert e.value.code == D.EINVAL
