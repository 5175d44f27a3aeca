"""The E_rms output, checkpoint / resume of a run, and the stability guard,
through the C ABI on the GPU.

* E_rms(x, y, t) (Sec. II.B, Sec. IV output) against the oracle's reading:
  the running RMS within a period, the completed period's value at a
  boundary (with growth filling new area by Eq. 5a).  FP64 <= 1e-12
  relative L2, FP32 <= 1e-4 with the oracle's log replayed.
* dmr_save_state / dmr_load_state: save, advance, load, advance again gives
  the bits of the first continuation, in the same context and in a fresh
  one; the rectangle and counters are restored.
* The stability guard (DMR_EUNSTABLE at a period end on a NaN, or on a
  density with w_p dt >= 2) is triggered by writing such a density through
  dmr_write: a host-side data injection, nothing faults the GPU.
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
QE, ME, EPS0 = 1.602176634e-19, 9.1093837015e-31, 8.8541878128e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2105_13276_gb300 import build as B
    B.build()
    D.load()


def rel_l2(g, o):
    no = np.linalg.norm(o)
    return float(np.linalg.norm(g.astype(np.float64) - o) / no) if no else float(np.linalg.norm(g))


@pytest.mark.parametrize("precision", [0, 1])
def test_erms_matches_oracle(precision):
    """Mid-period and at period boundaries, coarse and fine, through growth."""
    w = W.small_dmr(precision=precision)
    sim = O.sim_from_workload(w)
    NT = w["cfg"]["steps_per_period"]
    run = D.run_from_workload(w)
    if precision:
        ref = O.sim_from_workload(w)
        ref.advance(3 * NT)
        run.replay_log(ref.log)
    tol = 1e-12 if precision == 0 else 1e-4
    grew = False
    for steps in (5, NT - 5, 13, NT - 13, NT):
        sim.advance(steps)
        run.advance(steps)
        assert run.get_patch() == tuple(sim.rect)
        grew |= tuple(sim.rect) != tuple(w["rect"])
        for level in (0, 1):
            g = run.read("erms", level).T
            o = sim.erms(level)
            assert g.shape == o.shape
            assert o.max() > 0
            e = rel_l2(g, o)
            assert e <= tol, (steps, level, e)
    assert grew


def test_erms_is_read_only_and_shaped_like_the_density():
    w = W.small_dmr()
    run = D.run_from_workload(w)
    assert run.shape("erms", 0) == run.shape("n", 0)
    assert run.shape("erms", 1) == run.shape("n", 1)
    with pytest.raises(D.DMRError) as e:
        run.write("erms", 0, np.zeros(run.shape("erms", 0)[0]))
    assert e.value.code == D.EINVAL


def _snapshot(run):
    return {(lvl, f): run.read(f, lvl) for lvl in (0, 1) for f in FIELDS}


def _same(a, b):
    assert a.keys() == b.keys()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("precision,graphs", [(0, False), (1, True)])
def test_save_advance_load_advance_is_bit_identical(precision, graphs):
    """Save mid-period, advance through growth, load, advance the same steps:
    the same bits, rectangle and counters; a fresh context of the same
    configuration continues from the saved state with the same bits too."""
    w = W.small_dmr(precision=precision)
    NT = w["cfg"]["steps_per_period"]
    run = D.run_from_workload(w)
    run.set_graphs(graphs)
    run.advance(7)                               # mid-period, before the first growth
    rect0, st0 = run.get_patch(), run.stats()
    buf = run.save_state()
    assert buf.numel() == run.lib.dmr_state_bytes(run.ctx)
    run.advance(3 * NT)                          # through period ends and growth
    first = _snapshot(run)
    rect1, st1 = run.get_patch(), run.stats()
    assert rect1 != rect0, "the rectangle should grow after the save"
    run.load_state(buf)
    assert run.get_patch() == rect0
    assert run.stats() == st0
    run.advance(3 * NT)
    _same(_snapshot(run), first)
    assert run.get_patch() == rect1 and run.stats() == st1
    fresh = D.Run(w["cfg"])
    fresh.set_graphs(graphs)
    fresh.load_state(buf)
    assert fresh.get_patch() == rect0
    fresh.advance(3 * NT)
    _same(_snapshot(fresh), first)


def test_state_of_a_uniform_run_and_replay_position():
    """r = 1 runs save and load too; a replayed refinement log resumes at the
    period it stood at when the state was saved."""
    u = W.small_dmr(nx=40, ny=32, r=1, rect=None)
    a = D.run_from_workload(u)
    a.advance(40)
    buf = a.save_state()
    a.advance(50)
    ua = a.read("n")
    a.load_state(buf)
    a.advance(50)
    assert np.array_equal(a.read("n"), ua)

    w = W.small_dmr(precision=1)
    NT = w["cfg"]["steps_per_period"]
    ref = O.sim_from_workload(w)
    ref.advance(4 * NT)
    run = D.run_from_workload(w)
    run.replay_log(ref.log)
    run.advance(2 * NT)
    buf = run.save_state()
    run.advance(2 * NT)
    assert run.get_patch() == tuple(ref.log[3])
    other = D.run_from_workload(w)
    other.replay_log(ref.log)
    other.load_state(buf)
    other.advance(2 * NT)
    assert other.get_patch() == tuple(ref.log[3])
    assert np.array_equal(other.read("n", 1), run.read("n", 1))


def test_load_state_rejects_other_configurations_and_small_buffers():
    w = W.small_dmr()
    run = D.run_from_workload(w)
    buf = run.save_state()
    other = D.Run(dict(w["cfg"], E0=w["cfg"]["E0"] * 1.01))
    with pytest.raises(D.DMRError) as e:
        other.load_state(buf)
    assert e.value.code == D.EINVAL
    with pytest.raises(D.DMRError) as e:
        run.load_state(buf[:1024])
    assert e.value.code == D.ECAPACITY
    junk = torch.zeros_like(buf)
    with pytest.raises(D.DMRError) as e:
        run.load_state(junk)
    assert e.value.code == D.EINVAL
    with pytest.raises(D.DMRError) as e:
        run.save_state(torch.empty(1024, dtype=torch.uint8, device="cuda"))
    assert e.value.code == D.ECAPACITY


def _guard_case(precision, level, value, at_step):
    """A run with a density injected at one node after at_step coarse steps:
    a coarse node outside the rectangle (level 0, else the fine density
    would be injected over it at the period end) or the fine rectangle's
    centre node (level 1)."""
    w = W.small_dmr(precision=precision)
    NT = w["cfg"]["steps_per_period"]
    run = D.run_from_workload(w)
    run.advance(at_step)
    n = run.read("n", level).copy()
    j, i = (2, 2) if level == 0 else (n.shape[0] // 2, n.shape[1] // 2)
    if level == 0:
        i0, j0, i1, j1 = run.get_patch()
        assert not (i0 <= i <= i1 and j0 <= j <= j1)
    n[j, i] = value
    run.write("n", level, n)
    return run, NT


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("level", [0, 1])
def test_nan_density_stops_the_run_at_the_next_period_end(precision, level):
    w = W.small_dmr()
    NT = w["cfg"]["steps_per_period"]
    run, NT = _guard_case(precision, level, np.nan, NT)
    rect = run.get_patch()
    run.advance(NT - 1)                         # no period end yet: nothing checked
    with pytest.raises(D.DMRError) as e:
        run.advance(5)
    assert e.value.code == D.EUNSTABLE
    assert "NaN" in str(e.value)
    st = run.stats()
    # the run stopped right at the period end that found it, rectangle kept
    assert st["coarse_steps"] == 2 * NT and st["periods"] == 2
    assert run.get_patch() == rect


@pytest.mark.parametrize("precision", [0, 1])
def test_over_dense_plasma_stops_the_run(precision):
    """w_p dt >= 2 (the explicit plasma-current update's limit): the density
    bound n = (2/dt)^2 m eps0 / e^2 with the fine step dt of a DMR run.  The
    density is injected two coarse steps before a period end, so the fields
    it destabilises stay finite until the guard reads it."""
    w = W.small_dmr(precision=precision)
    c = w["cfg"]
    NT = c["steps_per_period"]
    dtf = 1.0 / (c["freq"] * c["r"] * NT)
    n_lim = (2.0 / dtf) ** 2 * ME * EPS0 / QE ** 2
    run, NT = _guard_case(precision, 0, 2.0 * n_lim, 2 * NT - 2)
    rect = run.get_patch()
    with pytest.raises(D.DMRError) as e:
        run.advance(2)
    assert e.value.code == D.EUNSTABLE
    assert "w_p dt" in str(e.value)
    st = run.stats()
    assert st["coarse_steps"] == 2 * NT and st["periods"] == 2 and st["n_max"] >= n_lim
    assert run.get_patch() == rect
