"""Batched runs: each run of a batch equals the same run done alone (bit for
bit, the batched launch evaluates the same operations), graphs equal direct
launches, the autotuner leaves the state unchanged, and a batched run matches
the FP64 oracle."""
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2105_13276_gb300 import build as B
    B.build()
    D.load()


def mixed(precision):
    """Uneven runs: sizes, E0, pressure, seed positions and rectangles differ."""
    out = []
    specs = [(40, 32, 5e6, 700.0, (12, 10, 24, 20)), (64, 48, 6e6, 500.0, (20, 14, 34, 30)),
             (36, 36, 4.5e6, 760.0, (0, 10, 12, 22)), (50, 30, 7e6, 300.0, (30, 0, 44, 12))]
    for q, (nx, ny, E0, p, rect) in enumerate(specs):
        w = W.small_dmr(nx=nx, ny=ny, rect=rect, precision=precision, E0=E0, p_torr=p)
        fx = (rect[0] + rect[2]) / 2 / nx
        fy = (rect[1] + rect[3]) / 2 / ny
        w["seeds"] = [(3e17, fx, fy, 0.1, 0.1)]
        out.append(w)
    return out


def same(a, b, levels=(0, 1)):
    assert a.get_patch() == b.get_patch()
    for level in levels:
        for name in FIELDS:
            x, y = a.read(name, level), b.read(name, level)
            assert np.array_equal(x, y), (level, name, np.abs(x - y).max())
    sa, sb = a.stats(), b.stats()
    for k in ("N_e", "P_abs", "W_abs"):
        assert sa[k] == sb[k], k


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("graphs", [False, True])
def test_batch_equals_single_runs(precision, graphs):
    ws = mixed(precision)
    b = D.batch_from_workloads(ws)
    b.set_graphs(graphs)
    singles = [D.run_from_workload(w) for w in ws]
    steps = 4 * 32 + 6
    b.advance(steps)
    for s in singles:
        s.advance(steps)
    for q in range(len(ws)):
        same(b.runs[q], singles[q])
    assert any(b.runs[q].get_patch() != tuple(ws[q]["rect"]) for q in range(len(ws)))
    assert b.launch_count() > 0


def test_batched_run_matches_oracle():
    ws = mixed(0)
    b = D.batch_from_workloads(ws)
    steps = 3 * 32 + 3
    b.advance(steps)
    for q in (0, 3):
        sim = O.sim_from_workload(ws[q])
        sim.advance(steps)
        run = b.runs[q]
        assert run.get_patch() == tuple(sim.rect)
        for level, mesh in ((0, sim.coarse), (1, sim.fine)):
            for name in FIELDS:
                g = run.read(name, level).T
                o = getattr(mesh, name)
                rel = np.linalg.norm(g - o) / max(np.linalg.norm(o), 1e-300)
                assert rel < 1e-12, (q, level, name, rel)


def test_full_size_batch_sampled_runs_match_oracle():
    """The 64-run batch the benchmark times (coarse 128^2 to 1024^2, r = 2,
    FP32), autotuned and in CUDA graphs, over one period and five steps; one
    run of each size (the first in the batch) against the FP64 oracle."""
    ws = W.batch_runs(64)
    steps = 64 + 5
    b = D.batch_from_workloads(ws)
    b.autotune()
    b.set_graphs(True)
    b.advance(steps)
    picks = {}
    for q, w in enumerate(ws):
        picks.setdefault(w["cfg"]["nx"], q)
    assert sorted(picks) == [128, 256, 512, 1024]
    for nx, q in sorted(picks.items()):
        sim = O.sim_from_workload(ws[q])
        sim.advance(steps)
        run = b.runs[q]
        assert run.get_patch() == tuple(sim.rect)
        for level, mesh in ((0, sim.coarse), (1, sim.fine)):
            for name in FIELDS + ("S2",):
                g = run.read(name, level).T.astype(np.float64)
                o = getattr(mesh, name)
                rel = np.linalg.norm(g - o) / max(np.linalg.norm(o), 1e-300)
                assert rel < 1e-4, (nx, q, level, name, rel)
        st = run.stats()
        assert abs(st["N_e"] / sim.N_e - 1) < 1e-4, (nx, q)


@pytest.mark.parametrize("graphs", [False, True])
def test_batch_with_threshold_line_growth(graphs):
    """Runs with both growth policies in one batch (Sec. III.D threshold lines
    for two of them): each batched run equals the same run alone, and the
    threshold-line run's rectangle log equals the FP64 oracle's."""
    ws = mixed(0)
    ws[1] = W.small_dmr(rect=(16, 14, 21, 18), growth=2, n_th=3e16)
    ws[2] = W.small_dmr(nx=44, ny=36, rect=(17, 15, 20, 17), growth=2, n_th=5e16, m_ex=30, m_ey=3)
    b = D.batch_from_workloads(ws)
    b.set_graphs(graphs)
    singles = [D.run_from_workload(w) for w in ws]
    steps = 3 * 32 + 4
    b.advance(steps)
    for s in singles:
        s.advance(steps)
    for q in range(len(ws)):
        same(b.runs[q], singles[q])
    sim = O.sim_from_workload(ws[1])
    sim.advance(steps)
    assert b.runs[1].get_patch() == tuple(sim.rect) != tuple(ws[1]["rect"])


def test_autotune_keeps_state_and_results():
    ws = mixed(1)
    a = D.batch_from_workloads(ws)
    b = D.batch_from_workloads(ws)
    a.advance(32)
    b.advance(32)
    wps, ms = b.autotune()
    assert wps in D.TUNE_WPS_BATCH and len(ms) == len(D.TUNE_WPS_BATCH) and all(t > 0 for t in ms)
    a.advance(2 * 32 + 5)
    b.advance(2 * 32 + 5)
    for q in range(len(ws)):
        same(a.runs[q], b.runs[q])


def test_batch_rejects_out_of_band_stepping():
    ws = mixed(1)
    b = D.batch_from_workloads(ws)
    b.advance(4)
    b.runs[1].advance(1)
    with pytest.raises(D.DMRError) as e:
        b.advance(4)
    assert e.value.code == D.ESTATE
