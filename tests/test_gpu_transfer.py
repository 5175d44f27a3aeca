"""Fine -> coarse E transfer (a8, Sec. III.C), which the last fine sub-step of
every coarse step writes into the coarse arrays: after any step the coarse E
edges of the transfer set hold the mean of their r collinear fine edges, bit
for bit (the same sum, q = 0 .. r-1, times 1/r, in the run's precision), for
every refinement factor (strip widths 30, 28 and 24, one or several rows per
warp) and for rectangle sides inside the domain and on its edges (Mur); and
runs with r = 3, 4 and 8 match the FP64 oracle."""
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
NX, NY = 40, 32


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2105_13276_gb300 import build as B
    B.build()
    D.load()


def fine_mean(run, r, dtype, nx=NX, ny=NY):
    """Expected coarse Ex, Ey on the transfer set from the fine arrays (coarse
    mesh nx x ny cells)."""
    I0, J0, I1, J1 = run.get_patch()
    fex, fey = run.read("Ex", 1), run.read("Ey", 1)          # [row, column]
    jlo = J0 if J0 == 0 else J0 + 1
    jhi = J1 if J1 == ny else J1 - 1
    ilo = I0 if I0 == 0 else I0 + 1
    ihi = I1 if I1 == nx else I1 - 1
    rinv = dtype(1.0 / r)
    ex = {}
    for J in range(jlo, jhi + 1):
        row = fex[r * (J - J0), :].reshape(I1 - I0, r)
        acc = row[:, 0].copy()
        for q in range(1, r):
            acc = acc + row[:, q]
        ex[J] = acc * rinv
    ey = {}
    for I in range(ilo, ihi + 1):
        col = fey[:, r * (I - I0)].reshape(J1 - J0, r)
        acc = col[:, 0].copy()
        for q in range(1, r):
            acc = acc + col[:, q]
        ey[I] = acc * rinv
    return (I0, J0, I1, J1), ex, ey


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("r", [2, 3, 4, 5, 8])
@pytest.mark.parametrize("rect", [(12, 10, 24, 20), (0, 0, 14, 12), (26, 20, 40, 32)])
def test_coarse_holds_fine_mean(precision, r, rect):
    w = W.small_dmr(nx=NX, ny=NY, r=r, rect=rect, precision=precision)
    run = D.run_from_workload(w)
    run.set_graphs(True)
    dtype = np.float32 if precision == 1 else np.float64
    for steps in (5, 38, 30):                 # checks at steps 5, 43, 73: mid-period, after growth
        run.advance(steps)
        (I0, J0, I1, J1), ex, ey = fine_mean(run, r, dtype)
        cex, cey = run.read("Ex", 0), run.read("Ey", 0)
        for J, v in ex.items():
            assert np.array_equal(cex[J, I0:I1], v), ("Ex", J)
        for I, v in ey.items():
            assert np.array_equal(cey[J0:J1, I], v), ("Ey", I)
    assert run.get_patch() != tuple(rect)      # grew on the way


@pytest.mark.parametrize("r", [3, 4, 8])
@pytest.mark.parametrize("rect", [(12, 10, 24, 20), (0, 0, 14, 12)])
def test_dmr_r3_r4_r8_match_oracle(r, rect):
    w = W.small_dmr(nx=NX, ny=NY, r=r, rect=rect)
    run = D.run_from_workload(w)
    run.set_graphs(True)
    sim = O.sim_from_workload(w)
    steps = 2 * 32 + 3
    run.advance(steps)
    sim.advance(steps)
    assert run.get_patch() == tuple(sim.rect)
    for level, mesh in ((0, sim.coarse), (1, sim.fine)):
        for name in FIELDS:
            g = run.read(name, level).T
            o = getattr(mesh, name)
            rel = np.linalg.norm(g - o) / max(np.linalg.norm(o), 1e-300)
            assert rel < 1e-12, (level, name, rel)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("r", [2, 4])
@pytest.mark.parametrize("wps", [1, 1024])
def test_coarse_holds_fine_mean_many_rows(precision, r, wps):
    """A larger rectangle: at a low warps-per-SM target the last sub-step's
    warps cover several rows (Ey summed in the warp), at a high one a single
    row (Ey summed across the warps of a block)."""
    nx, ny = 120, 96
    w = W.small_dmr(nx=nx, ny=ny, r=r, rect=(20, 16, 100, 80), precision=precision)
    w["seeds"] = [(3e17, 0.5, 0.5, 0.1, 0.1)]
    run = D.run_from_workload(w)
    run.set_graphs(True)
    run.set_launch_shape(wps)
    dtype = np.float32 if precision == 1 else np.float64
    for steps in (5, 38):
        run.advance(steps)
        (I0, J0, I1, J1), ex, ey = fine_mean(run, r, dtype, nx, ny)
        cex, cey = run.read("Ex", 0), run.read("Ey", 0)
        for J, v in ex.items():
            assert np.array_equal(cex[J, I0:I1], v), ("Ex", J)
        for I, v in ey.items():
            assert np.array_equal(cey[J0:J1, I], v), ("Ey", I)
