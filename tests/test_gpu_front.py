"""Front-velocity experiment of Sec. IV.B on the GPU: a 1.5 x 1.5 wavelength
domain in air at 760 Torr, E0 = 5.5 MV/m at 110 GHz, a Gaussian seed of
1e16 m^-3 at (0.85 Lx, 0.5 Ly).  The paper reports the plasma front moving
towards the source with the uniform fine mesh and DMR at r = 2 within 1-2 %
of each other.  Here the DMR runs (coarse lambda/64, r = 2, flag-box growth
and the paper's threshold-line growth) are checked against the uniform
lambda/128 mesh they refine to: the front (the
n = 1e19 m^-3 crossing on the central x line) is tracked every 50 periods
and its velocity fitted where it lies 1.0 to 0.3 wavelengths from the left
edge; the velocities agree within 2 %.  (The absolute velocity follows
the ionization and diffusion readings, which the paper leaves to cited
works; at r = 4 a slowly growing mode of the coarse-fine coupling drives the
density up near the interface; with coupling = 1, the density alone going
back to the coarse mesh, the interface has no growing mode, and r = 4 with
the threshold lines lands within 2 % as well.)"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from bench import front_x  # noqa: E402
from paper_2105_13276_gb300 import dmr as D  # noqa: E402
from paper_2105_13276_gb300 import workloads as W  # noqa: E402

LAM = 299792458.0 / 110e9
PERIOD = 1.0 / 110e9


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2105_13276_gb300 import build as B
    B.build()
    D.load()


def front_velocity(w, periods=5000, chunk=50):
    cfg = w["cfg"]
    run = D.run_from_workload(w)
    run.set_graphs(True)
    track = []
    for p in range(0, periods, chunk):
        run.advance(chunk * cfg["steps_per_period"])
        track.append(((p + chunk) * PERIOD, front_x(run, cfg, LAM)))
    pts = [(t, x) for t, x in track if x is not None and 0.3 * LAM <= x <= 1.0 * LAM]
    assert len(pts) >= 10, "the front should cross the fitting window"
    t, x = np.array(pts).T
    return -float(np.polyfit(t, x, 1)[0])


def test_dmr_r2_front_velocity_within_two_percent_of_uniform():
    v_uni = front_velocity(W.front_1p5(128, 1))
    v_dmr = front_velocity(W.front_1p5(64, 2, growth=1))
    print("front velocity: uniform lambda/128 %.1f km/s, DMR r=2 %.1f km/s (%+.2f %%)"
          % (v_uni / 1e3, v_dmr / 1e3, 100.0 * (v_dmr / v_uni - 1.0)))
    assert v_uni > 0 and v_dmr > 0
    assert abs(v_dmr / v_uni - 1.0) <= 0.02


def test_dmr_r2_threshold_lines_front_velocity_within_two_percent():
    """The paper's own expansion rule (threshold lines, Sec. III.D) with
    jumps m_ex = 32, m_ey = 16 coarse cells (the paper gives only m_ex > m_ey;
    with 8 and 4 the rectangle lags the front and it runs 5.6 % fast)."""
    v_uni = front_velocity(W.front_1p5(128, 1))
    w = W.front_1p5(64, 2, growth=2)
    w["cfg"] = dict(w["cfg"], m_ex=32, m_ey=16)
    v_dmr = front_velocity(w)
    print("front velocity: uniform lambda/128 %.1f km/s, DMR r=2 threshold lines %.1f km/s (%+.2f %%)"
          % (v_uni / 1e3, v_dmr / 1e3, 100.0 * (v_dmr / v_uni - 1.0)))
    assert abs(v_dmr / v_uni - 1.0) <= 0.02


def test_dmr_r4_one_way_threshold_lines_front_velocity_within_two_percent():
    """r = 4 (coarse lambda/64, fine lambda/256) with the threshold lines
    (m_ex = 32, m_ey = 16) and coupling = 1: the run stays bounded over the
    5000 periods and the front moves within 2 % of the uniform lambda/128
    mesh (-0.1 % measured; with the two-way coupling the r = 4 run runs away)."""
    v_uni = front_velocity(W.front_1p5(128, 1))
    w = W.front_1p5(64, 4, growth=2)
    w["cfg"] = dict(w["cfg"], m_ex=32, m_ey=16, coupling=1)
    v_dmr = front_velocity(w)
    print("front velocity: uniform lambda/128 %.1f km/s, DMR r=4 one-way threshold lines %.1f km/s (%+.2f %%)"
          % (v_uni / 1e3, v_dmr / 1e3, 100.0 * (v_dmr / v_uni - 1.0)))
    assert abs(v_dmr / v_uni - 1.0) <= 0.02
