"""Slab decomposition of the time step over 2 and 3 ranks (gloo, CPU):
every field of the split run equals the unsplit oracle's bit for bit after
several periods; the FP64 totals, all-reduced from per-rank partial sums,
agree within rounding; the flags' bounding box and count, all-reduced with
MIN / MAX / SUM, equal the unsplit mask's."""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dmr_oracle as O  # noqa: E402
from paper_2105_13276_gb300 import workloads as W  # noqa: E402

FIELDS = ("Ex", "Ey", "Hz", "vx", "vy", "n", "S2")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, w, steps, path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    from oracle import dmr_oracle as O
    from oracle.dmr_slab import SlabSim
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        sim = SlabSim(w["cfg"], rank, world, None)
        sim.seed_from(O.sim_from_workload(w).coarse.n)
        sim.advance(steps)
        mine = {"a": sim.a, "b": sim.b, "N_e": sim.N_e, "P_abs": sim.P_abs, "W_abs": sim.W_abs,
                "bbox": sim.bbox, "nflag": sim.nflag}
        for f in FIELDS:
            mine[f] = sim.owned(f).copy()
        allp = [None] * world
        dist.all_gather_object(allp, mine)
        if rank == 0:
            out = {}
            for f in FIELDS:
                out[f] = np.concatenate([p[f] for p in allp], axis=0)
            for k in ("N_e", "P_abs", "W_abs", "nflag"):
                out[k] = np.array([p[k] for p in allp])
            out["bbox"] = np.array([p["bbox"] if p["bbox"] is not None else (-1, -1, -1, -1) for p in allp])
            np.savez(path, **out)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_split_equals_unsplit_oracle(world):
    w = W.small_dmr(nx=41, ny=24, r=1, rect=None)
    NT = w["cfg"]["steps_per_period"]
    steps = 3 * NT + 5
    ref = O.sim_from_workload(w)
    ref.advance(steps)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "slab.npz")
        torch.multiprocessing.spawn(_worker, args=(world, _free_port(), w, steps, path),
                                    nprocs=world, join=True)
        got = dict(np.load(path))
    for f in FIELDS:
        g, o = got[f], getattr(ref.coarse, f)
        assert g.shape == o.shape, f
        assert np.array_equal(g, o), (f, float(np.abs(g - o).max()))
    # every rank holds the same all-reduced totals
    for k, v in (("N_e", ref.N_e), ("P_abs", ref.P_abs), ("W_abs", ref.W_abs)):
        assert np.all(got[k] == got[k][0])
        assert abs(got[k][0] / v - 1.0) < 1e-13, (k, got[k][0], v)
    mask = O.flag_mask(ref.coarse.n, ref.P.n_th, ref.P.g_th, ref.P.dxc)
    assert mask.any(), "the case should have flagged nodes"
    assert np.all(got["nflag"] == int(mask.sum()))
    assert tuple(got["bbox"][0]) == O.mask_bbox(mask)


def test_slab_bounds_cover_the_mesh():
    from oracle.dmr_slab import slab_bounds
    for nx, world in ((41, 2), (41, 3), (10, 5), (127, 8)):
        b = slab_bounds(nx, world)
        assert b[0][0] == 0 and b[-1][1] == nx + 1
        assert all(b[k][1] == b[k + 1][0] for k in range(world - 1))
        assert all(hi - lo >= 2 for lo, hi in b)
    with pytest.raises(ValueError):
        slab_bounds(4, 3)


DMR_FIELDS = ("Ex", "Ey", "Hz", "vx", "vy", "n", "S2", "erms_last")


def _dmr_worker(rank, world, port, w, steps, path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    from oracle.dmr_slab import dmr_slab_from_workload
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        sim = dmr_slab_from_workload(w, rank, world)
        sim.advance(steps)
        mine = {"N_e": sim.N_e, "P_abs": sim.P_abs, "W_abs": sim.W_abs, "log": list(sim.log),
                "rect": sim.rect}
        for level in (0, 1):
            for f in DMR_FIELDS:
                mine[(level, f)] = sim.owned(level, f).copy()
        allp = [None] * world
        dist.all_gather_object(allp, mine)
        if rank == 0:
            out = {}
            for level in (0, 1):
                for f in DMR_FIELDS:
                    out["%d_%s" % (level, f)] = np.concatenate([p[(level, f)] for p in allp], axis=0)
            for k in ("N_e", "P_abs", "W_abs"):
                out[k] = np.array([p[k] for p in allp])
            out["log"] = np.array([p["log"] for p in allp])
            out["rect"] = np.array([p["rect"] for p in allp])
            np.savez(path, **out)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,r,growth,coupling", [(2, 2, 1, 0), (3, 2, 1, 0), (2, 4, 1, 0),
                                                     (3, 2, 2, 0), (2, 2, 1, 1)])
def test_dmr_slab_split_equals_unsplit_oracle(world, r, growth, coupling):
    """The DMR step over 2 and 3 slabs: a 40x32 coarse mesh, the rectangle
    (12, 10)-(24, 20) (threshold lines: (11, 13)-(16, 18)) cut by the slab
    boundaries and growing at the period ends (flag box or threshold lines; at
    r = 2 and 4; with both coupling readings).  Every field of both meshes, S2 and the E_rms of the last
    period equal the unsplit oracle's bit for bit, every rank took the same
    growth decisions as the oracle, and the all-reduced totals agree within
    rounding."""
    if growth == 2:
        w = W.small_dmr(r=r, growth=2, coupling=coupling, rect=(11, 13, 16, 18), n_th=3e16)
    else:
        w = W.small_dmr(r=r, growth=growth, coupling=coupling)
    NT = w["cfg"]["steps_per_period"]
    steps = 3 * NT + 5
    ref = O.sim_from_workload(w)
    ref.advance(steps)
    assert ref.log[-1] != tuple(w["rect"]), "the rectangle should grow"
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "dmr_slab.npz")
        torch.multiprocessing.spawn(_dmr_worker, args=(world, _free_port(), w, steps, path),
                                    nprocs=world, join=True)
        got = dict(np.load(path))
    for k in range(world):
        assert [tuple(x) for x in got["log"][k]] == list(ref.log), k
        assert tuple(got["rect"][k]) == tuple(ref.rect)
    for level, mesh in ((0, ref.coarse), (1, ref.fine)):
        for f in DMR_FIELDS:
            g, o = got["%d_%s" % (level, f)], getattr(mesh, f)
            assert g.shape == o.shape, (level, f, g.shape, o.shape)
            assert np.array_equal(g, o), (level, f, float(np.nanmax(np.abs(g - o))))
    for k, v in (("N_e", ref.N_e), ("P_abs", ref.P_abs), ("W_abs", ref.W_abs)):
        assert np.all(got[k] == got[k][0])
        assert abs(got[k][0] / v - 1.0) < 1e-13, (k, got[k][0], v)
