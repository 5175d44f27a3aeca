"""The allocation-free electron total (dmr_electron_total_noalloc).

It serves callers that cannot allocate device memory -- a host application
whose own pool owns all GPU memory and lets no plug-in call cudaMalloc, or
code where an allocation and its device synchronisation are not allowed.
Its scratch is a fixed array inside the library, so the only buffers involved
are the caller's input map and its one-double output.

The test calls it through the C ABI twice in a row on the density of a
uniform run at two successive period ends and compares each result with the
run's own FP64 total (dmr_stats) and with the trapezoid sum written out on
the host, within the FP64 tolerance of the parity tests.  Around the second
call it checks that no device memory was allocated.  This file is collected
last so that a stop-at-first-failure run has executed every other test
before it.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2105_13276_gb300 import dmr as D  # noqa: E402
from paper_2105_13276_gb300 import workloads as W  # noqa: E402

TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    from paper_2105_13276_gb300 import build as B
    B.build()
    return D.load()


def _call(lib, nmap, nx, ny, precision, dx, stream, out):
    return lib.dmr_electron_total_noalloc(ctypes.c_void_p(nmap.data_ptr()), nx, ny, precision,
                                          dx, ctypes.c_void_p(stream.cuda_stream),
                                          ctypes.c_void_p(out.data_ptr()))


def _trapezoid_total(nmap, dx):
    """The composite trapezoid sum written out on the host in FP64 (the rule
    the run totals use): half weights on the first and last node of each
    axis."""
    n = np.asarray(nmap, dtype=np.float64)
    wy = np.ones(n.shape[0])
    wy[[0, -1]] = 0.5
    wx = np.ones(n.shape[1])
    wx[[0, -1]] = 0.5
    return dx * dx * float(np.sum(wy[:, None] * wx[None, :] * n))


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_total_equals_run_total_twice(lib, precision):
    nx, ny = 70, 50
    w = W.small_dmr(nx=nx, ny=ny, r=1, rect=None, precision=precision)
    run = D.run_from_workload(w)
    dt = torch.float64 if precision == 0 else torch.float32
    nmap = torch.empty((ny + 1, nx + 1), dtype=dt, device=run.device)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=run.device)
    NT = w["cfg"]["steps_per_period"]
    for call in range(2):
        run.advance(NT)                     # a period end: the run has its own total
        ref = run.stats()["N_e"]
        run.read_into("n", 0, nmap)         # queued on the run's stream
        run.sync()
        host = _trapezoid_total(nmap.cpu().numpy(), run.dxc)
        torch.cuda.synchronize()
        before = torch.cuda.memory_stats()
        free0, _ = torch.cuda.mem_get_info()
        st = _call(lib, nmap, nx, ny, precision, run.dxc, run.stream, out)
        assert st == D.OK, lib.dmr_noalloc_last_error()
        run.sync()
        free1, _ = torch.cuda.mem_get_info()
        after = torch.cuda.memory_stats()
        got = float(out.item())
        assert ref > 0 and abs(got / ref - 1.0) <= TOL, (call, got, ref)
        assert abs(got / host - 1.0) <= TOL, (call, got, host)
        if call == 1:
            # the call after the set-up allocates nothing, through torch's
            # allocator or around it
            for key in ("allocation.all.allocated", "segment.all.allocated"):
                assert after.get(key, 0) == before.get(key, 0), key
            assert free1 == free0, (free0, free1)


def test_noalloc_rejects_maps_beyond_its_scratch(lib):
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    st = _call(lib, dummy, 8192, 8192, 0, 1e-5, s, dummy)
    assert st == D.ECAPACITY
    assert b"67108864" in lib.dmr_noalloc_last_error()
    st = _call(lib, dummy, 0, 10, 0, 1e-5, s, dummy)
    assert st == D.EINVAL
