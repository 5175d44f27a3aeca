"""The C-ABI library builds, loads and exports every entry point declared in
include/dmr.h; host-only calls (configuration checks) behave.  No kernel runs."""
import os
import re
import shutil

import pytest

from paper_2105_13276_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "dmr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dmr_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2105_13276_gb300 import build as B
    B.build()
    from paper_2105_13276_gb300 import dmr as D
    return D.load()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_config_validation_host_only(lib):
    from paper_2105_13276_gb300 import dmr as D
    assert D.workspace_bytes(W.dmr_512_r2()["cfg"]) > 0
    assert D.workspace_bytes(W.uniform_256()["cfg"]) > 0
    with pytest.raises(D.DMRError, match="Courant"):
        D.workspace_bytes(W.base_cfg(n_lambda=32, steps_per_period=32))
    with pytest.raises(D.DMRError, match="nx and ny"):
        D.workspace_bytes(W.base_cfg(nx=2))
    with pytest.raises(D.DMRError, match="precision"):
        D.workspace_bytes(W.base_cfg(precision=3))
    with pytest.raises(D.DMRError, match="diffusion number"):
        D.workspace_bytes(W.base_cfg(De=1e4))
    with pytest.raises(D.DMRError, match="growth"):
        D.workspace_bytes(W.base_cfg(growth=3))
    assert D.workspace_bytes(W.base_cfg(growth=2, m_ex=6, m_ey=2)) > 0
    with pytest.raises(D.DMRError, match="nu_model"):
        D.workspace_bytes(W.base_cfg(nu_model=2))
    assert D.workspace_bytes(W.base_cfg(nu_model=1, town_A=1e3, town_B=3e4)) > 0
    with pytest.raises(D.DMRError, match="coupling"):
        D.workspace_bytes(W.base_cfg(coupling=2))
    assert D.workspace_bytes(W.base_cfg(coupling=1)) == D.workspace_bytes(W.base_cfg())


def test_workspace_grows_with_capacity_and_precision(lib):
    from paper_2105_13276_gb300 import dmr as D
    c = W.dmr_512_r2()["cfg"]
    small = D.workspace_bytes(dict(c, patch_cap_cells=64 * 64))
    full = D.workspace_bytes(c)
    f64 = D.workspace_bytes(dict(c, precision=0))
    assert small < full < f64


def test_create_rejects_bad_arguments_without_gpu(lib):
    import ctypes
    from paper_2105_13276_gb300 import dmr as D
    c = D.make_config(W.small_dmr()["cfg"])
    ctx = ctypes.c_void_p()
    # misaligned workspace pointer is rejected before any CUDA call
    st = lib.dmr_create(ctypes.byref(c), ctypes.c_void_p(8), 1 << 30, None, ctypes.byref(ctx))
    assert st == D.EINVAL
    assert b"aligned" in lib.dmr_last_error(None)
    st = lib.dmr_create(ctypes.byref(c), ctypes.c_void_p(256), 16, None, ctypes.byref(ctx))
    assert st == D.ECAPACITY
    assert lib.dmr_kernel_class_name(0) == b"em_step"
    assert lib.dmr_kernel_class_name(99) is None


def test_config_struct_layout_matches_the_header(tmp_path):
    """The binding's dmr_config mirror has the header's field offsets and size
    (compiled with the host C compiler)."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    import ctypes
    import subprocess
    from paper_2105_13276_gb300 import dmr as D
    names = [f[0] for f in D.DmrConfig._fields_]
    src = tmp_path / "layout.c"
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dmr.h"', "int main(void) {",
             '  printf("size %zu\\n", sizeof(dmr_config));']
    lines += ['  printf("%s %%zu\\n", offsetof(dmr_config, %s));' % (n, n) for n in names]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = dict(ln.split() for ln in subprocess.run([str(exe)], check=True, capture_output=True,
                                                    text=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(D.DmrConfig)
    for n in names:
        assert int(out[n]) == getattr(D.DmrConfig, n).offset, n
    # and no header field is missing from the mirror (one could hide in padding)
    txt = open(os.path.join(ROOT, "include", "dmr.h")).read()
    body = txt[txt.index("typedef struct dmr_config {"):txt.index("} dmr_config;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S).split("{", 1)[1]
    declared = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            declared += [v.strip() for v in decl.split(None, 1)[1].split(",")]
    assert declared == names


def test_binding_constants_match_the_header():
    """Status codes, field ids and statistics slots of the binding equal the
    header's enumerations."""
    from paper_2105_13276_gb300 import dmr as D
    txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "dmr.h")).read(), flags=re.S)
    enum = {k: int(v) for k, v in re.findall(r"\b(DMR_[A-Z_0-9]+)\s*=\s*(-?\d+)", txt)}
    for code, name in D.STATUS_NAMES.items():
        assert enum[name] == code, name
    field_ids = {"Ex": "EX", "Ey": "EY", "Hz": "HZ", "vx": "VX", "vy": "VY", "n": "NE", "S2": "S2",
                 "mask": "MASK", "erms": "ERMS"}
    for py, c in field_ids.items():
        assert D.FIELDS[py] == enum["DMR_FIELD_" + c], py
    stats = {"t": "T", "R": "R", "fine_cells": "FINE_CELLS", "N_e": "NE", "P_abs": "PABS",
             "W_abs": "WABS", "periods": "PERIODS", "coarse_steps": "COARSE_STEPS", "n_max": "NMAX",
             "flags": "FLAGS"}
    assert len(D.STATS) == enum["DMR_NSTATS"]
    for k, name in enumerate(D.STATS):
        assert enum["DMR_STAT_" + stats[name]] == k, name
