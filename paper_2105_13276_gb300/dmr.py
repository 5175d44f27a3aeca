"""Thin ctypes binding of ``libdmr.so`` (the C ABI in include/dmr.h).

Argument marshalling only: every step of the time stepping runs in the CUDA
kernels of the library.  PyTorch provides the device workspace and the
stream.  If the library is missing this module raises; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t, c_void_p

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libdmr.so")

# status codes
OK, EINVAL, ECAPACITY, ECUDA, EUNSTABLE, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "DMR_OK", -1: "DMR_EINVAL", -2: "DMR_ECAPACITY", -3: "DMR_ECUDA",
                -4: "DMR_EUNSTABLE", -5: "DMR_ETIMEOUT", -6: "DMR_ESTATE"}

FIELDS = {"Ex": 0, "Ey": 1, "Hz": 2, "vx": 3, "vy": 4, "n": 5, "S2": 6, "mask": 7,
          "erms": 8}
STATS = ["t", "R", "fine_cells", "N_e", "P_abs", "W_abs", "periods", "coarse_steps", "n_max",
         "flags"]
# strip heights the autotuners try, as warps-per-SM targets (trial_ms order)
TUNE_WPS = (8, 16, 32, 48, 96)          # dmr_autotune candidates (warps per SM)
TUNE_WPS_BATCH = (1, 2, 4, 8, 16)       # dmr_batch_autotune candidates

C0 = 299792458.0


class DmrConfig(ctypes.Structure):
    _fields_ = [("nx", c_int32), ("ny", c_int32), ("r", c_int32), ("n_lambda", c_int32),
                ("steps_per_period", c_int32), ("precision", c_int32),
                ("buffer_cells", c_int32), ("growth", c_int32), ("patch_cap_cells", c_int64),
                ("freq", c_double), ("E0", c_double), ("p_torr", c_double),
                ("De", c_double), ("Da", c_double), ("beta_rec", c_double), ("Te", c_double),
                ("nu_scale", c_double), ("nu_a", c_double), ("n_th", c_double),
                ("g_th", c_double), ("m_ex", c_int32), ("m_ey", c_int32),
                ("nu_model", c_int32), ("town_A", c_double), ("town_B", c_double),
                ("boundary", c_int32), ("pml_cells", c_int32),
                ("coupling", c_int32)]


class DMRError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, code), msg))
        self.code = code


_LIB = None


def load():
    """Load libdmr.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libdmr.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P = c_void_p
    sig = {
        "dmr_workspace_bytes": (c_size_t, [POINTER(DmrConfig)]),
        "dmr_create": (c_int, [POINTER(DmrConfig), P, c_size_t, P, POINTER(P)]),
        "dmr_destroy": (None, [P]),
        "dmr_last_error": (c_char_p, [P]),
        "dmr_seed_gaussian": (c_int, [P, c_double, c_double, c_double, c_double, c_double, c_int]),
        "dmr_set_patch": (c_int, [P, POINTER(c_int32)]),
        "dmr_get_patch": (c_int, [P, POINTER(c_int32)]),
        "dmr_advance": (c_int, [P, c_int64]),
        "dmr_replay_log": (c_int, [P, POINTER(c_int32), c_int64]),
        "dmr_field_shape": (c_int, [P, c_int, c_int, POINTER(c_int32), POINTER(c_int32)]),
        "dmr_read": (c_int, [P, c_int, c_int, P, c_size_t, c_int]),
        "dmr_write": (c_int, [P, c_int, c_int, P, c_size_t, c_int]),
        "dmr_stats": (c_int, [P, POINTER(c_double)]),
        "dmr_set_graphs": (c_int, [P, c_int]),
        "dmr_set_launch_shape": (c_int, [P, c_int32]),
        "dmr_set_strip_columns": (c_int, [P, c_int32]),
        "dmr_get_launch_shape": (c_int, [P, POINTER(c_int32)]),
        "dmr_set_persistent": (c_int, [P, c_int, c_int32, c_int32]),
        "dmr_test_stall": (c_int, [P, c_int, c_int64]),
        "dmr_set_timing": (c_int, [P, c_int]),
        "dmr_kernel_time": (c_int, [P, c_int, POINTER(c_double), POINTER(c_int64),
                                    POINTER(c_double)]),
        "dmr_kernel_class_name": (c_char_p, [c_int]),
        "dmr_launch_count": (c_int, [P, POINTER(c_int64)]),
        "dmr_sync": (c_int, [P]),
        "dmr_autotune": (c_int, [P, POINTER(c_int32), POINTER(c_double)]),
        "dmr_electron_total_noalloc": (c_int, [P, c_int32, c_int32, c_int32, c_double, P, P]),
        "dmr_adjoint_checkpoint_bytes": (c_size_t, [P, c_int64, c_int64]),
        "dmr_adjoint_record": (c_int, [P, c_int64, c_int64, P, c_size_t]),
        "dmr_adjoint_workspace_bytes": (c_size_t, [P]),
        "dmr_adjoint_backward": (c_int, [P, P, P, c_size_t, P, c_size_t, POINTER(c_double),
                                         POINTER(c_double), P]),
        "dmr_batch_workspace_bytes": (c_size_t, [POINTER(DmrConfig), c_int32]),
        "dmr_batch_create": (c_int, [POINTER(DmrConfig), c_int32, P, c_size_t, P, POINTER(P)]),
        "dmr_batch_destroy": (None, [P]),
        "dmr_batch_run": (P, [P, c_int32]),
        "dmr_batch_advance": (c_int, [P, c_int64]),
        "dmr_batch_set_graphs": (c_int, [P, c_int]),
        "dmr_batch_autotune": (c_int, [P, POINTER(c_int32), POINTER(c_double)]),
        "dmr_batch_launch_count": (c_int, [P, POINTER(c_int64)]),
        "dmr_batch_last_error": (c_char_p, [P]),
        "dmr_noalloc_last_error": (c_char_p, []),
        "dmr_time_launch": (c_int, [P, c_int, c_int, POINTER(c_double), POINTER(c_double)]),
        "dmr_state_bytes": (c_size_t, [P]),
        "dmr_save_state": (c_int, [P, P, c_size_t]),
        "dmr_load_state": (c_int, [P, P, c_size_t]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def make_config(cfg: dict) -> DmrConfig:
    """dmr_config from a plain parameter dict (None selects a default)."""
    def d(key, default=-1.0):
        v = cfg.get(key)
        return float(default if v is None else v)
    c = DmrConfig()
    c.nx, c.ny = int(cfg["nx"]), int(cfg["ny"])
    c.r = int(cfg.get("r") or 1)
    c.n_lambda = int(cfg["n_lambda"])
    c.steps_per_period = int(cfg["steps_per_period"])
    c.precision = int(cfg.get("precision") or 0)
    c.buffer_cells = int(4 if cfg.get("buffer_cells") is None else cfg["buffer_cells"])
    c.growth = int(1 if cfg.get("growth") is None else int(cfg["growth"]))
    c.m_ex = int(-1 if cfg.get("m_ex") is None else cfg["m_ex"])
    c.m_ey = int(-1 if cfg.get("m_ey") is None else cfg["m_ey"])
    c.nu_model = int(cfg.get("nu_model") or 0)
    c.town_A, c.town_B = d("town_A"), d("town_B")
    c.boundary = int(cfg.get("boundary") or 0)
    c.pml_cells = int(cfg.get("pml_cells") or -1)
    c.coupling = int(cfg.get("coupling") or 0)
    c.patch_cap_cells = int(-1 if cfg.get("patch_cap_cells") is None else cfg["patch_cap_cells"])
    c.freq, c.E0, c.p_torr = float(cfg["freq"]), float(cfg["E0"]), float(cfg["p_torr"])
    c.De, c.Da = d("De"), d("Da")
    c.beta_rec, c.Te = d("beta_rec"), d("Te")
    c.nu_scale = d("nu_scale")
    c.nu_a = d("nu_a", 0.0)
    c.n_th, c.g_th = d("n_th"), d("g_th")
    return c


def workspace_bytes(cfg: dict) -> int:
    lib = load()
    c = make_config(cfg)
    n = lib.dmr_workspace_bytes(byref(c))
    if n == 0:
        raise DMRError(EINVAL, lib.dmr_last_error(None).decode())
    return int(n)


class Run:
    """One DMR (or uniform, r = 1) run on a CUDA device."""

    def __init__(self, cfg: dict, device=None, stream=None):
        import torch
        self.lib = lib = load()
        self.cfg = dict(cfg)
        self._c = make_config(cfg)
        nbytes = lib.dmr_workspace_bytes(byref(self._c))
        if nbytes == 0:
            raise DMRError(EINVAL, lib.dmr_last_error(None).decode())
        self.device = torch.device(device if device is not None else "cuda")
        self.ws = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        # a dedicated stream: CUDA graphs cannot be captured on the legacy default stream
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        ctx = c_void_p()
        st = lib.dmr_create(byref(self._c), c_void_p(self.ws.data_ptr()), c_size_t(nbytes),
                            c_void_p(self.stream.cuda_stream), byref(ctx))
        if st != OK:
            raise DMRError(st, lib.dmr_last_error(None).decode())
        self.ctx = ctx
        self.fdtype = np.float32 if self._c.precision == 1 else np.float64
        self.lam = C0 / self._c.freq
        self.dxc = self.lam / self._c.n_lambda

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.dmr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != OK:
            raise DMRError(st, self.lib.dmr_last_error(self.ctx).decode())

    # -- set-up ---------------------------------------------------------------
    def seed_gaussian(self, n0, x0, y0, sx, sy, add=False):
        self._check(self.lib.dmr_seed_gaussian(self.ctx, n0, x0, y0, sx, sy, int(add)))

    def seed_workload(self, seeds):
        """Seeds given as (n0, x0/Lx, y0/Ly, sx/lambda, sy/lambda)."""
        Lx, Ly = self._c.nx * self.dxc, self._c.ny * self.dxc
        for q, (n0, fx, fy, sxl, syl) in enumerate(seeds):
            self.seed_gaussian(n0, fx * Lx, fy * Ly, sxl * self.lam, syl * self.lam, add=q > 0)

    def set_patch(self, rect):
        arr = (c_int32 * 4)(*[int(v) for v in rect])
        self._check(self.lib.dmr_set_patch(self.ctx, arr))

    def get_patch(self):
        arr = (c_int32 * 4)()
        self._check(self.lib.dmr_get_patch(self.ctx, arr))
        return tuple(arr)

    def replay_log(self, rects):
        flat = np.ascontiguousarray(np.asarray(rects, dtype=np.int32).reshape(-1))
        n = flat.size // 4
        ptr = flat.ctypes.data_as(POINTER(c_int32)) if n else None
        self._replay_keep = flat
        self._check(self.lib.dmr_replay_log(self.ctx, ptr, n))

    # -- stepping ---------------------------------------------------------------
    def advance(self, n_coarse_steps):
        self._check(self.lib.dmr_advance(self.ctx, int(n_coarse_steps)))

    def set_graphs(self, on=True):
        self._check(self.lib.dmr_set_graphs(self.ctx, int(bool(on))))

    def set_persistent(self, on=True, rows_coarse=0, rows_fine=0):
        """Each full period's EM steps in one persistent launch (same results)."""
        self._check(self.lib.dmr_set_persistent(self.ctx, int(bool(on)), int(rows_coarse), int(rows_fine)))

    def test_stall(self, on=True, polls=1 << 22):
        """Test of the persistent launch's bounded waits (see dmr.h)."""
        self._check(self.lib.dmr_test_stall(self.ctx, int(bool(on)), int(polls)))

    def set_launch_shape(self, warps_per_sm):
        """Strip height of the EM launches as a warps-per-SM target."""
        self._check(self.lib.dmr_set_launch_shape(self.ctx, int(warps_per_sm)))

    def set_strip_columns(self, columns_per_lane):
        """Node columns per lane of the EM strips (1 or 2; same results)."""
        self._check(self.lib.dmr_set_strip_columns(self.ctx, int(columns_per_lane)))

    def launch_shape(self):
        """(warps per SM of the coarse step's launch, of the later fine
        sub-steps, node columns per lane)."""
        s = (c_int32 * 3)()
        self._check(self.lib.dmr_get_launch_shape(self.ctx, s))
        return tuple(s)

    def set_timing(self, on=True, classes=None):
        """Time every kernel class (on=True), none (on=False) or the named
        classes (``classes``: iterable of class names)."""
        mask = -1 if on else 0
        if on and classes is not None:
            names = [self.lib.dmr_kernel_class_name(k) for k in range(32)]
            names = [n.decode() for n in names if n]
            mask = 0
            for c in classes:
                mask |= 1 << names.index(c)
        self._check(self.lib.dmr_set_timing(self.ctx, mask))

    def kernel_times(self):
        out = {}
        k = 0
        while True:
            name = self.lib.dmr_kernel_class_name(k)
            if not name:
                break
            ms, n, u = c_double(), c_int64(), c_double()
            self._check(self.lib.dmr_kernel_time(self.ctx, k, byref(ms), byref(n), byref(u)))
            out[name.decode()] = (ms.value, n.value, u.value)
            k += 1
        return out

    def launch_count(self):
        n = c_int64()
        self._check(self.lib.dmr_launch_count(self.ctx, byref(n)))
        return n.value

    def autotune(self):
        """Pick the strip height by timed trial launches (at a period boundary)."""
        w = c_int32()
        ms = (c_double * 5)()
        self._check(self.lib.dmr_autotune(self.ctx, byref(w), ms))
        return w.value, list(ms)

    def time_launch(self, form, reps=20):
        """(ms per launch, algorithmic bytes) of an EM launch form of the
        present step: 0 first launch at a period boundary, 1 the same launch
        mid-period (with E^2 samples), 2 the last fine sub-step."""
        ms, b = c_double(), c_double()
        self._check(self.lib.dmr_time_launch(self.ctx, int(form), int(reps), byref(ms), byref(b)))
        return ms.value, b.value

    def sync(self):
        self._check(self.lib.dmr_sync(self.ctx))

    # -- outputs ---------------------------------------------------------------
    def shape(self, field, level=0):
        s = (c_int32 * 2)()
        eb = c_int32()
        self._check(self.lib.dmr_field_shape(self.ctx, FIELDS[field], level, s, byref(eb)))
        return (s[0], s[1]), eb.value

    def _dtype(self, field):
        if field == "S2":
            return np.float64
        if field == "mask":
            return np.uint8
        return self.fdtype

    def read(self, field, level=0):
        """Field as a numpy array of shape (rows, cols) = (y, x)."""
        (rows, cols), eb = self.shape(field, level)
        out = np.empty((rows, cols), dtype=self._dtype(field))
        self._check(self.lib.dmr_read(self.ctx, FIELDS[field], level,
                                      c_void_p(out.ctypes.data), out.nbytes, 0))
        return out

    def read_into(self, field, level, dst_tensor):
        """Queue a device-to-device copy of a field into a torch tensor."""
        self._check(self.lib.dmr_read(self.ctx, FIELDS[field], level,
                                      c_void_p(dst_tensor.data_ptr()),
                                      dst_tensor.numel() * dst_tensor.element_size(), 1))

    def write(self, field, level, arr):
        (rows, cols), eb = self.shape(field, level)
        a = np.ascontiguousarray(np.asarray(arr, dtype=self._dtype(field)))
        if a.shape != (rows, cols):
            raise ValueError("expected shape %r, got %r" % ((rows, cols), a.shape))
        self._check(self.lib.dmr_write(self.ctx, FIELDS[field], level,
                                       c_void_p(a.ctypes.data), a.nbytes, 0))

    def read_to_host(self, field, level, host_tensor):
        """Copy a field into a (pinned) host torch tensor; returns after the copy."""
        self._check(self.lib.dmr_read(self.ctx, FIELDS[field], level,
                                      c_void_p(host_tensor.data_ptr()),
                                      host_tensor.numel() * host_tensor.element_size(), 0))

    def write_from_host(self, field, level, host_tensor):
        """Overwrite a field from a (pinned) host torch tensor."""
        self._check(self.lib.dmr_write(self.ctx, FIELDS[field], level,
                                       c_void_p(host_tensor.data_ptr()),
                                       host_tensor.numel() * host_tensor.element_size(), 0))

    def write_from(self, field, level, src_tensor):
        self._check(self.lib.dmr_write(self.ctx, FIELDS[field], level,
                                       c_void_p(src_tensor.data_ptr()),
                                       src_tensor.numel() * src_tensor.element_size(), 1))

    # -- adjoint ------------------------------------------------------------------
    def adjoint_record(self, n_steps, K):
        """Advance n_steps keeping checkpoints every K steps; returns the
        checkpoint buffer (a device tensor owned by the caller)."""
        import torch
        nb = self.lib.dmr_adjoint_checkpoint_bytes(self.ctx, int(n_steps), int(K))
        ckpt = torch.empty(max(int(nb), 1), dtype=torch.uint8, device=self.device)
        self._check(self.lib.dmr_adjoint_record(self.ctx, int(n_steps), int(K),
                                                c_void_p(ckpt.data_ptr()), c_size_t(nb)))
        return ckpt

    def adjoint_backward(self, dL_dn, ckpt, dseed):
        """dL/dn (device, dense coarse node map) -> (dL/dE0, dL/ds_nu); the
        seed-map gradient is written into the device tensor dseed."""
        import torch
        nb = self.lib.dmr_adjoint_workspace_bytes(self.ctx)
        ws = torch.empty(max(int(nb), 1), dtype=torch.uint8, device=self.device)
        dE0, dnu = c_double(), c_double()
        self._check(self.lib.dmr_adjoint_backward(
            self.ctx, c_void_p(dL_dn.data_ptr()), c_void_p(ws.data_ptr()), c_size_t(nb),
            c_void_p(ckpt.data_ptr()), c_size_t(ckpt.numel()), byref(dE0), byref(dnu),
            c_void_p(dseed.data_ptr()) if dseed is not None else None))
        return dE0.value, dnu.value

    # -- checkpoint / resume ---------------------------------------------------
    def save_state(self, buf=None):
        """Copy the run's state into a device buffer (a uint8 torch tensor,
        allocated here when not given); returns the buffer."""
        import torch
        nb = int(self.lib.dmr_state_bytes(self.ctx))
        if buf is None:
            buf = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self._check(self.lib.dmr_save_state(self.ctx, c_void_p(buf.data_ptr()),
                                            c_size_t(buf.numel())))
        return buf

    def load_state(self, buf):
        """Continue from a state saved by a run of the same configuration."""
        self._check(self.lib.dmr_load_state(self.ctx, c_void_p(buf.data_ptr()),
                                            c_size_t(buf.numel())))

    def stats(self):
        out = (c_double * len(STATS))()
        self._check(self.lib.dmr_stats(self.ctx, out))
        return dict(zip(STATS, list(out)))


class BatchRun(Run):
    """A run owned by a Batch (set-up, reads and stats; advanced by the batch)."""

    def __init__(self, batch, k):
        self.lib = batch.lib
        self.cfg = dict(batch.cfgs[k])
        self._c = make_config(self.cfg)
        self.ctx = c_void_p(self.lib.dmr_batch_run(batch.handle, k))
        self.device = batch.device
        self.stream = batch.stream
        self.fdtype = np.float32 if self._c.precision == 1 else np.float64
        self.lam = C0 / self._c.freq
        self.dxc = self.lam / self._c.n_lambda
        self._batch = batch

    def close(self):
        self.ctx = None


class Batch:
    """Independent runs advanced together (one launch per phase for all runs,
    one CUDA graph per period)."""

    def __init__(self, cfgs, device=None, stream=None):
        import torch
        self.lib = lib = load()
        self.cfgs = [dict(c) for c in cfgs]
        arr = (DmrConfig * len(cfgs))(*[make_config(c) for c in cfgs])
        self._arr = arr
        nbytes = lib.dmr_batch_workspace_bytes(arr, len(cfgs))
        if nbytes == 0:
            raise DMRError(EINVAL, lib.dmr_batch_last_error(None).decode())
        self.device = torch.device(device if device is not None else "cuda")
        self.ws = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        h = c_void_p()
        st = lib.dmr_batch_create(arr, len(cfgs), c_void_p(self.ws.data_ptr()), c_size_t(nbytes),
                                  c_void_p(self.stream.cuda_stream), byref(h))
        if st != OK:
            raise DMRError(st, lib.dmr_batch_last_error(None).decode())
        self.handle = h
        self.runs = [BatchRun(self, k) for k in range(len(cfgs))]

    def _check(self, st):
        if st != OK:
            raise DMRError(st, self.lib.dmr_batch_last_error(self.handle).decode())

    def advance(self, n_coarse_steps):
        self._check(self.lib.dmr_batch_advance(self.handle, int(n_coarse_steps)))

    def set_graphs(self, on=True):
        self._check(self.lib.dmr_batch_set_graphs(self.handle, int(bool(on))))

    def autotune(self):
        w = c_int32()
        ms = (c_double * 5)()
        self._check(self.lib.dmr_batch_autotune(self.handle, byref(w), ms))
        return w.value, list(ms)

    def launch_count(self):
        n = c_int64()
        self._check(self.lib.dmr_batch_launch_count(self.handle, byref(n)))
        return n.value

    def close(self):
        if getattr(self, "handle", None):
            for r in self.runs:
                r.close()
            self.lib.dmr_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_from_workloads(ws, device=None):
    """Batch of runs, each patched and seeded from its workload dict."""
    b = Batch([w["cfg"] for w in ws], device=device)
    for run, w in zip(b.runs, ws):
        if w["cfg"].get("r", 1) > 1 and w.get("rect") is not None:
            run.set_patch(w["rect"])
        run.seed_workload(w["seeds"])
    return b


def run_from_workload(w, device=None, precision=None, cfg_overrides=None, rect=None):
    """Create, patch and seed a run from a workload dict."""
    cfg = dict(w["cfg"])
    if precision is not None:
        cfg["precision"] = precision
    if cfg_overrides:
        cfg.update(cfg_overrides)
    run = Run(cfg, device=device)
    rect = rect if rect is not None else w.get("rect")
    if cfg.get("r", 1) > 1 and rect is not None:
        run.set_patch(rect)
    run.seed_workload(w["seeds"])
    return run
