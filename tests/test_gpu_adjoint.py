"""Hand-written adjoint (backward) of the time stepping against the oracle's
complex-step derivatives (exact to rounding) and central finite differences.

Loss L = sum over coarse nodes of (n(t_end) - target)^2; gradients with
respect to E0, the ionization scale s_nu and the seed map (the initial fine
density map, or the coarse one for r = 1); the refinement schedule of the
forward run is held fixed (replayed in the oracle).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import dmr_oracle as O  # noqa: E402
from paper_2105_13276_gb300 import adjoint as A  # noqa: E402
from paper_2105_13276_gb300 import dmr as D  # noqa: E402
from paper_2105_13276_gb300 import workloads as W  # noqa: E402

# FP64 GPU adjoint against the oracle's complex-step derivative (exact to
# rounding): relative error bound of the parity gate
TOL_ADJ64 = 1e-10
# FP32 forward and backward against the same FP64 reference
TOL_ADJ32 = 5e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2105_13276_gb300 import build as B
    B.build()
    D.load()


def case(r):
    if r == 1:
        w = W.small_dmr(nx=40, ny=32, r=1, rect=None)
    else:
        w = W.small_dmr()
    sim = O.sim_from_workload(w)
    seed = (sim.fine if r > 1 else sim.coarse).n.copy()      # oracle layout [i, j]
    return w, seed


def oracle_run(w, E0, nu, seed, steps, log=None, dtype=np.float64):
    cfg = dict(w["cfg"], E0=E0, nu_scale=nu)
    sim = O.Sim(cfg, rect=w["rect"], dtype=dtype)
    if sim.fine is not None:
        sim.seed_map(seed, 0, 0)
    else:
        sim.coarse.n[...] = seed
    if log is not None:
        sim.replay = list(log)
    sim.advance(steps)
    return sim


def cs_grads(w, seed, steps, log, target, u):
    """Complex-step derivatives of L: dL/dE0, dL/ds_nu, dL/dseed . u."""
    E0, nu = w["cfg"]["E0"], 1.0
    out = []
    for which in ("E0", "nu", "seed"):
        h = 1e-20
        e, s, sd = complex(E0), complex(nu), seed.astype(np.complex128)
        if which == "E0":
            e = complex(E0, h * E0)
            scale = h * E0
        elif which == "nu":
            s = complex(nu, h)
            scale = h
        else:
            sd = seed + 1j * h * u
            scale = h
        sim = oracle_run(w, e, s, sd, steps, log, dtype=np.complex128)
        L = np.sum((sim.coarse.n - target) ** 2)
        out.append(L.imag / scale)
    return out


def gpu_grads(w, seed, steps, K, target, precision=0):
    cfg = dict(w["cfg"], precision=precision)
    dt = torch.float64 if precision == 0 else torch.float32
    E0 = torch.tensor(float(w["cfg"]["E0"]), dtype=torch.float64, requires_grad=True)
    nu = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    sm = torch.tensor(seed.T.copy(), dtype=dt, device="cuda", requires_grad=True)
    n_end = A.dmr_density(E0, nu, sm, cfg, w["rect"], steps, K)
    tg = torch.tensor(target.T.copy(), dtype=n_end.dtype, device="cuda")
    L = ((n_end.double() - tg.double()) ** 2).sum()
    L.backward()
    return n_end.detach().cpu().numpy().T, E0.grad.item(), nu.grad.item(), sm.grad.detach().cpu().double().numpy().T


@pytest.mark.parametrize("r", [1, 2])
def test_fp64_adjoint_matches_complex_step(r):
    w, seed = case(r)
    NT = w["cfg"]["steps_per_period"]
    steps, K = 3 * NT, 2 * NT                     # two checkpoint segments
    ref = oracle_run(w, w["cfg"]["E0"], 1.0, seed, steps)
    log = ref.log
    if r > 1:
        assert log[-1] != tuple(w["rect"]), "the rectangle should grow during the run"
    rng = np.random.default_rng(3)
    target = ref.coarse.n * (1 + 0.05 * rng.standard_normal(ref.coarse.n.shape))
    u = rng.standard_normal(seed.shape)
    n_end, gE0, gnu, gseed = gpu_grads(w, seed, steps, K, target)
    assert np.linalg.norm(n_end - ref.coarse.n) / np.linalg.norm(ref.coarse.n) < 1e-12
    cE0, cnu, cseed = cs_grads(w, seed, steps, log, target, u)
    dir_g = float(np.sum(gseed * u))
    errs = (abs(gE0 / cE0 - 1), abs(gnu / cnu - 1), abs(dir_g / cseed - 1))
    print("FP64 adjoint vs complex step, r=%d (E0, s_nu, seed dir):" % r, errs)
    assert max(errs) <= TOL_ADJ64, errs


def test_fp64_adjoint_townsend_matches_complex_step():
    """The adjoint with the Townsend coefficient set (nu_model = 1)."""
    w = W.small_dmr(nu_model=1)
    seed = O.sim_from_workload(w).fine.n.copy()
    NT = w["cfg"]["steps_per_period"]
    steps, K = 2 * NT, NT
    ref = oracle_run(w, w["cfg"]["E0"], 1.0, seed, steps)
    rng = np.random.default_rng(5)
    target = ref.coarse.n * (1 + 0.05 * rng.standard_normal(ref.coarse.n.shape))
    u = rng.standard_normal(seed.shape)
    n_end, gE0, gnu, gseed = gpu_grads(w, seed, steps, K, target)
    assert np.linalg.norm(n_end - ref.coarse.n) / np.linalg.norm(ref.coarse.n) < 1e-12
    cE0, cnu, cseed = cs_grads(w, seed, steps, ref.log, target, u)
    errs = (abs(gE0 / cE0 - 1), abs(gnu / cnu - 1), abs(float(np.sum(gseed * u)) / cseed - 1))
    print("FP64 adjoint vs complex step, Townsend (E0, s_nu, seed dir):", errs)
    assert max(errs) <= TOL_ADJ64, errs


def test_fp64_adjoint_one_way_coupling_matches_complex_step():
    """The adjoint with the density-only transfer back (coupling = 1: no
    fine->coarse E means, so no transposed means either)."""
    w = W.small_dmr(coupling=1)
    seed = O.sim_from_workload(w).fine.n.copy()
    NT = w["cfg"]["steps_per_period"]
    steps, K = 2 * NT, NT
    ref = oracle_run(w, w["cfg"]["E0"], 1.0, seed, steps)
    rng = np.random.default_rng(6)
    target = ref.coarse.n * (1 + 0.05 * rng.standard_normal(ref.coarse.n.shape))
    u = rng.standard_normal(seed.shape)
    n_end, gE0, gnu, gseed = gpu_grads(w, seed, steps, K, target)
    assert np.linalg.norm(n_end - ref.coarse.n) / np.linalg.norm(ref.coarse.n) < 1e-12
    cE0, cnu, cseed = cs_grads(w, seed, steps, ref.log, target, u)
    errs = (abs(gE0 / cE0 - 1), abs(gnu / cnu - 1), abs(float(np.sum(gseed * u)) / cseed - 1))
    print("FP64 adjoint vs complex step, one-way coupling (E0, s_nu, seed dir):", errs)
    assert max(errs) <= TOL_ADJ64, errs


def test_fp64_adjoint_matches_central_differences():
    w, seed = case(2)
    NT = w["cfg"]["steps_per_period"]
    steps = 2 * NT
    ref = oracle_run(w, w["cfg"]["E0"], 1.0, seed, steps)
    target = 0.9 * ref.coarse.n
    _, gE0, gnu, _ = gpu_grads(w, seed, steps, NT, target)

    def L_gpu(E0, nu):
        cfg = dict(w["cfg"], E0=E0, nu_scale=nu)
        run = D.Run(cfg)
        run.set_patch(w["rect"])
        run.write("n", 1, seed.T)
        run.replay_log(ref.log)
        run.advance(steps)
        return float(np.sum((run.read("n").T - target) ** 2))

    E0 = w["cfg"]["E0"]
    h = 1e-6 * E0
    fd = (L_gpu(E0 + h, 1.0) - L_gpu(E0 - h, 1.0)) / (2 * h)
    assert abs(fd / gE0 - 1) < 1e-5, (fd, gE0)
    h = 1e-6
    fd = (L_gpu(E0, 1.0 + h) - L_gpu(E0, 1.0 - h)) / (2 * h)
    assert abs(fd / gnu - 1) < 1e-5, (fd, gnu)


def test_fp32_adjoint_close_to_fp64_reference():
    """FP32 forward and backward against the FP64 complex-step reference:
    the error is printed and bounded at about ten times its measured size."""
    w, seed = case(2)
    NT = w["cfg"]["steps_per_period"]
    steps = 2 * NT
    ref = oracle_run(w, w["cfg"]["E0"], 1.0, seed, steps)
    rng = np.random.default_rng(4)
    target = ref.coarse.n * (1 + 0.05 * rng.standard_normal(ref.coarse.n.shape))
    u = rng.standard_normal(seed.shape)
    _, gE0, gnu, gseed = gpu_grads(w, seed, steps, NT, target, precision=1)
    cE0, cnu, cseed = cs_grads(w, seed, steps, ref.log, target, u)
    errs = (abs(gE0 / cE0 - 1), abs(gnu / cnu - 1), abs(float(np.sum(gseed * u)) / cseed - 1))
    print("FP32 adjoint relative errors (E0, s_nu, seed dir):", errs)
    # measured 1.1e-6, 1.1e-6, 5.6e-6 on a GB300: gated at about ten times that
    assert max(errs) < TOL_ADJ32, errs


def test_fp64_adjoint_at_the_benchmark_geometry_matches_central_differences():
    """The adjoint workload's geometry (coarse 512^2 at lambda/32, r = 2, the
    65 x 65-node seed map, checkpoints every 256 coarse steps) over four
    checkpoint segments in FP64: dL/dE0, dL/ds_nu and the derivative along a
    random seed-map direction against GPU central differences (h = 1e-6
    relative) of the same forward with its refinement schedule replayed."""
    w = W.dmr_512_r2(precision=0)
    cfg = dict(w["cfg"], precision=0)
    NT = cfg["steps_per_period"]
    K, steps = 4 * NT, 16 * NT
    base = D.run_from_workload(w)
    seed = base.read("n", 1)                              # [j, i] layout of the device map
    del base
    pert = W.adjoint_target_map(seed.shape)
    fwd = D.Run(cfg)
    fwd.set_patch(w["rect"])
    fwd.write("n", 1, seed * pert)
    fwd.advance(steps)
    target = fwd.read("n")
    log_run = D.Run(cfg)
    log_run.set_patch(w["rect"])
    log_run.write("n", 1, seed)
    log = []
    for _ in range(steps // NT):
        log_run.advance(NT)
        log.append(log_run.get_patch())
    rng = np.random.default_rng(11)
    u = seed * rng.standard_normal(seed.shape)            # a relative seed-map direction

    E0 = torch.tensor(float(cfg["E0"]), dtype=torch.float64, requires_grad=True)
    nu = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    sm = torch.tensor(seed, dtype=torch.float64, device="cuda", requires_grad=True)
    n_end = A.dmr_density(E0, nu, sm, cfg, w["rect"], steps, K)
    tg = torch.tensor(target, dtype=torch.float64, device="cuda")
    L = ((n_end - tg) ** 2).sum()
    L.backward()
    gE0, gnu = E0.grad.item(), nu.grad.item()
    gdir = float(np.sum(sm.grad.cpu().numpy() * u))

    def loss(E0_, nu_, seed_):
        run = D.Run(dict(cfg, E0=E0_, nu_scale=nu_))
        run.set_patch(w["rect"])
        run.write("n", 1, seed_)
        run.replay_log(log)
        run.advance(steps)
        return float(np.sum((run.read("n") - target) ** 2))

    e0 = cfg["E0"]
    h = 1e-6
    fd = ((loss(e0 * (1 + h), 1.0, seed) - loss(e0 * (1 - h), 1.0, seed)) / (2 * h * e0),
          (loss(e0, 1.0 + h, seed) - loss(e0, 1.0 - h, seed)) / (2 * h),
          (loss(e0, 1.0, seed + h * u) - loss(e0, 1.0, seed - h * u)) / (2 * h))
    errs = (abs(fd[0] / gE0 - 1), abs(fd[1] / gnu - 1), abs(fd[2] / gdir - 1))
    print("FP64 adjoint at 512^2, 16 periods, K = 256 vs central differences "
          "(E0, s_nu, seed dir):", errs)
    assert max(errs) < 1e-5, (errs, fd, (gE0, gnu, gdir))
