"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Every comparison runs both sides on the same seeded inputs.  Tolerances: relative
L2 <= 1e-12 for the FP64 and double-float passes (the FP64 bar of the 512^3
workload), and a bound derived from FP32 rounding for the mixed passes.  Sizes
span one to several column tiles and always a ragged last tile (N/2 + 1 columns).
"""
import math
import os

import numpy as np
import pytest

from paper_1501_04552_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = 32.0
TOL = {"fp64": 1e-12, "df64": 1e-12, "mixed": 1e-6}
PRECS = ["fp64", "df64", "mixed"]
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def kg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build_library()
    from paper_1501_04552_gb300 import kg as K
    yield K
    K.kg_finalize()
    K.kg_set_options()


@pytest.fixture(scope="module")
def oracle():
    from oracle import oracle as O
    O.lib()
    return O


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def smooth_ic(N, seed=0):
    rng = np.random.default_rng(seed)
    u0 = I.gaussian(N, L, 1.1, 2.2) + 0.08 * I.plane_wave(N, L, (1, -2, 3), "cos")
    u0 += 0.03 * I.plane_wave(N, L, (N // 2, 1, 0), "cos")          # Nyquist content in x
    u0 += 0.02 * I.plane_wave(N, L, (2, N // 2, N // 2), "sin") * rng.uniform(0.5, 1.0)
    v0 = 0.2 * I.gaussian(N, L, 1.0, 3.0) * I.plane_wave(N, L, (0, 1, 1), "cos")
    return u0, v0


def run_gpu(kg, prec, N, dt, u0, v0, steps, lam=1.0, energy_every=0, threshold=0.0):
    kg.kg_set_options(precision=prec, energy_every=energy_every, nonlinearity=lam, blowup_threshold=threshold)
    kg.kg_init(N, L, dt, u0, v0)
    if steps:
        kg.kg_step(steps)
    return kg.kg_fetch(N)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [16, 32, 64, 128])
def test_steps_match_oracle(kg, oracle, prec, N):
    dt, steps = 0.02, 12
    u0, v0 = smooth_ic(N)
    ref = oracle.Solver(N, L, dt, u0, v0)
    ref.step(steps)
    u = run_gpu(kg, prec, N, dt, u0, v0, steps)
    err = rel(u, ref.fetch())
    assert err <= TOL[prec], (prec, N, err)
    a, b = kg.kg_fetch_spectral(N)
    ra, rb = ref.spectral()
    assert rel(a, ra) <= TOL[prec] and rel(b, rb) <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
def test_initial_state_and_startup_level(kg, oracle, prec):
    N, dt = 32, 0.03
    u0, v0 = smooth_ic(N, 1)
    u = run_gpu(kg, prec, N, dt, u0, v0, 0)
    # set-up and read-out transforms run in FP64, except for the double-float passes, which
    # run them in double-float (2^-48 rounding per operation)
    tol = 5e-14 if prec == "df64" else 1e-14
    assert rel(u, u0) <= tol
    a, b = kg.kg_fetch_spectral(N)
    ref = oracle.Solver(N, L, dt, u0, v0)
    ra, rb = ref.spectral()
    assert rel(a, ra) <= tol and rel(b, rb) <= tol


@pytest.mark.parametrize("prec", PRECS)
def test_energy_matches_oracle(kg, oracle, prec):
    N, dt = 32, 0.02
    u0, v0 = smooth_ic(N, 2)
    ref = oracle.Solver(N, L, dt, u0, v0)
    kg.kg_set_options(precision=prec)
    kg.kg_init(N, L, dt, u0, v0)
    tol = 1e-12 if prec != "mixed" else 1e-6
    done = 0
    for lvl in [0, 1, 5, 9]:
        kg.kg_step(lvl - done)
        ref.step(lvl - done)
        done = lvl
        E, Er = kg.kg_energy(), ref.energy()
        assert abs(E - Er) <= tol * abs(Er), (prec, lvl, E, Er)


@pytest.mark.parametrize("prec", PRECS)
def test_recorded_energy_equals_on_demand(kg, prec):
    """energy_every records Q and P inside the step passes; the on-demand path recomputes them"""
    N, dt = 32, 0.02
    u0, v0 = smooth_ic(N, 3)
    out = []
    for every in [0, 4]:
        kg.kg_set_options(precision=prec, energy_every=every)
        kg.kg_init(N, L, dt, u0, v0)
        kg.kg_step(8)
        out.append(kg.kg_energy())
    # mixed: the recorded P^{n-1} comes from the FP32 x pass, the on-demand one from an FP64 inverse
    tol = 1e-13 if prec != "mixed" else 1e-7
    assert abs(out[0] - out[1]) <= tol * abs(out[0])


def test_bump_64_workload(kg, oracle):
    """64^3, u0 = 0.5 exp(-|x|^2), dt = 0.01, 100 steps, energy every step"""
    w = I.bump_64()
    N, dt = w["N"], w["dt"]
    ref = oracle.Solver(N, w["L"], dt, w["u0"])
    e_ref = []
    for _ in range(w["steps"]):
        ref.step(1)
        e_ref.append(ref.energy())
    u_ref = ref.fetch()
    for prec in PRECS:
        kg.kg_set_options(precision=prec, energy_every=1)
        kg.kg_init(N, w["L"], dt, w["u0"], None)
        es = []
        for _ in range(w["steps"]):
            kg.kg_step(1)
            es.append(kg.kg_energy())
        err = rel(kg.kg_fetch(N), u_ref)
        assert err <= (1e-12 if prec != "mixed" else 1e-5), (prec, err)
        de = max(abs(a - b) / abs(b) for a, b in zip(es, e_ref))
        assert de <= (1e-12 if prec != "mixed" else 1e-6), (prec, de)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("m", [(1, 2, 3), (32, 0, 0), (0, -32, 5), (7, 32, 32)])
def test_linear_single_mode_closed_form(kg, prec, m):
    """lam = 0: u^n = cos(n th) cos(k.x) + dt b sin(n th)/sin(th) sin(k.x), th = 2 arctan(dt omega/2)"""
    N, dt, b, n = 64, 0.01, 0.6, 200
    u0 = I.plane_wave(N, L, m, "cos")
    v0 = b * I.plane_wave(N, L, m, "sin")
    k2 = sum((2 * np.pi * mi / L) ** 2 for mi in m)
    th = 2 * math.atan(dt * math.sqrt(1 + k2) / 2)
    u = run_gpu(kg, prec, N, dt, u0, v0, n, lam=0.0)
    ref = math.cos(n * th) * u0 + dt * b * math.sin(n * th) / math.sin(th) * I.plane_wave(N, L, m, "sin")
    assert np.abs(u - ref).max() <= 1e-12, (prec, m)


@pytest.mark.parametrize("prec", PRECS)
def test_constant_field_golden_levels(kg, prec):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "constant_field.txt")) if not l.startswith("#")]
    seq = [(int(r[4]), float(r[5])) for r in rows if r[0] == "1"]    # a0 = 1.2, dt = 0.005, lam = 1
    N, dt, a0 = 16, 0.005, 1.2
    kg.kg_set_options(precision=prec)
    kg.kg_init(N, L, dt, np.full((N, N, N), a0), None)
    theta = 2 * math.atan(dt / 2)
    amax = max(abs(a) for _, a in seq)
    done = 0
    for n, an in seq[::25]:
        kg.kg_step(n - done)
        done = n
        u = kg.kg_fetch(N)
        eps = 1e-15 if prec != "mixed" else 1e-8
        tol = eps * max(n, 1) * min(max(n, 1), 1 / theta) * amax
        if prec == "df64":          # set-up and read-out transforms in double-float
            tol += 1e-14 * amax
        assert np.abs(u - an).max() <= tol, (prec, n, u.flat[0], an)


@pytest.mark.parametrize("prec", PRECS)
def test_radial_symmetry(kg, prec):
    N = 64
    u = run_gpu(kg, prec, N, 0.01, I.gaussian(N, L, 1.5, 1.2), None, 30)
    tol = 1e-13 if prec != "mixed" else 1e-7
    for perm in [(0, 2, 1), (1, 0, 2), (2, 1, 0)]:
        assert np.abs(u - np.transpose(u, perm)).max() <= tol * np.abs(u).max()
    assert np.abs(u - np.roll(u[:, ::-1, :], 1, axis=1)).max() <= tol * np.abs(u).max()


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_blowup_freezes_at_oracle_level(kg, oracle, prec):
    N, dt = 32, 0.01
    u0 = I.gaussian(N, L, 4.0, 1.0)
    ref = oracle.Solver(N, L, dt, u0)
    blown, lvl = ref.step(2000, threshold=1e3)
    assert blown
    kg.kg_set_options(precision=prec, blowup_threshold=1e3)
    kg.kg_init(N, L, dt, u0, None)
    kg.kg_step(lvl + 40)
    st = kg.kg_status()
    assert st["frozen"] and st["blowup_level"] == lvl and st["level"] == lvl
    a, _ = kg.kg_fetch_spectral(N)
    ra, _ = ref.spectral()
    assert rel(a, ra) <= 1e-9           # the field is large and steep near blow-up


def test_device_entry_points_and_streams(kg):
    import torch
    N, dt = 32, 0.02
    u0, v0 = smooth_ic(N, 4)
    kg.kg_set_options(precision="df64")
    kg.kg_init(N, L, dt, u0, v0)
    kg.kg_step(5)
    host = kg.kg_fetch(N)
    d_u0 = torch.from_numpy(u0).cuda()
    d_v0 = torch.from_numpy(v0).cuda()
    s = torch.cuda.Stream()
    kg.kg_set_stream(s)
    kg.kg_init_device(N, L, dt, d_u0, d_v0)
    kg.kg_step(5)
    out = torch.empty((N, N, N), dtype=torch.float64, device="cuda")
    kg.kg_fetch_device(out)
    s.synchronize()
    kg.kg_set_stream(None)
    assert np.array_equal(out.cpu().numpy(), host)


def test_allocation_failure_is_clean(kg, monkeypatch):
    import torch
    N = 64
    u0, v0 = smooth_ic(N, 5)
    kg.kg_finalize()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in [1, 3, 6]:
        monkeypatch.setenv("KG_TEST_FAIL_ALLOC", str(k))
        with pytest.raises(kg.KgError) as ei:
            kg.kg_init(N, L, 0.01, u0, v0)
        assert ei.value.code == kg.KG_ENOMEM
        assert kg.kg_memory() == 0
    monkeypatch.delenv("KG_TEST_FAIL_ALLOC")
    assert abs(torch.cuda.mem_get_info()[0] - free0) < 64 << 20
    kg.kg_set_options(precision="df64")
    kg.kg_init(N, L, 0.01, u0, v0)
    assert kg.kg_memory() > 0


def test_drift_watchdog(kg):
    N, dt = 32, 0.05
    u0 = I.gaussian(N, L, 2.0, 1.5)
    kg.kg_set_options(precision="df64", drift_tol=1e-9)
    kg.kg_init(N, L, dt, u0, None)
    kg.kg_energy()
    kg.kg_step(20)
    with pytest.raises(kg.KgError) as ei:
        kg.kg_energy()
    assert ei.value.code == kg.KG_EDRIFT
    assert math.isfinite(kg.kg_energy(allow_drift=True))
    kg.kg_set_options()


@pytest.mark.parametrize("prec", PRECS)
def test_degenerate_inputs(kg, oracle, prec):
    """the zero field stays exactly zero with zero energy; a start from rest position with
    a velocity only (u0 = 0) follows the oracle; kg_step(0) changes nothing"""
    N, dt = 32, 0.02
    z = np.zeros((N, N, N))
    kg.kg_set_options(precision=prec, energy_every=2)
    kg.kg_init(N, L, dt, z, None)
    kg.kg_step(6)
    assert not np.any(kg.kg_fetch(N)) and kg.kg_energy() == 0.0
    v0 = 0.3 * I.gaussian(N, L, 1.0, 2.5) * I.plane_wave(N, L, (1, 0, 2), "cos")
    kg.kg_init(N, L, dt, z, v0)
    ref = oracle.Solver(N, L, dt, z, v0)
    kg.kg_step(9)
    ref.step(9)
    u = kg.kg_fetch(N)
    assert rel(u, ref.fetch()) <= TOL[prec]
    a0, b0 = kg.kg_fetch_spectral(N)
    kg.kg_step(0)
    a1, b1 = kg.kg_fetch_spectral(N)
    assert np.array_equal(a0, a1) and np.array_equal(b0, b1) and kg.kg_status()["level"] == 9
    kg.kg_set_options()


@pytest.mark.parametrize("prec", PRECS)
def test_max_abs_matches_oracle(kg, oracle, prec):
    """max|u| of the last stepped level, read from integer keys: FP64 bit patterns for the
    FP64 passes, FP32 bit patterns otherwise"""
    N, dt = 32, 0.02
    u0, v0 = smooth_ic(N, 4)
    kg.kg_set_options(precision=prec)
    kg.kg_init(N, L, dt, u0, v0)
    kg.kg_step(7)
    ref = oracle.Solver(N, L, dt, u0, v0)
    ref.step(7)
    tol = {"fp64": 1e-12, "df64": 2.0 ** -23, "mixed": 1e-5}[prec]
    assert abs(kg.kg_status()["maxabs"] - ref.last_maxabs) <= tol * ref.last_maxabs
    kg.kg_set_options()


@pytest.mark.parametrize("prec", PRECS)
def test_linear_mode_large_dt(kg, prec):
    """the linear part is unconditionally stable: dt = 0.9 still follows the discrete dispersion"""
    N, dt, m, b, n = 32, 0.9, (2, -1, 3), 0.3, 40
    u0 = I.plane_wave(N, L, m, "cos")
    v0 = b * I.plane_wave(N, L, m, "sin")
    kg.kg_set_options(precision=prec, nonlinearity=0.0)
    kg.kg_init(N, L, dt, u0, v0)
    kg.kg_step(n)
    k2 = sum((2 * np.pi * mi / L) ** 2 for mi in m)
    th = 2 * math.atan(dt * math.sqrt(1 + k2) / 2)
    ref = math.cos(n * th) * u0 + dt * b * math.sin(n * th) / math.sin(th) * I.plane_wave(N, L, m, "sin")
    assert np.abs(kg.kg_fetch(N) - ref).max() <= (1e-12 if prec != "mixed" else 1e-5)
    kg.kg_set_options()


@pytest.mark.parametrize("prec", PRECS)
def test_timed_steps_match_graph_steps(kg, prec):
    """kg_step_timed launches the same kernels as the graph kg_step replays: the same
    state bit for bit; the z pass is one kernel in the double-float and FP32 passes
    (its update and inverse-z slots read 0) and three in the IEEE FP64 passes"""
    N, dt = 64, 0.01
    u0, v0 = smooth_ic(N, seed=3)
    kg.kg_set_options(precision=prec, energy_every=4)
    kg.kg_init(N, L, dt, u0, v0)
    kg.kg_step(12)
    ref_u, ref_E = kg.kg_fetch(N), kg.kg_energy()
    kg.kg_init(N, L, dt, u0, v0)
    ms = kg.kg_step_timed(12)
    assert kg.kg_status()["level"] == 12
    assert np.array_equal(kg.kg_fetch(N), ref_u) and kg.kg_energy() == ref_E
    fused = prec != "fp64"
    assert all(t > 0 for i, t in enumerate(ms) if not (fused and i in (3, 4)))
    if fused:
        assert ms[3] == 0.0 and ms[4] == 0.0
    kg.kg_set_options()
