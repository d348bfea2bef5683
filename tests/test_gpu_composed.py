"""GPU parity of the fourth-order composed scheme (KG_SCHEME_COMPOSED4) against the
oracle's composed solver (oracle/composed_oracle.py, plain FP64 with numpy's FFT), its
measured order on the GPU, blow-up freezing, checkpoint resume and the calls the scheme
does not define.  Tolerances as for Eq. (2): relative L2 <= 1e-12 for the FP64 and
double-float passes, 1e-6 for the FP32 passes."""
import numpy as np
import pytest

from paper_1501_04552_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = 32.0
TOL = {"fp64": 1e-12, "df64": 1e-12, "mixed": 1e-6}
PRECS = ["fp64", "df64", "mixed"]


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
    K.kg_set_scheme()
    K.kg_set_options()


@pytest.fixture(scope="module")
def CO():
    from oracle import composed_oracle
    return composed_oracle


def ic(N, seed=0):
    rng = np.random.default_rng(seed)
    u0 = I.gaussian(N, L, 1.2, 2.2) + 0.06 * I.plane_wave(N, L, (1, -2, 3), "cos")
    u0 += 0.03 * I.plane_wave(N, L, (N // 2, 1, 0), "cos") + 0.01 * rng.standard_normal((N, N, N))
    v0 = 0.2 * I.gaussian(N, L, 1.0, 3.0) * I.plane_wave(N, L, (0, 1, 1), "cos")
    return u0, v0


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def start(kg, prec, N, dt, u0, v0, threshold=0.0):
    kg.kg_set_scheme("composed4")
    kg.kg_set_options(precision=prec, blowup_threshold=threshold)
    kg.kg_init(N, L, dt, u0, v0)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [16, 32, 64])
def test_composed_matches_oracle(kg, CO, prec, N):
    dt = 0.02
    u0, v0 = ic(N, seed=N)
    start(kg, prec, N, dt, u0, v0)
    s = CO.Composed4Solver(N, L, dt, u0, v0)
    for n in (1, 12):
        kg.kg_step(n - kg.kg_status()["level"])
        s.step(n - s.level)
        assert kg.kg_status()["level"] == n
        assert rel(kg.kg_fetch(N), s.field()) <= TOL[prec], (prec, N, n)
        a, P = kg.kg_fetch_spectral(N)
        assert rel(a, s.a) <= TOL[prec]
        assert rel(P, s.stored_velocity()) <= 10 * TOL[prec]
    kg.kg_finalize()
    kg.kg_set_scheme()


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_order_four_on_the_gpu(kg, CO, prec):
    """the GPU's error at T = 1 against a fine-step oracle solution falls ~16x when dt halves"""
    N, T = 16, 1.0
    u0, v0 = I.gaussian(N, L, 1.4, 2.5), 0.2 * I.gaussian(N, L, 1.0, 3.0)
    fine = CO.Composed4Solver(N, L, T / 256, u0, v0)
    fine.step(256)
    errs = []
    for dt in (0.1, 0.05):
        start(kg, prec, N, dt, u0, v0)
        kg.kg_step(int(round(T / dt)))
        errs.append(rel(kg.kg_fetch(N), fine.field()))
    assert 13.0 < errs[0] / errs[1] < 19.0, errs
    kg.kg_set_scheme()


def test_blowup_freezes_at_oracle_level(kg, CO):
    N, dt = 32, 0.05
    u0 = I.gaussian(N, L, 4.0, 1.8)
    start(kg, "df64", N, dt, u0, None, threshold=50.0)
    kg.kg_step(400)
    st = kg.kg_status()
    s = CO.Composed4Solver(N, L, dt, u0)
    blown, lvl = s.step(400, threshold=50.0)
    assert blown and st["frozen"] and st["blowup_level"] == lvl and st["level"] == lvl
    # the double-float max keys are FP32 bit patterns of the high words
    assert abs(st["maxabs"] - s.last_maxabs) <= 2.0 ** -23 * s.last_maxabs
    u = kg.kg_fetch(N)
    kg.kg_step(3)
    assert np.array_equal(kg.kg_fetch(N), u)
    kg.kg_set_scheme()
    kg.kg_set_options()


def test_checkpoint_resume_bit_identical(kg):
    N = 32
    u0, v0 = ic(N, seed=5)
    start(kg, "df64", N, 0.02, u0, v0)
    kg.kg_step(4)
    ck = kg.kg_save_state()
    assert kg.state_header(ck).scheme == kg.KG_SCHEME_COMPOSED4
    kg.kg_step(5)
    ref = kg.kg_fetch(N)
    kg.kg_finalize()
    kg.kg_set_scheme()
    kg.kg_load_state(ck)
    assert kg.kg_get_scheme() == kg.KG_SCHEME_COMPOSED4
    assert kg.kg_status()["level"] == 4
    kg.kg_step(5)
    assert np.array_equal(kg.kg_fetch(N), ref)
    kg.kg_finalize()
    kg.kg_set_scheme()


def test_timed_steps_match_graph_steps(kg):
    """kg_step_timed runs the same three substeps per step as kg_step"""
    N = 32
    u0, v0 = ic(N, seed=2)
    start(kg, "mixed", N, 0.02, u0, v0)
    kg.kg_step(6)
    ref = kg.kg_fetch(N)
    start(kg, "mixed", N, 0.02, u0, v0)
    ms = kg.kg_step_timed(6)
    assert kg.kg_status()["level"] == 6 and ms[2] > 0.0
    assert np.array_equal(kg.kg_fetch(N), ref)
    kg.kg_finalize()
    kg.kg_set_scheme()


@pytest.mark.parametrize("prec", PRECS)
def test_energy_matches_oracle(kg, CO, prec):
    """kg_energy of the composed scheme: the continuous energy with the synchronised velocity,
    against the oracle's at steps 0, 5 and 15"""
    N, dt = 32, 0.02
    u0, v0 = ic(N, seed=6)
    start(kg, prec, N, dt, u0, v0)
    s = CO.Composed4Solver(N, L, dt, u0, v0)
    for n in (0, 5, 15):
        kg.kg_step(n - kg.kg_status()["level"])
        s.step(n - s.level)
        E, Eo = kg.kg_energy(), s.energy()
        assert abs(E - Eo) <= 10 * TOL[prec] * abs(Eo), (prec, n, E, Eo)
    kg.kg_finalize()
    kg.kg_set_scheme()


def test_eq2_runs_unchanged_after_a_composed_run(kg):
    """switching back to Eq. (2) on a context of the same shape gives the Eq. (2) result"""
    from oracle import oracle as O
    N, dt = 32, 0.02
    u0, v0 = ic(N, seed=8)
    start(kg, "df64", N, dt, u0, v0)
    kg.kg_step(3)
    kg.kg_set_scheme("eq2")
    kg.kg_set_options(precision="df64")
    kg.kg_init(N, L, dt, u0, v0)
    kg.kg_step(10)
    s = O.Solver(N, L, dt, u0, v0)
    s.step(10)
    assert rel(kg.kg_fetch(N), s.fetch()) <= 1e-12
    s.close()
    kg.kg_finalize()


def composed_linear_amplitude(w, dt, n):
    """the exact discrete solution of the composed scheme for one mode of the linear
    equation: (a, p) after n steps from (1, 0), by products of the 2x2 substep maps"""
    import math
    g1 = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
    M = np.eye(2)
    for h in (g1 * dt, (1.0 - 2.0 * g1) * dt, g1 * dt):
        g = -w * w / (1.0 + w * w * h * h / 4.0)     # G_h(a) = g a for F = 0
        kick = np.array([[1.0, 0.0], [0.5 * h * g, 1.0]])
        drift = np.array([[1.0, h], [0.0, 1.0]])
        M = kick @ drift @ kick @ M
    v = np.array([1.0, 0.0])
    for _ in range(n):
        v = M @ v
    assert math.isfinite(v[0])
    return v[0]


@pytest.mark.parametrize("prec", ["df64", "mixed"])
def test_linear_mode_closed_form_512(kg, prec):
    """the benchmark's grid size: lam = 0, u0 = cos(k.x), v0 = 0; after n steps the field is
    a_n cos(k.x) with a_n from the 2x2 substep maps (independent of the oracle)"""
    import math
    N, dt, n, m = 512, 0.01, 20, (5, -7, 3)
    w = math.sqrt(1.0 + sum((2 * math.pi * mi / L) ** 2 for mi in m))
    u0 = I.plane_wave(N, L, m, "cos")
    kg.kg_set_scheme("composed4")
    kg.kg_set_options(precision=prec, nonlinearity=0.0)
    kg.kg_init(N, L, dt, u0, None)
    kg.kg_step(n)
    u = kg.kg_fetch(N)
    err = np.abs(u - composed_linear_amplitude(w, dt, n) * u0).max()
    assert err <= (2e-12 if prec == "df64" else 2e-5), (prec, err)
    kg.kg_finalize()
    kg.kg_set_scheme()
    kg.kg_set_options()


def test_composed_matches_oracle_128(kg, CO):
    N, dt, steps = 128, 0.02, 4
    u0, v0 = ic(N, seed=11)
    start(kg, "df64", N, dt, u0, v0)
    kg.kg_step(steps)
    s = CO.Composed4Solver(N, L, dt, u0, v0)
    s.step(steps)
    assert rel(kg.kg_fetch(N), s.field()) <= 1e-12
    kg.kg_finalize()
    kg.kg_set_scheme()
