"""512^3 checks in the benchmark's launch configuration.

The oracle finishes a few 512^3 steps in well under a minute, so the first levels
are compared element by element; the 200-step behaviour is checked through
properties that hold at any size: the exact linear single-mode solution, the
constant-field levels, and the energy drift of the scheme."""
import math
import os

import numpy as np
import pytest

from paper_1501_04552_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N = 512
L = 32.0
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
def workload():
    return I.bump_noise(N)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_first_levels_match_oracle(kg, workload):
    from oracle import oracle as O
    w = workload
    ref = O.Solver(N, L, w["dt"], w["u0"], None)
    ref.step(2)
    u_ref = ref.fetch()
    e_ref = ref.energy()
    ref.close()
    for prec, tol, etol in [("df64", 1e-12, 1e-12), ("fp64", 1e-12, 1e-12), ("mixed", 1e-6, 1e-6)]:
        kg.kg_set_options(precision=prec, energy_every=10)
        kg.kg_init(N, L, w["dt"], w["u0"], None)
        kg.kg_step(2)
        err = rel(kg.kg_fetch(N), u_ref)
        assert err <= tol, (prec, err)
        E = kg.kg_energy()
        assert abs(E - e_ref) <= etol * abs(e_ref), (prec, E, e_ref)


@pytest.mark.parametrize("prec", ["df64", "mixed"])
def test_linear_mode_200_steps_exact(kg, prec):
    """lam = 0 on the full grid: the Nyquist-containing mode follows the discrete dispersion exactly"""
    m, dt, b, n = (5, 256, -3), 0.005, 0.4, 200
    u0 = I.plane_wave(N, L, m, "cos")
    v0 = b * I.plane_wave(N, L, m, "sin")
    kg.kg_set_options(precision=prec, nonlinearity=0.0)
    kg.kg_init(N, L, dt, u0, v0)
    kg.kg_step(n)
    u = kg.kg_fetch(N)
    k2 = sum((2 * np.pi * mi / L) ** 2 for mi in m)
    th = 2 * math.atan(dt * math.sqrt(1 + k2) / 2)
    ref = math.cos(n * th) * u0 + dt * b * math.sin(n * th) / math.sin(th) * I.plane_wave(N, L, m, "sin")
    assert np.abs(u - ref).max() <= 1e-12
    kg.kg_set_options()


def test_constant_field_200_steps(kg):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "constant_field.txt")) if not l.startswith("#")]
    seq = {int(r[4]): float(r[5]) for r in rows if r[0] == "1"}      # a0 = 1.2, dt = 0.005
    kg.kg_set_options(precision="df64")
    kg.kg_init(N, L, 0.005, np.full((N, N, N), 1.2), None)
    kg.kg_step(200)
    u = kg.kg_fetch(N)
    theta = 2 * math.atan(0.005 / 2)
    tol = 1e-15 * 200 * min(200, 1 / theta) * 1.2
    assert np.abs(u - seq[200]).max() <= tol
    assert np.ptp(u) <= 1e-13


def test_200_step_energy_and_precision_split(kg, workload):
    """200 steps, energy every 10: the drift stays at the O(dt^2) level of the scheme and the
    FP32-FFT form stays within 1e-5 of the double-float one"""
    w = workload
    res = {}
    for prec in ["df64", "mixed"]:
        kg.kg_set_options(precision=prec, energy_every=10)
        kg.kg_init(N, L, w["dt"], w["u0"], None)
        es = [kg.kg_energy()]
        for _ in range(20):
            kg.kg_step(10)
            es.append(kg.kg_energy())
        res[prec] = (kg.kg_fetch(N), np.array(es))
    e = res["df64"][1]
    assert np.all(np.abs(e - e[0]) <= 1e-6 * abs(e[0])), np.abs(e - e[0]).max() / abs(e[0])
    assert rel(res["mixed"][0], res["df64"][0]) <= 1e-5
    assert np.abs(res["mixed"][1] - e).max() <= 1e-6 * abs(e[0])


def test_double_float_set_up_and_read_out(kg, workload):
    """the double-float set-up and read-out transforms against the IEEE-FP64 ones at 512^3:
    the initial state (uh^0, uh^{-1}) and the fetched field agree to double-float rounding"""
    w = workload
    kg.kg_set_options(precision="fp64")
    kg.kg_init(N, L, w["dt"], w["u0"], None)
    a64, b64 = kg.kg_fetch_spectral(N)
    u64 = kg.kg_fetch(N)
    kg.kg_set_options(precision="df64")
    kg.kg_init(N, L, w["dt"], w["u0"], None)
    a, b = kg.kg_fetch_spectral(N)
    assert rel(a, a64) <= 5e-14 and rel(b, b64) <= 5e-14
    u = kg.kg_fetch(N)
    assert rel(u, u64) <= 5e-14 and rel(u, w["u0"]) <= 5e-14
    kg.kg_finalize()
    kg.kg_set_options()
