"""GPU parity of the complex-field path (|u|^2 u on the full N^3 spectrum) against the
oracle's complex solver, the exact discrete plane-wave solution on the GPU itself, real
data through the complex path against the real path, energies, checkpoint resume and the
blow-up freeze.  Tolerances as for the real field: relative L2 <= 1e-12 for the FP64 and
double-float passes, 1e-6 for the FP32 passes."""
import math

import numpy as np
import pytest

from paper_1501_04552_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = 32.0
TOL = {"fp64": 1e-12, "df64": 1e-12, "mixed": 1e-6}
# max|u| comes from integer keys: FP64 bit patterns for the FP64 passes, FP32 bit patterns
# of |u|^2 (the high word for double-float) otherwise, so it is exact to that resolution
KEY_TOL = {"fp64": 1e-12, "df64": 2.0 ** -23, "mixed": 1e-5}
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
    K.kg_set_options()


@pytest.fixture(scope="module")
def oracle():
    from oracle import oracle as O
    O.lib()
    return O


def plane(N, m):
    x = I.axis(N, L)
    kx, ky, kz = (2 * np.pi * mi / L for mi in m)
    return np.exp(1j * (kz * x[:, None, None] + ky * x[None, :, None] + kx * x[None, None, :]))


def complex_ic(N, seed=0):
    rng = np.random.default_rng(seed)
    u0 = (I.gaussian(N, L, 1.0, 2.3) * np.exp(1j * 0.4 * I.plane_wave(N, L, (1, 0, 0), "cos"))
          + 0.1 * plane(N, (1, -2, 3)) + 0.04j * plane(N, (N // 2, 1, -1)))
    u0 = u0 + 0.01 * (rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N)))
    v0 = 0.2j * I.gaussian(N, L, 1.0, 3.0) + 0.05 * plane(N, (0, 1, -1))
    return u0, v0


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [16, 32, 64])
def test_complex_parity_with_oracle(kg, oracle, prec, N):
    dt, steps = 0.01, 24
    u0, v0 = complex_ic(N, seed=N)
    kg.kg_set_options(precision=prec, energy_every=4)
    kg.kg_init_complex(N, L, dt, u0, v0)
    s = oracle.ComplexSolver(N, L, dt, u0, v0)
    for n in (1, steps):
        kg.kg_step(n - kg.kg_status()["level"])
        s.step(n - s.level)
        u = kg.kg_fetch_complex(N)
        ref = s.fetch()
        assert rel(u, ref) <= TOL[prec], (prec, N, n, rel(u, ref))
        a, b = kg.kg_fetch_spectral(N)
        ra, rb = s.spectral()
        assert rel(a, ra) <= TOL[prec] and rel(b, rb) <= TOL[prec]
        E = kg.kg_energy(allow_drift=True)
        Eo = s.energy()
        assert abs(E - Eo) <= max(TOL[prec], 1e-12) * 10 * abs(Eo), (prec, N, E, Eo)
        st = kg.kg_status()
        assert st["level"] == n
        assert abs(st["maxabs"] - s.last_maxabs) <= KEY_TOL[prec] * s.last_maxabs
    s.close()
    kg.kg_set_options()


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_complex_parity_128(kg, oracle, prec):
    N, dt, steps = 128, 0.01, 6
    u0, v0 = complex_ic(N, seed=11)
    kg.kg_set_options(precision=prec)
    kg.kg_init_complex(N, L, dt, u0, v0)
    kg.kg_step(steps)
    s = oracle.ComplexSolver(N, L, dt, u0, v0)
    s.step(steps)
    assert rel(kg.kg_fetch_complex(N), s.fetch()) <= TOL[prec]
    s.close()
    kg.kg_set_options()


@pytest.mark.parametrize("prec", PRECS)
def test_plane_wave_closed_form_on_gpu(kg, prec):
    """u = A e^{i k.x}: the discrete solution is A e^{-i n theta} e^{i k.x} exactly, with
    cos(theta) = c_k + beta_k A^2 (independent of the oracle)"""
    N, dt, A, m = 32, 0.02, 0.8, (3, -1, 2)
    k2 = sum((2 * np.pi * mi / L) ** 2 for mi in m)
    a = dt * dt * (1 + k2) / 4
    c, beta = (1 - a) / (1 + a), (dt * dt / 2) / (1 + a)
    th = math.acos(c + beta * A * A)
    e = plane(N, m)
    kg.kg_set_options(precision=prec)
    kg.kg_init_complex(N, L, dt, A * e, -1j * A * math.sin(th) / dt * e)
    for n in (1, 50, 200):
        kg.kg_step(n - kg.kg_status()["level"])
        u = kg.kg_fetch_complex(N)
        ref = A * np.exp(-1j * n * th) * e
        tol = 2e-12 if prec != "mixed" else 2e-5
        assert np.abs(u - ref).max() <= tol * A, (prec, n, np.abs(u - ref).max())
    kg.kg_set_options()


@pytest.mark.parametrize("prec", PRECS)
def test_real_data_through_the_complex_path(kg, prec):
    N, dt, steps = 32, 0.01, 20
    rng = np.random.default_rng(4)
    u0 = I.gaussian(N, L, 1.1, 2.0) + 0.03 * rng.standard_normal((N, N, N))
    kg.kg_set_options(precision=prec, energy_every=5)
    kg.kg_init(N, L, dt, u0, None)
    kg.kg_step(steps)
    ur = kg.kg_fetch(N)
    Er = kg.kg_energy(allow_drift=True)
    kg.kg_init_complex(N, L, dt, u0.astype(np.complex128), None)
    kg.kg_step(steps)
    uz = kg.kg_fetch_complex(N)
    Ez = kg.kg_energy(allow_drift=True)
    assert np.abs(uz.imag).max() <= 10 * TOL[prec] * np.abs(ur).max()
    assert rel(uz.real, ur) <= 10 * TOL[prec]
    assert abs(Ez - Er) <= 10 * TOL[prec] * abs(Er)
    kg.kg_set_options()


def test_complex_checkpoint_resume_bit_identical(kg):
    N = 32
    u0, v0 = complex_ic(N, seed=9)
    kg.kg_set_options(precision="df64", energy_every=3)
    kg.kg_init_complex(N, L, 0.01, u0, v0)
    kg.kg_step(5)
    ck = kg.kg_save_state()
    h = kg.state_header(ck)
    assert h.complex_field == 1 and h.payload_bytes == 2 * 16 * N ** 3
    kg.kg_step(7)
    ref = kg.kg_fetch_complex(N), kg.kg_energy()
    kg.kg_finalize()
    kg.kg_set_options()
    kg.kg_load_state(ck)
    kg.kg_step(7)
    got = kg.kg_fetch_complex(N), kg.kg_energy()
    assert np.array_equal(ref[0], got[0]) and ref[1] == got[1]
    kg.kg_set_options()


def test_complex_blowup_freezes(kg, oracle):
    N, dt = 32, 0.01
    u0 = I.gaussian(N, L, 5.0, 1.6) * np.exp(1j * 0.5 * I.plane_wave(N, L, (1, 1, 0), "cos"))
    kg.kg_set_options(precision="df64", blowup_threshold=20.0)
    kg.kg_init_complex(N, L, dt, u0, None)
    kg.kg_step(300)
    st = kg.kg_status()
    s = oracle.ComplexSolver(N, L, dt, u0)
    blown, lvl = s.step(300, threshold=20.0)
    assert blown and st["frozen"] and st["blowup_level"] == lvl
    u = kg.kg_fetch_complex(N)
    kg.kg_step(3)
    assert np.array_equal(kg.kg_fetch_complex(N), u)
    s.close()
    kg.kg_set_options()


def test_wrong_kind_calls_are_refused(kg):
    N = 16
    kg.kg_init_complex(N, L, 0.01, np.ones((N, N, N), dtype=np.complex128) * 0.1, None)
    out = np.empty((N, N, N))
    assert kg.lib.kg_fetch(out.ctypes.data) == kg.KG_ESTATE
    kg.kg_init(N, L, 0.01, np.ones((N, N, N)) * 0.1, None)
    outc = np.empty((N, N, N), dtype=np.complex128)
    assert kg.lib.kg_fetch_complex(outc.ctypes.data) == kg.KG_ESTATE
    bad = np.ones((N, N, N), dtype=np.complex128)
    bad[1, 2, 3] = complex(0, np.nan)
    assert kg.lib.kg_init_complex(N, L, 0.01, bad.ctypes.data, None) == kg.KG_EINVAL
    kg.kg_finalize()


@pytest.mark.parametrize("prec", ["df64", "mixed"])
def test_plane_wave_closed_form_512(kg, prec):
    """the benchmark's grid size: the exact discrete plane wave after 60 steps"""
    N, dt, A, m = 512, 0.005, 0.9, (5, -7, 3)
    k2 = sum((2 * np.pi * mi / L) ** 2 for mi in m)
    a = dt * dt * (1 + k2) / 4
    c, beta = (1 - a) / (1 + a), (dt * dt / 2) / (1 + a)
    th = math.acos(c + beta * A * A)
    e = plane(N, m)
    kg.kg_set_options(precision=prec)
    kg.kg_init_complex(N, L, dt, A * e, -1j * A * math.sin(th) / dt * e)
    kg.kg_step(60)
    u = kg.kg_fetch_complex(N)
    err = np.abs(u - A * np.exp(-60j * th) * e).max()
    assert err <= (2e-12 if prec == "df64" else 2e-5) * A, (prec, err)
    kg.kg_finalize()
    kg.kg_set_options()
