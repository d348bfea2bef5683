"""The object interface (paper_1501_04552_gb300.solver) against the plain binding: the same
results bit for bit, host and device inputs and outputs, the complex field, checkpoints."""
import numpy as np
import pytest

from paper_1501_04552_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = 32.0


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build_library()
    from paper_1501_04552_gb300 import kg as K
    from paper_1501_04552_gb300 import solver as S
    yield torch, K, S
    K.kg_finalize()
    K.kg_set_options()


def test_solver_matches_the_binding(mods):
    torch, kg, S = mods
    N, dt = 32, 0.01
    u0 = I.gaussian(N, L, 1.2, 2.0) + 0.05 * I.plane_wave(N, L, (1, 2, -1), "cos")
    kg.kg_set_options(precision="df64", energy_every=5)
    kg.kg_init(N, L, dt, u0, None)
    kg.kg_step(15)
    ref_u, ref_E = kg.kg_fetch(N), kg.kg_energy()
    with S.Solver(u0, L, dt, precision="df64", energy_every=5) as s:
        s.step(10).step(5)
        assert s.level == 15
        assert np.array_equal(s.field(), ref_u) and s.energy() == ref_E
        d = s.field(device=True)
        assert d.is_cuda and d.dtype == torch.float64
        assert np.array_equal(d.cpu().numpy(), ref_u)
    assert kg.kg_memory() == 0          # closed


def test_device_inputs_and_complex_field(mods):
    torch, kg, S = mods
    N, dt = 32, 0.01
    u0 = I.gaussian(N, L, 1.0, 2.2) * np.exp(0.4j * I.plane_wave(N, L, (1, 0, 0), "cos"))
    with S.Solver(u0, L, dt, precision="mixed") as a:
        a.step(8)
        ua = a.field()
    with S.Solver(torch.from_numpy(u0).cuda(), L, dt, precision="mixed") as b:
        assert b.complex
        b.step(8)
        ub = b.field(device=True)
        assert ub.dtype == torch.complex128
    assert np.array_equal(ua, ub.cpu().numpy())


def test_save_and_load(mods):
    torch, kg, S = mods
    N, dt = 32, 0.01
    u0 = I.gaussian(N, L, 1.3, 1.8)
    s = S.Solver(u0, L, dt, precision="df64", energy_every=2)
    s.step(4)
    ck = s.save()
    s.step(6)
    ref = s.field()
    s.close()
    r = S.Solver.load(ck)
    assert r.N == N and r.level == 4 and not r.complex
    r.step(6)
    assert np.array_equal(r.field(), ref)
    r.close()
    kg.kg_set_options()


def test_composed_scheme_through_the_object_interface(mods):
    torch, kg, S = mods
    N, dt = 32, 0.02
    u0 = I.gaussian(N, L, 1.1, 2.0)
    kg.kg_set_scheme("composed4")
    kg.kg_set_options(precision="df64")
    kg.kg_init(N, L, dt, u0, None)
    kg.kg_step(7)
    ref = kg.kg_fetch(N)
    with S.Solver(u0, L, dt, precision="df64", scheme="composed4") as s:
        s.step(7)
        assert s.level == 7 and np.array_equal(s.field(), ref)
    kg.kg_set_scheme()
    kg.kg_set_options()
