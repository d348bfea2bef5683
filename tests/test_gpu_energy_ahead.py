"""kg_energy on a real field stepped by separate passes runs the next step's x pass ahead of
time (with P^n recorded) instead of a read-only peek pass, and kg_step then skips that x pass.
The trajectory must not depend on when, or whether, the energy is asked for: bitwise the same
field with and without energy evaluations, with kg_step_timed, after a checkpoint taken with
the x pass pending, and with the fused xy form switched on in between; a second kg_energy at
the same level returns the same value; the energies equal the FP64 oracle's."""
import numpy as np
import pytest

from paper_1501_04552_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N, L, DT = 32, 32.0, 0.01


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
    K.kg_set_xy_fusion(0)


def field(n=N):
    rng = np.random.default_rng(1501)
    return I.gaussian(n, L, 1.5, 2.0) + 0.01 * rng.standard_normal((n, n, n))


@pytest.mark.parametrize("prec", ["df64", "fp64", "mixed"])
def test_energy_leaves_the_trajectory_bitwise(kg, prec):
    u0 = field()
    kg.kg_set_options(precision=prec, energy_every=4)
    kg.kg_init(N, L, DT, u0, None)
    kg.kg_step(13)
    u_plain = kg.kg_fetch(N)
    st_plain = kg.kg_status()
    kg.kg_init(N, L, DT, u0, None)
    energies = []
    for _ in range(13):
        kg.kg_step(1)
        e1 = kg.kg_energy()
        assert kg.kg_energy() == e1          # asked again at the same level
        energies.append(e1)
    assert np.array_equal(kg.kg_fetch(N), u_plain)
    assert kg.kg_status() == st_plain        # max |u| of the last step (u^12), not of u^13
    # timed steps and plain steps after an energy evaluation
    kg.kg_step(2)
    kg.kg_energy()
    kg.kg_step_timed(3)
    u_timed = kg.kg_fetch(N)
    kg.kg_init(N, L, DT, u0, None)
    kg.kg_step(18)
    assert np.array_equal(kg.kg_fetch(N), u_timed)
    kg.kg_set_options()


def test_checkpoint_with_the_x_pass_pending(kg):
    u0 = field()
    kg.kg_set_options(precision="df64", energy_every=5)
    kg.kg_init(N, L, DT, u0, None)
    kg.kg_step(7)
    e7 = kg.kg_energy()                      # x pass of step 7 -> 8 now pending
    ck = kg.kg_save_state()
    kg.kg_step(6)
    u_a = kg.kg_fetch(N)
    kg.kg_finalize()
    kg.kg_load_state(ck)
    assert kg.kg_energy() == pytest.approx(e7, rel=1e-14, abs=0.0)
    kg.kg_step(6)
    assert np.array_equal(kg.kg_fetch(N), u_a)
    kg.kg_set_options()


def test_fused_form_switched_on_with_the_x_pass_pending(kg):
    n = 64                                   # the fused form serves N >= 64
    u0 = field(n)
    kg.kg_set_options(precision="mixed", energy_every=0)
    kg.kg_set_xy_fusion(0)
    kg.kg_init(n, L, DT, u0, None)
    kg.kg_step(6)
    u_ref = kg.kg_fetch(n)
    kg.kg_init(n, L, DT, u0, None)
    kg.kg_step(3)
    kg.kg_energy()                           # x pass of step 3 -> 4 pending
    kg.kg_set_xy_fusion(1)
    kg.kg_step(3)
    assert kg.kg_get_xy_fusion()[1]          # the fused form is what ran
    u_fused = kg.kg_fetch(n)
    kg.kg_set_xy_fusion(0)
    rel = np.linalg.norm(u_fused - u_ref) / np.linalg.norm(u_ref)
    assert rel <= 1e-6                       # the fused form rounds its FP32 passes in another order
    kg.kg_set_options()


@pytest.mark.parametrize("prec", ["df64", "fp64"])
def test_energies_match_the_oracle(kg, prec):
    from oracle import oracle as O
    u0 = field()
    kg.kg_set_options(precision=prec, energy_every=0)
    kg.kg_init(N, L, DT, u0, None)
    ahead = []
    for _ in range(6):
        kg.kg_step(2)
        ahead.append(kg.kg_energy())
    kg.kg_finalize()
    ref = O.Solver(N, L, DT, u0, None)
    oracle_e = []
    for _ in range(6):
        ref.step(2)
        oracle_e.append(ref.energy())
    ref.close()
    a, o = np.array(ahead), np.array(oracle_e)
    assert np.max(np.abs(a - o) / np.abs(o)) <= 1e-12
    kg.kg_set_options()
