"""Checkpoint / resume on the GPU: a run saved at level n and resumed continues bit for
bit as the uninterrupted run (field, Fourier state, energies, blow-up state), in all
three pass precisions, including across kg_finalize and with other options set in
between; a corrupted checkpoint is refused and the running context survives."""
import numpy as np
import pytest

from paper_1501_04552_gb300 import inputs as I

pytestmark = pytest.mark.gpu

L = 32.0


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


def field(N, seed=3):
    rng = np.random.default_rng(seed)
    u0 = I.gaussian(N, L, 1.3, 2.0) + 0.05 * I.plane_wave(N, L, (2, -1, 3), "cos")
    u0 += 0.01 * rng.standard_normal((N, N, N))
    v0 = 0.1 * I.gaussian(N, L, 1.0, 2.5)
    return u0, v0


def tail(kg, N, steps):
    kg.kg_step(steps)
    u = kg.kg_fetch(N)
    a, b = kg.kg_fetch_spectral(N)
    E = kg.kg_energy()
    return u, a, b, E, kg.kg_status()


@pytest.mark.parametrize("prec", ["fp64", "df64", "mixed"])
@pytest.mark.parametrize("N", [32, 64])
def test_resume_is_bit_identical(kg, prec, N):
    u0, v0 = field(N)
    kg.kg_set_options(precision=prec, energy_every=4)
    kg.kg_init(N, L, 0.01, u0, v0)
    kg.kg_step(7)
    ck = kg.kg_save_state()
    h = kg.state_header(ck)
    assert h.level == 7 and h.N == N and h.payload_bytes == 2 * 16 * N * N * (N // 2 + 1)
    ref = tail(kg, N, 9)
    # resume in a fresh process state: other options set, context gone
    kg.kg_finalize()
    kg.kg_set_options(precision="fp64", energy_every=0, nonlinearity=0.0)
    kg.kg_load_state(ck)
    o = kg.kg_get_options()
    assert o["precision"] == {"fp64": 0, "df64": 1, "mixed": 2}[prec]
    assert o["energy_every"] == 4 and o["nonlinearity"] == 1.0
    assert kg.kg_status()["level"] == 7
    got = tail(kg, N, 9)
    for r, g in zip(ref[:3], got[:3]):
        assert np.array_equal(r, g)
    assert got[3] == ref[3]
    assert got[4] == ref[4]


def test_checkpoint_of_initial_level_and_spectral_payload(kg):
    N = 32
    u0, v0 = field(N, seed=5)
    kg.kg_set_options(precision="df64")
    kg.kg_init(N, L, 0.02, u0, v0)
    ck = kg.kg_save_state()
    a, b = kg.kg_fetch_spectral(N)
    n = a.size * 16
    pay = ck[kg.STATE_HEADER_BYTES:]
    assert np.array_equal(pay[:n].view(np.complex128).reshape(a.shape), a)
    assert np.array_equal(pay[n:].view(np.complex128).reshape(b.shape), b)
    assert kg.state_header(ck).checksum == kg.kg_state_checksum(pay)
    ref = tail(kg, N, 5)
    kg.kg_load_state(ck)
    got = tail(kg, N, 5)
    assert np.array_equal(ref[0], got[0]) and got[3] == ref[3]


def test_frozen_state_survives_resume(kg):
    N = 32
    u0 = I.gaussian(N, L, 6.0, 1.5)
    kg.kg_set_options(precision="df64", blowup_threshold=10.0)
    kg.kg_init(N, L, 0.01, u0, None)
    kg.kg_step(400)
    st = kg.kg_status()
    assert st["frozen"] == 1
    ck = kg.kg_save_state()
    u_frozen = kg.kg_fetch(N)
    kg.kg_finalize()
    kg.kg_set_options()
    kg.kg_load_state(ck)
    st2 = kg.kg_status()
    assert st2["frozen"] == 1 and st2["blowup_level"] == st["blowup_level"]
    kg.kg_step(5)
    assert np.array_equal(kg.kg_fetch(N), u_frozen)
    assert kg.kg_get_options()["blowup_threshold"] == 10.0
    kg.kg_set_options()


def test_corrupt_checkpoint_keeps_running_context(kg):
    N = 32
    u0, v0 = field(N, seed=8)
    kg.kg_set_options(precision="mixed")
    kg.kg_init(N, L, 0.01, u0, v0)
    kg.kg_step(3)
    ck = kg.kg_save_state()
    bad = ck.copy()
    bad[-5] ^= 0x40
    with pytest.raises(kg.KgError) as e:
        kg.kg_load_state(bad)
    assert e.value.code == kg.KG_EINVAL
    with pytest.raises(kg.KgError):
        kg.kg_load_state(ck[:-8])
    # the context in place is untouched and still steps
    assert kg.kg_status()["level"] == 3
    kg.kg_step(2)
    assert kg.kg_status()["level"] == 5
    kg.kg_set_options()
