"""Batched ensemble (one persistent launch per step): every instance must follow the
single-instance path and the oracle, blow-up flags and levels must match, features
must match the oracle, and a barrier that cannot complete must end in KG_ETIMEOUT."""
import os

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
    K.kg_ens_finalize()
    K.kg_finalize()
    K.kg_set_options()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASE_NS = np.array([64, 128, 64, 128, 64, 128, 64], dtype=np.int32)
CASE_A = np.array([0.7, 1.1, 1.9, 0.6, 2.4, 1.4, 0.9])
CASE_S = np.array([1.3, 0.9, 0.8, 1.7, 1.1, 1.2, 2.0])


@pytest.mark.parametrize("prec", ["df64", "mixed", "fp64"])
def test_instances_follow_single_instance_path(kg, prec):
    dt, steps = 0.005, 37
    kg.kg_set_options(precision=prec)
    kg.kg_ens_init(CASE_NS, L, dt, CASE_A, CASE_S)
    done, ms = kg.kg_ens_run(steps)
    assert done == steps and ms > 0
    res = kg.kg_ens_results()
    assert not res["frozen"].any() and (res["level"] == steps).all()
    ens_u = [kg.kg_ens_fetch(i) for i in range(len(CASE_NS))]
    kg.kg_ens_finalize()
    tol = 1e-13 if prec != "mixed" else 1e-9
    for i, N in enumerate(CASE_NS):
        u0 = I.gaussian(int(N), L, CASE_A[i], CASE_S[i])
        kg.kg_init(int(N), L, dt, u0, None)
        kg.kg_step(steps)
        single = kg.kg_fetch(int(N))
        assert rel(ens_u[i], single) <= tol, (prec, i, rel(ens_u[i], single))
    kg.kg_set_options()


def test_instance_matches_oracle(kg):
    from oracle import oracle as O
    dt, steps = 0.005, 25
    kg.kg_set_options(precision="df64")
    kg.kg_ens_init(CASE_NS[:2], L, dt, CASE_A[:2], CASE_S[:2])
    kg.kg_ens_run(steps)
    for i in range(2):
        N = int(CASE_NS[i])
        ref = O.Solver(N, L, dt, I.gaussian(N, L, CASE_A[i], CASE_S[i]))
        ref.step(steps)
        assert rel(kg.kg_ens_fetch(i), ref.fetch()) <= 1e-12
        ref.close()
    kg.kg_ens_finalize()


def test_blowup_levels_match_oracle_and_freeze(kg):
    from oracle import oracle as O
    dt, thr = 0.005, 1e3
    Ns = np.array([64, 64, 128, 64], dtype=np.int32)
    A = np.array([4.0, 3.6, 4.0, 0.6])
    S = np.array([1.2, 1.5, 1.2, 1.0])
    kg.kg_set_options(precision="df64")
    kg.kg_ens_init(Ns, L, dt, A, S)
    done, _ = kg.kg_ens_run(300, thr)
    res = kg.kg_ens_results()
    kg.kg_ens_finalize()
    for i in range(len(Ns)):
        N = int(Ns[i])
        ref = O.Solver(N, L, dt, I.gaussian(N, L, A[i], S[i]))
        blown, lvl = ref.step(int(done), threshold=thr)
        ref.close()
        assert bool(res["frozen"][i]) == blown, i
        if blown:
            assert res["blowup_level"][i] == lvl and res["level"][i] == lvl, (i, res["blowup_level"][i], lvl)
            assert res["maxabs"][i] > thr
        else:
            assert res["level"][i] == done


def test_features_match_oracle(kg):
    from oracle import oracle as O
    kg.kg_set_options(precision="df64")
    kg.kg_ens_init(CASE_NS[:4], L, 0.005, CASE_A[:4], CASE_S[:4])
    f = kg.kg_ens_features()
    kg.kg_ens_finalize()
    for i in range(4):
        N = int(CASE_NS[i])
        ref = O.shell_energies(I.gaussian(N, L, CASE_A[i], CASE_S[i]), L)
        assert np.allclose(f[i], ref, rtol=1e-12, atol=1e-300), (i, f[i], ref)


def test_tuned_shape_is_kept_and_results_unchanged(kg):
    kg.kg_set_options(precision="df64")
    kg.kg_ens_init(CASE_NS, L, 0.005, CASE_A, CASE_S)
    b, o = kg.kg_ens_tune(2)
    assert b >= 1 and o in (0, 1)
    kg.kg_ens_init(CASE_NS, L, 0.005, CASE_A, CASE_S)
    kg.kg_ens_run(12)
    u = kg.kg_ens_fetch(3)
    kg.kg_ens_finalize()
    N = int(CASE_NS[3])
    kg.kg_init(N, L, 0.005, I.gaussian(N, L, CASE_A[3], CASE_S[3]), None)
    kg.kg_step(12)
    assert rel(u, kg.kg_fetch(N)) <= 1e-13


def test_barrier_timeout_is_reported_not_hung(kg, monkeypatch):
    kg.kg_set_options(precision="df64")
    monkeypatch.setenv("KG_TEST_ENS_MISSING_CTA", "1")
    kg.kg_ens_init(CASE_NS[:2], L, 0.005, CASE_A[:2], CASE_S[:2])
    monkeypatch.delenv("KG_TEST_ENS_MISSING_CTA")
    with pytest.raises(kg.KgError) as ei:
        kg.kg_ens_run(3)
    assert ei.value.code == kg.KG_ETIMEOUT
    # the context survives: a fresh ensemble runs normally
    kg.kg_ens_init(CASE_NS[:2], L, 0.005, CASE_A[:2], CASE_S[:2])
    done, _ = kg.kg_ens_run(5)
    assert done == 5
    kg.kg_ens_finalize()


@pytest.mark.parametrize("prec", ["df64", "mixed"])
def test_every_schedule_computes_the_same_step(kg, prec):
    """the autotuner's schedules against schedule 0: half-width tiles change nothing of the
    arithmetic (bitwise); the short radix stage first changes the rounding of the 128-point
    transforms only (double-float: 1e-13; FP32 passes: 1e-9 of the FP64 state)"""
    dt, steps = 0.005, 23
    kg.kg_set_options(precision=prec)
    fields = {}
    for sched in range(4):
        kg.kg_ens_init(CASE_NS, L, dt, CASE_A, CASE_S)
        kg.kg_ens_set_schedule(sched, 2, 1)
        assert kg.kg_ens_schedule() == (sched, 2, 1)
        kg.kg_ens_run(steps)
        fields[sched] = [kg.kg_ens_fetch(i) for i in range(len(CASE_NS))]
        kg.kg_ens_finalize()
    tol = 1e-13 if prec == "df64" else 1e-9
    for i in range(len(CASE_NS)):
        assert np.array_equal(fields[1][i], fields[0][i]), i
        assert np.array_equal(fields[3][i], fields[2][i]), i
        assert rel(fields[2][i], fields[0][i]) <= tol, (i, rel(fields[2][i], fields[0][i]))
    kg.kg_set_options()


def test_tuned_schedule_is_cached_and_not_slower(kg, tmp_path):
    """kg_ens_tune searches schedule x unit order x CTAs per SM; its choice is written to the
    cache file, read back by a later kg_ens_init, and is at least as fast as the default shape
    (schedule 0, two CTAs per SM, larger grids first) on the same ensemble"""
    Ns, A, s = I.ensemble_params(96, 11)
    cache = str(tmp_path / "ens_tune.txt")
    kg.kg_set_options(precision="df64")
    kg.kg_ens_set_tune_cache(cache)
    kg.kg_ens_init(Ns, L, 0.005, A, s)
    kg.kg_ens_tune(2)
    tuned = kg.kg_ens_schedule()
    kg.kg_ens_finalize()
    lines = [l.split() for l in open(cache)]
    assert len(lines) == 1 and lines[0][0] == "kgens" and [int(x) for x in lines[0][6:9]] == list(tuned)

    def timed(shape):
        kg.kg_ens_init(Ns, L, 0.005, A, s)
        if shape is not None:
            kg.kg_ens_set_schedule(*shape)
        got = kg.kg_ens_schedule()
        kg.kg_ens_run(3)
        best = min(kg.kg_ens_run(20)[1] for _ in range(3))
        kg.kg_ens_finalize()
        return got, best

    got, t_tuned = timed(None)          # a fresh init takes the tuned shape
    assert got == tuned
    _, t_default = timed((0, 2, 1))
    assert t_tuned <= 1.03 * t_default, (tuned, t_tuned, t_default)
    # an entry for another grid mix (written as a later process would find it) is read
    # back by kg_ens_init for that mix
    dev = lines[0][4:6]
    with open(cache, "a") as f:
        f.write("kgens 1 5 3 %s %s 3 1 0 9.0\n" % (dev[0], dev[1]))
    mixNs = np.array([64] * 5 + [128] * 3, dtype=np.int32)
    kg.kg_ens_init(mixNs, L, 0.005, A[:8], s[:8])
    assert kg.kg_ens_schedule() == (3, 1, 0)
    kg.kg_ens_finalize()
    kg.kg_ens_set_tune_cache(None)
    kg.kg_set_options()
