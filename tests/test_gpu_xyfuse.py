"""xy-plane fusion of the FP32 passes (kg_set_xy_fusion): inverse y, x pass and forward
y of each z-plane in one kernel of thread-block clusters.

The fused kernel runs the same transforms as the separate passes, so the field, the
spectral state and the energies must agree with the separate-pass form to FP32
rounding effects (compiler contraction may differ between the kernels): on the FP64
state they are damped by dt^2 |u|^2 (bound 1e-9); the energy's P = lam (h^3/4) sum u^4
is summed from the FP32 values of u, so E carries FP32 rounding of P (P is below 1e-2
of E here: bound 1e-9 of E).  Against the FP64 oracle the bound is the FP32/FP64
split's 1e-5.  The step sequence of
the fused form (first step of a call without the inverse y transforms, a closing inverse
y pass) is checked by splitting the steps over several kg_step calls, by reading the
energy between calls and by switching the fusion on and off mid-run.
"""
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
    K.kg_set_xy_fusion(False)
    K.kg_finalize()
    K.kg_set_options()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def field(N):
    return (I.gaussian(N, L, 0.9, 2.0) + 0.05 * I.plane_wave(N, L, (1, 2, -3), "cos")
            + 0.03 * I.plane_wave(N, L, (N // 2, 0, 5), "cos"))


def run(kg, N, dt, chunks, fused, energy_every=4):
    """kg_step over the given chunks; energies read after each chunk"""
    kg.kg_set_options(precision="mixed", energy_every=energy_every)
    kg.kg_set_xy_fusion(fused)
    kg.kg_init(N, L, dt, field(N), 0.2 * I.gaussian(N, L, 1.0, 3.0))
    assert kg.kg_get_xy_fusion() == (fused, fused)
    es = []
    for k in chunks:
        kg.kg_step(k)
        es.append(kg.kg_energy())
    u = kg.kg_fetch(N)
    a, b = kg.kg_fetch_spectral(N)
    st = kg.kg_status()
    kg.kg_finalize()
    kg.kg_set_xy_fusion(False)
    return u, a, b, np.array(es), st


@pytest.mark.parametrize("N", [64, 128, 256])
def test_fused_matches_separate_passes(kg, N):
    chunks = [1, 3, 4, 2, 6]
    u0, a0, b0, e0, s0 = run(kg, N, 0.02, chunks, False)
    u1, a1, b1, e1, s1 = run(kg, N, 0.02, chunks, True)
    assert rel(u1, u0) <= 1e-9
    assert rel(a1, a0) <= 1e-9 and rel(b1, b0) <= 1e-9
    assert np.abs(e1 - e0).max() <= 1e-9 * np.abs(e0).max()
    assert s1["level"] == s0["level"] == sum(chunks)
    assert abs(s1["maxabs"] - s0["maxabs"]) <= 1e-6 * s0["maxabs"]   # max |u| of the last x pass


def test_fused_against_oracle(kg):
    from oracle import oracle as O
    N, dt, n = 64, 0.02, 12
    v0 = 0.2 * I.gaussian(N, L, 1.0, 3.0)
    ref = O.Solver(N, L, dt, field(N), v0)
    ref.step(n)
    u_ref, e_ref = ref.fetch(), ref.energy()
    ref.close()
    u, _, _, e, _ = run(kg, N, dt, [5, 7], True, energy_every=0)
    assert rel(u, u_ref) <= 1e-5
    assert abs(e[-1] - e_ref) <= 1e-6 * abs(e_ref)


def test_fused_512_matches_separate_passes(kg):
    """the 512^3 shape (three rounds of column and line transforms per CTA) on the
    benchmark's workload, 20 steps with the energy every 10"""
    N = 512
    w = I.bump_noise(N)
    out = {}
    for fused in (False, True):
        kg.kg_set_options(precision="mixed", energy_every=10)
        kg.kg_set_xy_fusion(fused)
        kg.kg_init(N, L, w["dt"], w["u0"], None)
        es = []
        for _ in range(2):
            kg.kg_step(10)
            es.append(kg.kg_energy())
        out[fused] = (kg.kg_fetch(N), np.array(es))
    kg.kg_finalize()
    kg.kg_set_xy_fusion(False)
    assert rel(out[True][0], out[False][0]) <= 1e-9
    assert np.abs(out[True][1] - out[False][1]).max() <= 1e-9 * abs(out[False][1][0])


def test_toggle_mid_run(kg):
    N, dt = 64, 0.02
    u_ref = run(kg, N, dt, [9], False)[0]
    kg.kg_set_options(precision="mixed", energy_every=0)
    kg.kg_init(N, L, dt, field(N), 0.2 * I.gaussian(N, L, 1.0, 3.0))
    kg.kg_set_xy_fusion(True)
    kg.kg_step(4)
    kg.kg_set_xy_fusion(False)
    kg.kg_step(2)
    kg.kg_set_xy_fusion(True)
    kg.kg_step(3)
    u = kg.kg_fetch(N)
    kg.kg_finalize()
    kg.kg_set_xy_fusion(False)
    assert rel(u, u_ref) <= 1e-9


def test_other_contexts_ignore_it(kg):
    kg.kg_set_xy_fusion(True)
    for prec in ("df64", "fp64"):
        kg.kg_set_options(precision=prec)
        kg.kg_init(32 if prec == "fp64" else 64, L, 0.02, field(32 if prec == "fp64" else 64), None)
        assert kg.kg_get_xy_fusion() == (True, False)
        kg.kg_step(2)
        kg.kg_finalize()
    kg.kg_set_options(precision="mixed")
    kg.kg_init(32, L, 0.02, field(32), None)     # below the fused kernel's smallest grid
    assert kg.kg_get_xy_fusion() == (True, False)
    kg.kg_finalize()
    kg.kg_set_xy_fusion(False)
    kg.kg_set_options()
