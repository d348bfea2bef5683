"""Pins of the composed fourth-order oracle (oracle/composed_oracle.py) against facts that
do not come from the oracle itself: the C oracle's Eq. (2) solver (an independent
implementation with its own FFT), the defining equations of the triple-jump weights, the
order of accuracy measured against a fine-step solution, exact reversibility of a
symmetric method, and the exact solution of the linear equation."""
import math

import numpy as np
import pytest

from oracle import composed_oracle as CO
from paper_1501_04552_gb300 import inputs as I

L = 32.0


def bump(N, amp=1.0, width=2.0):
    return I.gaussian(N, L, amp, width)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_triple_jump_weights():
    g1, g2 = CO.G1, CO.G2
    assert abs(2 * g1 + g2 - 1.0) < 1e-15
    assert abs(2 * g1 ** 3 + g2 ** 3) < 1e-14
    assert g2 < 0 < g1


def test_one_substep_is_eq2_of_the_c_oracle():
    """gammas = (1,) is Eq. (2) with the C oracle's startup level"""
    from oracle import oracle as O
    N, dt, steps = 16, 0.05, 25
    rng = np.random.default_rng(7)
    u0 = bump(N, 1.2) + 0.05 * rng.standard_normal((N, N, N))
    v0 = 0.3 * bump(N, 1.0, 3.0)
    s = CO.Composed4Solver(N, L, dt, u0, v0, gammas=(1.0,))
    c = O.Solver(N, L, dt, u0, v0)
    for n in (1, 7, steps):
        s.step(n - s.level)
        c.step(n - c.level)
        assert rel(s.field(), c.fetch()) < 1e-12, n
        a, b = c.spectral()                 # uh^n, uh^{n-1}
        assert rel(s.a, a) < 1e-12
    c.close()


def _error(gammas, dt, T, ref, N, u0, v0):
    s = CO.Composed4Solver(N, L, dt, u0, v0, gammas=gammas)
    s.step(int(round(T / dt)))
    return rel(s.a, ref)


def test_order_four_and_order_two():
    """error at T = 1 against a fine-step solution: halving dt divides it by ~16 for the
    triple jump and by ~4 for Eq. (2)"""
    N, T = 16, 1.0
    u0, v0 = bump(N, 1.4, 2.5), 0.2 * bump(N, 1.0, 3.0)
    fine = CO.Composed4Solver(N, L, T / 256, u0, v0)
    fine.step(256)
    ref = fine.a
    e4 = [_error(CO.TRIPLE_JUMP, dt, T, ref, N, u0, v0) for dt in (0.1, 0.05)]
    e2 = [_error((1.0,), dt, T, ref, N, u0, v0) for dt in (0.1, 0.05)]
    assert 13.0 < e4[0] / e4[1] < 19.0, e4
    assert 3.5 < e2[0] / e2[1] < 4.5, e2
    assert e4[1] < e2[1] / 50


def test_reversible():
    """a symmetric method run back with -dt returns to its start"""
    N, dt, n = 16, 0.07, 20
    rng = np.random.default_rng(3)
    u0 = bump(N, 1.3) + 0.03 * rng.standard_normal((N, N, N))
    s = CO.Composed4Solver(N, L, dt, u0, 0.1 * bump(N))
    a0, p0 = s.a.copy(), s.p.copy()
    s.step(n)
    assert rel(s.a, a0) > 1e-3
    s.dt = -dt
    s.step(n)
    assert rel(s.a, a0) < 1e-12 and rel(s.p, p0) < 1e-12


@pytest.mark.parametrize("m", [(1, 0, 0), (2, -3, 1)])
def test_linear_mode_fourth_order(m):
    """lam = 0, u0 = cos(k.x), v0 = 0: the exact solution is cos(omega t) cos(k.x); the
    composed error after T = 2 falls by ~16 when dt halves"""
    N, T = 16, 2.0
    u0 = I.plane_wave(N, L, m, "cos")
    k2 = sum((2 * math.pi * mi / L) ** 2 for mi in m)
    w = math.sqrt(1.0 + k2)
    errs = []
    for dt in (0.2, 0.1):
        s = CO.Composed4Solver(N, L, dt, u0, None, lam=0.0)
        s.step(int(round(T / dt)))
        errs.append(np.abs(s.field() - math.cos(w * T) * u0).max())
    assert 13.0 < errs[0] / errs[1] < 19.0, errs


def test_energy_error_is_fourth_order():
    """the continuous energy at t = T differs from its initial value by O(dt^4)"""
    N, T = 16, 1.0
    u0 = bump(N, 1.2, 2.5)
    drifts = []
    for dt in (0.1, 0.05):
        s = CO.Composed4Solver(N, L, dt, u0, None)
        E0 = s.energy()
        s.step(int(round(T / dt)))
        drifts.append(abs(s.energy() - E0) / abs(E0))
    assert drifts[1] < drifts[0] / 10, drifts


def test_blowup_freezes():
    N, dt = 16, 0.05
    s = CO.Composed4Solver(N, L, dt, bump(N, 4.0, 1.8), None)
    blown, lvl = s.step(400, threshold=50.0)
    assert blown and 0 < lvl < 400 and s.level == lvl
    a = s.a.copy()
    s.step(5, threshold=50.0)
    assert np.array_equal(s.a, a)
