"""Pins of the oracle's time stepping, startup and energy against closed forms,
Eq. (2) itself evaluated with an independent library Laplacian, golden decimal
levels, conservation laws, symmetries and the order of accuracy."""
import math
import os

import numpy as np
import pytest

from paper_1501_04552_gb300 import inputs as I

L = 32.0
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def np_laplacian(u, L):
    """spectral Laplacian by numpy.fft (library), Nyquist kept: the reading used throughout"""
    N = u.shape[0]
    k = 2 * np.pi * np.fft.fftfreq(N, 1.0 / N) / L
    kx = 2 * np.pi * np.fft.rfftfreq(N, 1.0 / N) / L
    k2 = kx[None, None, :] ** 2 + k[None, :, None] ** 2 + k[:, None, None] ** 2
    return np.fft.irfftn(-k2 * np.fft.rfftn(u), s=u.shape, axes=(0, 1, 2))


def test_coefficients_match_discrete_dispersion(oracle):
    """c_k = cos(theta_k), theta_k = 2 arctan(dt omega_k / 2); beta_k = (1 - c_k) / omega_k^2"""
    for dt in [1e-3, 0.005, 0.01, 0.1, 1.0, 7.0]:
        for k2 in [0.0, 0.3, 1.0, 38.5, 2.4e3, 1.9e5]:
            c, b = oracle.coeffs(dt, k2)
            w = math.sqrt(1 + k2)
            assert abs(c - math.cos(2 * math.atan(dt * w / 2))) < 1e-14
            assert abs(b * (1 + k2) - (1 - c)) < 1e-15     # both sides lie in [0, 2]
            assert abs(c) <= 1.0


def single_mode_case(oracle, N, m, dt, steps_list, b=0.0):
    """lam = 0: u0 = cos(k.x), v0 = b sin(k.x)  =>  u^n = cos(n th) cos(k.x) + dt b sin(n th)/sin(th) sin(k.x)"""
    u0 = I.plane_wave(N, L, m, "cos")
    v0 = b * I.plane_wave(N, L, m, "sin")
    k2 = sum((2 * np.pi * mi / L) ** 2 for mi in m)
    th = 2 * math.atan(dt * math.sqrt(1 + k2) / 2)
    s = oracle.Solver(N, L, dt, u0, v0, lam=0.0)
    done = 0
    for n in steps_list:
        s.step(n - done)
        done = n
        ref = math.cos(n * th) * u0 + (dt * b * math.sin(n * th) / math.sin(th)) * I.plane_wave(N, L, m, "sin")
        err = np.abs(s.fetch() - ref).max()
        assert err < 1e-12, (m, n, err)
    s.close()


@pytest.mark.parametrize("m", [(1, 2, 3), (0, 0, 0), (8, -8, 8), (-3, 8, 1)])
def test_linear_single_mode_closed_form(oracle, m):
    single_mode_case(oracle, 16, m, 0.01, [1, 7, 50, 200], b=0.0 if m == (8, -8, 8) else 0.7)


def test_linear_single_mode_large_dt(oracle):
    """the linear part is unconditionally stable: |c_k| <= 1 for any dt"""
    single_mode_case(oracle, 16, (2, 1, 0), 0.9, [1, 3, 40], b=0.3)


def test_constant_field_matches_golden_decimal_levels(oracle):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "constant_field.txt")) if not l.startswith("#")]
    cases = {}
    for r in rows:
        cases.setdefault(int(r[0]), []).append((float(r[1]), float(r[2]), float(r[3]), int(r[4]), float(r[5])))
    for ci, seq in cases.items():
        a0, dt, lam = seq[0][0], seq[0][1], seq[0][2]
        N = 8
        s = oracle.Solver(N, L, dt, np.full((N, N, N), a0), None, lam=lam)
        amax = max(abs(r[4]) for r in seq)
        theta = 2 * math.atan(dt / 2)            # k = 0: omega = 1
        for (_, _, _, n, an) in seq[:: max(1, len(seq) // 7)]:
            s.step(n - s.level)
            u = s.fetch()
            # rounding injected each step is carried by the neutral k = 0 recurrence with
            # weight sin((n-j) theta) / sin(theta) <= min(n, 1/theta)
            tol = 1e-15 * max(n, 1) * min(max(n, 1), 1 / theta) * amax
            assert np.abs(u - an).max() < tol, (ci, n, u.flat[0], an)
            assert np.ptp(u) < 1e-14
        s.close()


def smooth_ic(N, seed=0):
    u0 = I.gaussian(N, L, 0.9, 2.5)
    u0 += 0.2 * I.plane_wave(N, L, (1, 0, 2), "cos") + 0.1 * I.plane_wave(N, L, (0, 3, -1), "sin")
    v0 = 0.3 * I.gaussian(N, L, 1.0, 3.0) * I.plane_wave(N, L, (1, 1, 0), "cos")
    return u0, v0


def test_eq2_residual_in_physical_space(oracle):
    """u^{n-1}, u^n, u^{n+1} from the oracle satisfy Eq. (2) with numpy's spectral Laplacian"""
    N, dt = 16, 0.02
    u0, v0 = smooth_ic(N)
    s = oracle.Solver(N, L, dt, u0, v0)
    s.step(3)
    levels = []
    for _ in range(3):
        levels.append(s.fetch())
        s.step(1)
    um, u, up = levels
    avg = (up + 2 * u + um) / 4
    res = (up - 2 * u + um) / dt ** 2 - np_laplacian(avg, L) + avg - u ** 3
    scale = np.abs(u).max() / dt ** 2
    assert np.abs(res).max() < 1e-12 * scale, np.abs(res).max() / scale
    s.close()


def test_startup_level(oracle):
    """level -1 satisfies (u^1 - u^{-1}) / (2 dt) = v0 and Eq. (2) at n = 0"""
    N, dt = 16, 0.02
    u0, v0 = smooth_ic(N)
    s = oracle.Solver(N, L, dt, u0, v0)
    a, b = s.spectral()
    um1 = oracle.c2r3d(b)
    s.step(1)
    u1 = s.fetch()
    assert np.abs((u1 - um1) / (2 * dt) - v0).max() < 1e-11
    avg = (u1 + 2 * u0 + um1) / 4
    res = (u1 - 2 * u0 + um1) / dt ** 2 - np_laplacian(avg, L) + avg - u0 ** 3
    assert np.abs(res).max() < 1e-12 * np.abs(u0).max() / dt ** 2
    s.close()


@pytest.mark.parametrize("dt", [0.05, 0.01])
def test_linear_quadratic_energy_exactly_conserved(oracle, dt):
    """lam = 0: Q^{n+1/2} is invariant; only rounding moves it, and Q carries |(uh^{n+1}-uh^n)/dt|^2,
    so the rounding floor scales like eps / dt^2"""
    N = 16
    u0, v0 = smooth_ic(N)
    s = oracle.Solver(N, L, dt, u0, v0, lam=0.0)
    E0 = s.energy()
    Q0, P0, _ = s.energy_parts()
    assert P0 == 0.0 and E0 == Q0
    for _ in range(10):
        s.step(100)
        assert abs(s.energy() - E0) < 5e-16 / dt ** 2 * abs(E0)
    s.close()


def test_linear_energy_detects_a_wrong_weight(oracle):
    """the same run with omega^2 |(a+b)/2|^2 replaced by omega^2 |a|^2 is far from invariant,
    so the conservation pin above can tell the exact quadratic form from near misses"""
    N, dt = 16, 0.05
    u0, v0 = smooth_ic(N)
    s = oracle.Solver(N, L, dt, u0, v0, lam=0.0)

    def wrong_Q():
        a, b = s.spectral()
        kx = 2 * np.pi * np.fft.rfftfreq(N, 1.0 / N) / L
        k = 2 * np.pi * np.fft.fftfreq(N, 1.0 / N) / L
        w2 = 1 + kx[None, None, :] ** 2 + k[None, :, None] ** 2 + k[:, None, None] ** 2
        wt = np.full(a.shape, 2.0)
        wt[:, :, 0] = wt[:, :, -1] = 1.0
        h = L / N
        return (h ** 3 / N ** 3) * np.sum(wt * (0.5 * np.abs((a - b) / dt) ** 2 + 0.5 * w2 * np.abs(a) ** 2))

    q0 = wrong_Q()
    s.step(37)
    assert abs(wrong_Q() - q0) > 1e-6 * abs(q0)
    s.close()


@pytest.mark.parametrize("A,s_", [(0.5, 1.0), (2.0, 1.5), (3.0, 2.0)])
def test_gaussian_energy_closed_form(oracle, A, s_):
    """E(0) of A exp(-r^2/s^2), v0 = 0: (pi s^2/2)^{3/2} (A^2/2)(1 + 3/s^2) - (A^4/4)(pi s^2/4)^{3/2}"""
    N = 128
    u0 = I.gaussian(N, L, A, s_)
    ref = (math.pi * s_ ** 2 / 2) ** 1.5 * (A ** 2 / 2) * (1 + 3 / s_ ** 2) - (A ** 4 / 4) * (math.pi * s_ ** 2 / 4) ** 1.5
    got = oracle.energy_initial(u0, L)
    assert abs(got - ref) < 1e-10 * abs(ref) + 1e-12, (got, ref)


def test_discrete_energy_tends_to_continuous_energy(oracle):
    """E^{-1/2} at level 0 differs from E(0) by O(dt^2)"""
    N = 32
    u0 = I.gaussian(N, L, 1.0, 2.0)
    v0 = 0.4 * I.gaussian(N, L, 1.0, 2.5)
    E0 = oracle.energy_initial(u0, L, v0)
    diffs = []
    for dt in [0.04, 0.02, 0.01]:
        s = oracle.Solver(N, L, dt, u0, v0)
        diffs.append(abs(s.energy() - E0))
        s.close()
    assert diffs[0] < 1e-2 * abs(E0)
    for a, b in zip(diffs, diffs[1:]):
        assert 3.5 < a / b < 4.5, diffs


def test_nonlinear_energy_drift_is_second_order(oracle):
    N, T = 16, 1.0
    u0 = I.gaussian(N, L, 1.5, 1.5)
    drifts = []
    for dt in [0.04, 0.02]:
        s = oracle.Solver(N, L, dt, u0)
        e0 = s.energy()
        es = []
        for _ in range(int(round(T / dt))):
            s.step(1)
            es.append(s.energy())
        drifts.append(max(abs(e - e0) for e in es))
        s.close()
    assert drifts[0] < 3e-3 * abs(e0)
    assert 3.0 < drifts[0] / drifts[1] < 5.0, drifts


def test_radial_symmetry_is_preserved(oracle):
    N = 32
    s = oracle.Solver(N, L, 0.05, I.gaussian(N, L, 1.8, 1.2))
    s.step(20)
    u = s.fetch()
    for perm in [(0, 2, 1), (1, 0, 2), (2, 1, 0), (1, 2, 0)]:
        assert np.abs(u - np.transpose(u, perm)).max() < 1e-13
    refl = np.roll(u[::-1, :, :], 1, axis=0)         # j -> N - j (mod N) is x -> -x
    assert np.abs(u - refl).max() < 1e-13
    refl = np.roll(u[:, :, ::-1], 1, axis=2)
    assert np.abs(u - refl).max() < 1e-13


def test_second_order_in_time(oracle):
    N, T = 16, 0.48
    u0 = I.gaussian(N, L, 1.4, 1.5)
    v0 = 0.2 * I.gaussian(N, L, 1.0, 2.0)

    def run(dt):
        s = oracle.Solver(N, L, dt, u0, v0)
        s.step(int(round(T / dt)))
        u = s.fetch()
        s.close()
        return u

    ref = run(0.0025)
    errs = [np.abs(run(dt) - ref).max() for dt in [0.04, 0.02, 0.01]]
    for a, b in zip(errs, errs[1:]):
        assert 3.3 < a / b < 4.7, errs


def test_blowup_flag_freezes_state(oracle):
    N = 32
    s = oracle.Solver(N, L, 0.01, I.gaussian(N, L, 4.0, 1.0))
    blown, lvl = s.step(2000, threshold=1e3)
    assert blown and 0 < lvl < 2000 and s.level == lvl
    assert s.last_maxabs > 1e3
    a, _ = s.spectral()
    blown2, lvl2 = s.step(5, threshold=1e3)      # stays frozen
    assert blown2 and lvl2 == lvl
    assert np.array_equal(a, s.spectral()[0])
    s.close()
    q = oracle.Solver(N, L, 0.01, I.gaussian(N, L, 0.5, 1.0))
    assert q.step(300, threshold=1e3) == (False, -1)
    assert q.level == 300
    q.close()


@pytest.mark.parametrize("m,shell", [((0, 0, 0), 0), ((1, 0, 0), 1), ((0, -1, 1), 2), ((2, 0, 0), 2),
                                     ((2, 2, 0), 3), ((0, 4, 0), 3), ((3, 3, 0), None)])
def test_shell_energies_of_single_modes(oracle, m, shell):
    """cos(k.x) carries (1/2) omega^2 int cos^2 = omega^2 L^3 / 4 (L^3 / 2 for the constant mode
    of amplitude 1, whose 'cosine' is 1) in the shell of its integer wavenumber norm"""
    N = 16
    u = I.plane_wave(N, L, m, "cos")
    k2 = sum((2 * np.pi * mi / L) ** 2 for mi in m)
    ref = (1 + k2) * L ** 3 / (2 if m == (0, 0, 0) else 4)
    got = oracle.shell_energies(u, L)
    for j in range(4):
        want = ref if j == shell else 0.0
        assert abs(got[j] - want) < 1e-12 * ref, (j, got)
