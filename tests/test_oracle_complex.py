"""Pins of the oracle's complex-field solver (section 1.1.2: the implementation allows a
complex u; Eq. (1) with |u|^2 u; Eq. (2) on the full N^3 spectrum):

- its 3D transform against a brute-force DFT and numpy (library special case);
- the exact discrete solution of a nonlinear plane wave: for u = A e^{i k.x}, |u|^2 = A^2
  is constant, so Eq. (2) reduces to a^{n+1} + a^{n-1} = 2 (c_k + beta_k A^2) a^n, solved
  by a^n = A e^{-i n theta} with cos(theta) = c_k + beta_k A^2 once the startup level is
  a^{-1} = A e^{+i theta}, i.e. v0 = -i A sin(theta)/dt e^{i k.x};
- phase invariance (u -> e^{i phi} u maps solutions to solutions; u^3 would not);
- agreement with the independent real-field solver on real data;
- exact conservation of Q and of the charge Im sum conj(uh^n) uh^{n+1} by the linear scheme."""
import math

import numpy as np
import pytest

from paper_1501_04552_gb300 import inputs as I

L = 32.0


def plane(N, m):
    x = I.axis(N, L)
    kx, ky, kz = (2 * np.pi * mi / L for mi in m)
    ph = kz * x[:, None, None] + ky * x[None, :, None] + kx * x[None, None, :]
    return np.exp(1j * ph)


def smooth_complex(N, seed=0):
    rng = np.random.default_rng(seed)
    u0 = (I.gaussian(N, L, 0.9, 2.4) * np.exp(1j * 0.3 * I.plane_wave(N, L, (1, 0, 0), "cos"))
          + 0.1 * plane(N, (1, -2, 3)) + 0.05j * plane(N, (N // 2, 1, 0)))
    u0 = u0 + 0.01 * (rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N)))
    v0 = 0.2j * I.gaussian(N, L, 1.0, 3.0) + 0.05 * plane(N, (0, 1, -1))
    return u0, v0


def test_fft3d_against_brute_force_and_numpy(oracle):
    rng = np.random.default_rng(1)
    N = 4
    a = rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N))
    j = np.arange(N)
    W = np.exp(-2j * np.pi * np.outer(j, j) / N)
    brute = np.einsum("az,by,cx,zyx->abc", W, W, W, a)
    assert np.abs(oracle.fft3d(a, -1) - brute).max() < 1e-13
    assert np.abs(oracle.fft3d(a, +1) - np.conj(np.einsum("az,by,cx,zyx->abc", W, W, W, np.conj(a)))).max() < 1e-13
    for N in (6, 16, 32):
        a = rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N))
        ref = np.fft.fftn(a)
        assert np.abs(oracle.fft3d(a, -1) - ref).max() < 1e-12 * np.abs(ref).max()
        back = oracle.fft3d(oracle.fft3d(a, -1), +1) / N ** 3
        assert np.abs(back - a).max() < 1e-13


@pytest.mark.parametrize("m,A,lam", [((1, 2, 3), 0.8, 1.0), ((0, 0, 0), 0.6, 1.0), ((8, -8, 5), 0.9, 1.0),
                                     ((-3, 1, 0), 1.1, 0.0), ((2, 0, -1), 0.7, -0.5)])
def test_plane_wave_exact_discrete_solution(oracle, m, A, lam):
    N, dt = 16, 0.02
    k2 = sum((2 * np.pi * mi / L) ** 2 for mi in m)
    c, beta = oracle.coeffs(dt, k2)
    cth = c + beta * lam * A * A
    th = math.acos(cth)
    e = plane(N, m)
    u0 = A * e
    v0 = -1j * A * math.sin(th) / dt * e
    s = oracle.ComplexSolver(N, L, dt, u0, v0, lam=lam)
    done = 0
    for n in (1, 5, 40, 200):
        s.step(n - done)
        done = n
        ref = A * np.exp(-1j * n * th) * e
        err = np.abs(s.fetch() - ref).max()
        assert err < 2e-12 * A, (m, n, err)
    s.close()


def test_plane_wave_pins_the_modulus_form(oracle):
    """the same plane wave with the phase advance of a u^3 nonlinearity is not a solution"""
    N, dt, A, m = 16, 0.02, 0.8, (1, 2, 3)
    k2 = sum((2 * np.pi * mi / L) ** 2 for mi in m)
    c, beta = oracle.coeffs(dt, k2)
    th = math.acos(c + beta * A * A)
    e = plane(N, m)
    s = oracle.ComplexSolver(N, L, dt, A * e, -1j * A * math.sin(th) / dt * e)
    s.step(40)
    u = s.fetch()
    assert np.abs(np.abs(u) - A).max() < 1e-12                     # |u| stays A
    assert np.abs(u - A * np.exp(-1j * 40 * math.acos(c)) * e).max() > 1e-4   # not the linear phase
    s.close()


def test_phase_invariance(oracle):
    N, dt, steps = 16, 0.01, 25
    u0, v0 = smooth_complex(N)
    a = oracle.ComplexSolver(N, L, dt, u0, v0)
    a.step(steps)
    ua = a.fetch()
    phi = np.exp(0.7j)
    b = oracle.ComplexSolver(N, L, dt, phi * u0, phi * v0)
    b.step(steps)
    ub = b.fetch()
    assert np.linalg.norm(ub - phi * ua) / np.linalg.norm(ua) < 1e-13
    Ea, Eb = a.energy(), b.energy()
    assert abs(Ea - Eb) < 1e-13 * abs(Ea)
    a.close(); b.close()


def test_real_data_matches_the_real_field_solver(oracle):
    N, dt, steps = 16, 0.01, 30
    rng = np.random.default_rng(3)
    u0 = I.gaussian(N, L, 1.2, 2.0) + 0.05 * rng.standard_normal((N, N, N))
    v0 = 0.1 * I.gaussian(N, L, 1.0, 3.0)
    r = oracle.Solver(N, L, dt, u0, v0)
    z = oracle.ComplexSolver(N, L, dt, u0.astype(np.complex128), v0.astype(np.complex128))
    for n in (1, steps):
        r.step(n - r.level)
        z.step(n - z.level)
        ur, uz = r.fetch(), z.fetch()
        assert np.abs(uz.imag).max() < 1e-13 * np.abs(ur).max()
        assert np.linalg.norm(uz.real - ur) / np.linalg.norm(ur) < 1e-13
        # spectra: the complex solver's kx = 0..N/2 slab is the real solver's half spectrum
        ar, _ = r.spectral()
        az, _ = z.spectral()
        assert np.abs(az[:, :, : N // 2 + 1] - ar).max() < 1e-12 * np.abs(ar).max()
        Qr, Pr, Pmr = r.energy_parts()
        Qz, Pz, Pmz = z.energy_parts()
        assert abs(Qz - Qr) < 1e-13 * abs(Qr)
        assert abs(Pz - Pr) < 1e-13 * abs(Pr) and abs(Pmz - Pmr) < 1e-13 * abs(Pmr)
    r.close(); z.close()


@pytest.mark.parametrize("dt", [0.01, 0.3])
def test_linear_invariants_exactly_conserved(oracle, dt):
    """lam = 0: Q^{n+1/2} and the charge Im sum conj(uh^n) uh^{n+1} are exact invariants
    of the scheme (real coefficients; multiply Eq. (2) by the conjugate levels).  Only
    rounding moves them; Q carries |(uh^{n+1}-uh^n)/dt|^2, so its floor scales like
    eps / dt^2, as for the real field"""
    N = 16
    u0, v0 = smooth_complex(N, seed=5)
    s = oracle.ComplexSolver(N, L, dt, u0, v0, lam=0.0)
    Q0 = s.energy_parts()[0]
    a, b = s.spectral()
    q0 = np.sum(np.conj(b) * a).imag
    for _ in range(4):
        s.step(50)
        Q = s.energy_parts()[0]
        a, b = s.spectral()
        q = np.sum(np.conj(b) * a).imag
        assert abs(Q - Q0) < 5e-16 / dt ** 2 * abs(Q0)
        assert abs(q - q0) < 1e-12 * abs(q0)
    assert abs(q0) > 1e-3 * np.sum(np.abs(a) ** 2) * dt      # a non-trivial charge
    s.close()


def test_nonlinear_energy_drift_is_second_order(oracle):
    N, T = 16, 1.0
    u0, v0 = smooth_complex(N, seed=7)
    drifts = []
    for dt in (0.02, 0.01):
        s = oracle.ComplexSolver(N, L, dt, u0, v0)
        s.step(1)
        E0 = s.energy()
        s.step(int(round(T / dt)) - 1)
        drifts.append(abs(s.energy() - E0))
        s.close()
    ratio = drifts[0] / drifts[1]
    assert 3.0 < ratio < 5.5, drifts
