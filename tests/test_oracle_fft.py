"""Pins of the oracle's transforms against brute force, numpy and exact trigonometry.

The transforms are the building block of the spectral scheme (section 1.1.2: time
stepping in Fourier space, two FFTs per step).  Conventions: forward sign -1,
unnormalised; inverse sign +1 with 1/N^3 in the 3D complex-to-real transform.
"""
import math

import numpy as np
import pytest

from paper_1501_04552_gb300 import inputs as I


def brute_dft(x, sign):
    n = len(x)
    j = np.arange(n)
    t = np.outer(j, j) % n                      # exact integer phase index
    W = np.cos(2 * np.pi * t / n) + 1j * sign * np.sin(2 * np.pi * t / n)
    return W @ x


def brute_dft_matrix(n, sign):
    j = np.arange(n)
    t = np.outer(j, j) % n
    return np.cos(2 * np.pi * t / n) + 1j * sign * np.sin(2 * np.pi * t / n)


@pytest.mark.parametrize("sign", [-1, 1])
def test_dft1d_against_brute_force_all_lengths(oracle, sign):
    rng = np.random.default_rng(7)
    for n in range(1, 65):
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        ref = brute_dft(x, sign)
        got = oracle.dft1d(x, sign)
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
        assert err < 1e-14 * max(4.0, math.log2(n + 1)), (n, err)


@pytest.mark.parametrize("n", [512, 1000, 997, 2310, 4096])
def test_dft1d_against_numpy(oracle, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.linalg.norm(oracle.dft1d(x, -1) - np.fft.fft(x)) / np.linalg.norm(x) < 1e-13
    assert np.linalg.norm(oracle.dft1d(x, 1) - n * np.fft.ifft(x)) / np.linalg.norm(x) < 1e-13


@pytest.mark.parametrize("N", [2, 4, 6, 8])
def test_r2c3d_against_brute_force(oracle, N):
    rng = np.random.default_rng(N)
    u = rng.standard_normal((N, N, N))
    F = brute_dft_matrix(N, -1)
    full = np.einsum("az,by,cx,zyx->abc", F, F, F, u)   # [kz][ky][kx]
    got = oracle.r2c3d(u)
    assert got.shape == (N, N, N // 2 + 1)
    assert np.abs(got - full[:, :, : N // 2 + 1]).max() < 1e-13 * N ** 3


@pytest.mark.parametrize("N", [16, 32])
def test_r2c3d_against_numpy(oracle, N):
    u = np.random.default_rng(3).standard_normal((N, N, N))
    ref = np.fft.rfftn(u)
    assert np.abs(oracle.r2c3d(u) - ref).max() / np.abs(ref).max() < 1e-14


@pytest.mark.parametrize("N", [4, 6])
def test_c2r3d_rule_brute_force(oracle, N):
    """general (non-Hermitian) half spectrum: Re of the inverse of its Hermitian x-extension"""
    rng = np.random.default_rng(11 + N)
    M = N // 2
    h = rng.standard_normal((N, N, M + 1)) + 1j * rng.standard_normal((N, N, M + 1))
    G = brute_dft_matrix(N, +1)
    # inverse along z then y (complex), then the x-line extension X[N-k] = conj(X[k]), 0<k<M
    w = np.einsum("za,yb,abk->zyk", G, G, h)
    full = np.zeros((N, N, N), dtype=complex)
    full[:, :, : M + 1] = w
    for k in range(1, M):
        full[:, :, N - k] = np.conj(w[:, :, k])
    ref = np.real(np.einsum("xk,zyk->zyx", G, full)) / N ** 3
    assert np.abs(oracle.c2r3d(h) - ref).max() < 1e-14 * np.abs(ref).max() * N


@pytest.mark.parametrize("N", [8, 16, 32])
def test_c2r3d_against_numpy_and_roundtrip(oracle, N):
    rng = np.random.default_rng(5)
    u = rng.standard_normal((N, N, N))
    assert np.abs(oracle.c2r3d(oracle.r2c3d(u)) - u).max() < 1e-14 * N
    h = rng.standard_normal((N, N, N // 2 + 1)) + 1j * rng.standard_normal((N, N, N // 2 + 1))
    ref = np.fft.irfftn(h, s=(N, N, N), axes=(0, 1, 2))   # drops Im of the kx = 0 and kx = N/2 entries too
    assert np.abs(oracle.c2r3d(h) - ref).max() / np.abs(ref).max() < 1e-13


def test_axis_pieces_compose_to_3d(oracle):
    N = 16
    u = np.random.default_rng(9).standard_normal((N, N, N))
    a = oracle.r2c_x(u)
    a = oracle.fft_axis(a, 1, -1)
    a = oracle.fft_axis(a, 2, -1)
    assert np.abs(a - oracle.r2c3d(u)).max() < 1e-12
    b = oracle.fft_axis(a, 2, +1)
    b = oracle.fft_axis(b, 1, +1)
    back = oracle.c2r_x(b, 1.0 / N ** 3)
    assert np.abs(back - u).max() < 1e-13


L = 32.0


@pytest.mark.parametrize("m", [(1, 2, 3), (0, 0, 1), (8, 0, 0), (0, -8, 8), (8, 8, 8), (-7, 5, -3)])
def test_spectral_laplacian_exact_on_trig_modes(oracle, m):
    """Laplace cos(k.x) = -k^2 cos(k.x) on the grid, Nyquist m = +-N/2 kept (k^2 = (pi N/L)^2)"""
    N = 16
    u = I.plane_wave(N, L, m, "cos")
    k2 = sum((2 * np.pi * mi / L) ** 2 for mi in m)
    lap = sum(oracle.spectral_deriv(u, L, *o) for o in [(2, 0, 0), (0, 2, 0), (0, 0, 2)])
    assert np.abs(lap + k2 * u).max() < 1e-12 * max(k2, 1.0)


@pytest.mark.parametrize("m", [(1, 0, 0), (3, -2, 5), (0, 7, 0)])
def test_spectral_first_derivative_exact(oracle, m):
    N = 16
    kx = 2 * np.pi * m[0] / L
    ky = 2 * np.pi * m[1] / L
    u = I.plane_wave(N, L, m, "sin")
    assert np.abs(oracle.spectral_deriv(u, L, 1, 0, 0) - kx * I.plane_wave(N, L, m, "cos")).max() < 1e-12
    assert np.abs(oracle.spectral_deriv(u, L, 0, 1, 0) - ky * I.plane_wave(N, L, m, "cos")).max() < 1e-12


def test_odd_derivative_drops_nyquist(oracle):
    N = 16
    u = I.plane_wave(N, L, (8, 0, 0), "cos")     # (-1)^j on the grid: its x-derivative is not representable
    assert np.abs(oracle.spectral_deriv(u, L, 1, 0, 0)).max() < 1e-12
    lap = oracle.spectral_deriv(u, L, 2, 0, 0)
    assert np.abs(lap + (np.pi * N / L) ** 2 * u).max() < 1e-11
