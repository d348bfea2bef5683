"""Seeded synthetic inputs for the cubic Klein-Gordon solver.

These generators feed both the CUDA library and the CPU oracle, so they hold none
of the method's arithmetic: they only build initial fields on the grid
x_j = -L/2 + j L/N (physical arrays [z][y][x], x fastest) and draw parameters.

Random numbers come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) mapped to
uniforms on (0, 1] and to normals by the Box-Muller transform.  The low-pass noise
of the 512^3 workload is i.i.d. N(0,1) on the grid, transformed with scipy/numpy's
FFT, truncated to integer wavenumbers |m|_2 <= mmax and transformed back.
"""
import os

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, start, count):
    """outputs start .. start+count-1 of the SplitMix64 stream seeded with `seed`"""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, count, start=0):
    """uniforms on (0, 1] with 53 random bits"""
    z = splitmix64(seed, start, count)
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def normal(seed, count, chunk=1 << 24):
    """count standard normals by Box-Muller on consecutive uniform pairs"""
    out = np.empty(count, dtype=np.float64)
    npairs = (count + 1) // 2
    done = 0
    while done < npairs:
        m = min(chunk, npairs - done)
        u = uniform(seed, 2 * m, start=2 * done)
        r = np.sqrt(-2.0 * np.log(u[0::2]))
        t = 2.0 * np.pi * u[1::2]
        lo = 2 * done
        hi = min(count, lo + 2 * m)
        pair = np.empty(2 * m, dtype=np.float64)
        pair[0::2] = r * np.cos(t)
        pair[1::2] = r * np.sin(t)
        out[lo:hi] = pair[: hi - lo]
        done += m
    return out


def axis(N, L):
    h = L / N
    return -L / 2.0 + h * np.arange(N, dtype=np.float64)


def radius2(N, L):
    x = axis(N, L)
    return x[None, None, :] ** 2 + x[None, :, None] ** 2 + x[:, None, None] ** 2


def gaussian(N, L, A, s):
    """A exp(-|x|^2 / s^2) on the N^3 grid"""
    return A * np.exp(-radius2(N, L) / (s * s))


def plane_wave(N, L, m, phase="cos", amp=1.0):
    """amp cos(k.x) or amp sin(k.x) with k = 2 pi m / L, m = (mx, my, mz) integers"""
    x = axis(N, L)
    kx, ky, kz = (2.0 * np.pi * mi / L for mi in m)
    arg = kx * x[None, None, :] + ky * x[None, :, None] + kz * x[:, None, None]
    return amp * (np.cos(arg) if phase == "cos" else np.sin(arg))


def _rfftn(a):
    try:
        import scipy.fft as sf
        return sf.rfftn(a, workers=os.cpu_count() or 1)
    except ImportError:
        return np.fft.rfftn(a)


def _irfftn(a, shape):
    try:
        import scipy.fft as sf
        return sf.irfftn(a, s=shape, axes=(0, 1, 2), workers=os.cpu_count() or 1)
    except ImportError:
        return np.fft.irfftn(a, s=shape, axes=(0, 1, 2))


def lowpass_noise(N, seed, mmax=8.0):
    """i.i.d. N(0,1) grid noise keeping only integer wavenumbers with |m|_2 <= mmax"""
    g = normal(seed, N * N * N).reshape(N, N, N)
    gh = _rfftn(g)
    del g
    m = np.fft.fftfreq(N, 1.0 / N)
    mx = np.arange(N // 2 + 1, dtype=np.float64)
    m2 = mx[None, None, :] ** 2 + m[None, :, None] ** 2 + m[:, None, None] ** 2
    gh[m2 > mmax * mmax] = 0.0
    return np.ascontiguousarray(_irfftn(gh, (N, N, N)))


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------
L_BOX = 32.0


def bump_64():
    """64^3, u0 = 0.5 exp(-|x|^2), v0 = 0, dt = 0.01, 100 steps, energy every step"""
    N = 64
    return dict(N=N, L=L_BOX, dt=0.01, steps=100, energy_every=1,
                u0=gaussian(N, L_BOX, 0.5, 1.0), v0=None)


def bump_noise(N=512, seed=1501):
    """u0 = 0.1 exp(-|x|^2) + 1e-3 lowpass(N(0,1), |m| <= 8), v0 = 0, dt = 0.005"""
    u0 = gaussian(N, L_BOX, 0.1, 1.0)
    u0 += 1e-3 * lowpass_noise(N, seed, 8.0)
    return dict(N=N, L=L_BOX, dt=0.005, steps=200, energy_every=10, u0=u0, v0=None)


def ensemble_params(count=512, seed=4):
    """(A, s) ~ U[0.5, 4] x U[0.5, 2]; first half 64^3, second half 128^3"""
    u = uniform(seed, 2 * count)
    A = 0.5 + 3.5 * u[0::2]
    s = 0.5 + 1.5 * u[1::2]
    Ns = np.array([64] * (count // 2) + [128] * (count - count // 2), dtype=np.int32)
    return Ns, A, s
