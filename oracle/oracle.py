"""ctypes binding of the FP64 CPU oracle (oracle/kg_oracle.c).

TEST INFRASTRUCTURE: only the test suite, the package smoke check and the
CPU-baseline leg of the benchmark import this module.  Conventions (grid,
transform signs, half-spectrum layout [kz][ky][kx], C2R rule, Nyquist, startup
level, discrete energy) are those stated at the top of kg_oracle.c, which follow
Eq. (1), Eq. (2) and the energy functional of section 1.1 of Aseeri et al.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        vp = C.c_void_p
        L.kgo_dft1d.argtypes = [C.c_int, C.c_int, vp, C.c_ssize_t, vp]
        L.kgo_r2c3d.argtypes = [C.c_int, vp, vp]
        L.kgo_c2r3d.argtypes = [C.c_int, vp, vp]
        L.kgo_r2c_x.argtypes = [C.c_int, vp, vp]
        L.kgo_c2r_x.argtypes = [C.c_int, vp, vp, C.c_double]
        L.kgo_fft_axis.argtypes = [C.c_int, vp, C.c_int, C.c_int]
        L.kgo_coeffs.argtypes = [C.c_double, C.c_double, dp, dp]
        L.kgo_spectral_deriv.argtypes = [C.c_int, C.c_double, vp, C.c_int, C.c_int, C.c_int, vp]
        L.kgo_create.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, vp, vp]
        L.kgo_create.restype = vp
        L.kgo_destroy.argtypes = [vp]
        L.kgo_step.argtypes = [vp, C.c_int, C.c_double, C.POINTER(C.c_long)]
        L.kgo_level.argtypes = [vp]
        L.kgo_level.restype = C.c_long
        L.kgo_last_maxabs.argtypes = [vp]
        L.kgo_last_maxabs.restype = C.c_double
        L.kgo_fetch.argtypes = [vp, vp]
        L.kgo_fetch_spectral.argtypes = [vp, vp, vp]
        L.kgo_energy_parts.argtypes = [vp, dp, dp, dp]
        L.kgo_energy.argtypes = [vp, dp]
        L.kgo_energy_initial.argtypes = [C.c_int, C.c_double, C.c_double, vp, vp, dp]
        L.kgo_shell_energies.argtypes = [C.c_int, C.c_double, vp, vp]
        L.kgo_fft3d.argtypes = [C.c_int, vp, C.c_int]
        L.kgoc_create.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, vp, vp]
        L.kgoc_create.restype = vp
        L.kgoc_destroy.argtypes = [vp]
        L.kgoc_step.argtypes = [vp, C.c_int, C.c_double, C.POINTER(C.c_long)]
        L.kgoc_level.argtypes = [vp]
        L.kgoc_level.restype = C.c_long
        L.kgoc_last_maxabs.argtypes = [vp]
        L.kgoc_last_maxabs.restype = C.c_double
        L.kgoc_fetch.argtypes = [vp, vp]
        L.kgoc_fetch_spectral.argtypes = [vp, vp, vp]
        L.kgoc_energy_parts.argtypes = [vp, dp, dp, dp]
        L.kgoc_energy.argtypes = [vp, dp]
        L.kgo_num_threads.restype = C.c_int
        L.kgo_set_num_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with code %d" % (what, rc))


def dft1d(x, sign=-1):
    x = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(x)
    _check(lib().kgo_dft1d(x.size, sign, _p(x), 1, _p(out)), "dft1d")
    return out


def r2c3d(u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    N = u.shape[0]
    out = np.empty((N, N, N // 2 + 1), dtype=np.complex128)
    _check(lib().kgo_r2c3d(N, _p(u), _p(out)), "r2c3d")
    return out


def c2r3d(uh):
    uh = np.ascontiguousarray(uh, dtype=np.complex128)
    N = uh.shape[0]
    out = np.empty((N, N, N), dtype=np.float64)
    _check(lib().kgo_c2r3d(N, _p(uh), _p(out)), "c2r3d")
    return out


def r2c_x(u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    N = u.shape[-1]
    out = np.empty(u.shape[:-1] + (N // 2 + 1,), dtype=np.complex128)
    _check(lib().kgo_r2c_x(N, _p(u), _p(out)), "r2c_x")
    return out


def c2r_x(uh, scale=1.0):
    uh = np.ascontiguousarray(uh, dtype=np.complex128)
    N = uh.shape[0]
    out = np.empty((N, N, N), dtype=np.float64)
    _check(lib().kgo_c2r_x(N, _p(uh), _p(out), scale), "c2r_x")
    return out


def fft_axis(a, axis, sign):
    """complex DFT along axis 1 (y) or 2 (z) of a [kz][ky][kx] array, returns a copy"""
    a = np.array(a, dtype=np.complex128, order="C", copy=True)
    _check(lib().kgo_fft_axis(a.shape[0], _p(a), axis, sign), "fft_axis")
    return a


def coeffs(dt, k2):
    c = C.c_double()
    b = C.c_double()
    lib().kgo_coeffs(dt, k2, C.byref(c), C.byref(b))
    return c.value, b.value


def spectral_deriv(u, L, ox, oy, oz):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty_like(u)
    _check(lib().kgo_spectral_deriv(u.shape[0], L, _p(u), ox, oy, oz, _p(out)), "spectral_deriv")
    return out


def energy_initial(u0, L, v0=None, lam=1.0):
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    v = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float64)
    E = C.c_double()
    _check(lib().kgo_energy_initial(u0.shape[0], L, lam, _p(u0), None if v is None else _p(v), C.byref(E)),
           "energy_initial")
    return E.value


def shell_energies(u0, L):
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    out = np.empty(4, dtype=np.float64)
    _check(lib().kgo_shell_energies(u0.shape[0], L, _p(u0), _p(out)), "shell_energies")
    return out


def num_threads():
    return lib().kgo_num_threads()


def set_num_threads(n):
    lib().kgo_set_num_threads(int(n))


class Solver:
    """FP64 oracle solver: Eq. (2) stepped in Fourier space (state uh^n, uh^{n-1})."""

    def __init__(self, N, L, dt, u0, v0=None, lam=1.0):
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        assert u0.shape == (N, N, N)
        v = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float64)
        self.N, self.L, self.dt, self.lam = N, L, dt, lam
        self._s = lib().kgo_create(N, L, dt, lam, _p(u0), None if v is None else _p(v))
        if not self._s:
            raise RuntimeError("oracle kgo_create failed")

    def close(self):
        if self._s:
            lib().kgo_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n, threshold=0.0):
        """advance n steps; returns (blown_up, blowup_level)"""
        lvl = C.c_long(-1)
        rc = lib().kgo_step(self._s, int(n), float(threshold), C.byref(lvl))
        if rc < 0:
            raise RuntimeError("oracle kgo_step failed with code %d" % rc)
        return rc == 1, lvl.value

    @property
    def level(self):
        return lib().kgo_level(self._s)

    @property
    def last_maxabs(self):
        return lib().kgo_last_maxabs(self._s)

    def fetch(self):
        out = np.empty((self.N,) * 3, dtype=np.float64)
        _check(lib().kgo_fetch(self._s, _p(out)), "fetch")
        return out

    def spectral(self):
        N = self.N
        a = np.empty((N, N, N // 2 + 1), dtype=np.complex128)
        b = np.empty_like(a)
        _check(lib().kgo_fetch_spectral(self._s, _p(a), _p(b)), "fetch_spectral")
        return a, b

    def energy_parts(self):
        Q, Pn, Pm = C.c_double(), C.c_double(), C.c_double()
        _check(lib().kgo_energy_parts(self._s, C.byref(Q), C.byref(Pn), C.byref(Pm)), "energy_parts")
        return Q.value, Pn.value, Pm.value

    def energy(self):
        E = C.c_double()
        _check(lib().kgo_energy(self._s, C.byref(E)), "energy")
        return E.value


def fft3d(a, sign=-1):
    """full complex 3D DFT of an N^3 array (unnormalised), returns a copy"""
    a = np.array(a, dtype=np.complex128, order="C", copy=True)
    _check(lib().kgo_fft3d(a.shape[0], _p(a), sign), "fft3d")
    return a


class ComplexSolver:
    """FP64 oracle for a complex field u (F = lam |u|^2 u): Eq. (2) on the full N^3
    spectrum (the complex-field reading of section 1.1.2); same interface as Solver"""

    def __init__(self, N, L, dt, u0, v0=None, lam=1.0):
        u0 = np.ascontiguousarray(u0, dtype=np.complex128)
        assert u0.shape == (N, N, N)
        v = None if v0 is None else np.ascontiguousarray(v0, dtype=np.complex128)
        self.N, self.L, self.dt, self.lam = N, L, dt, lam
        self._s = lib().kgoc_create(N, L, dt, lam, _p(u0), None if v is None else _p(v))
        if not self._s:
            raise RuntimeError("oracle kgoc_create failed")

    def close(self):
        if self._s:
            lib().kgoc_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n, threshold=0.0):
        lvl = C.c_long(-1)
        rc = lib().kgoc_step(self._s, int(n), float(threshold), C.byref(lvl))
        if rc < 0:
            raise RuntimeError("oracle kgoc_step failed with code %d" % rc)
        return rc == 1, lvl.value

    @property
    def level(self):
        return lib().kgoc_level(self._s)

    @property
    def last_maxabs(self):
        return lib().kgoc_last_maxabs(self._s)

    def fetch(self):
        out = np.empty((self.N,) * 3, dtype=np.complex128)
        _check(lib().kgoc_fetch(self._s, _p(out)), "fetch")
        return out

    def spectral(self):
        N = self.N
        a = np.empty((N, N, N), dtype=np.complex128)
        b = np.empty_like(a)
        _check(lib().kgoc_fetch_spectral(self._s, _p(a), _p(b)), "fetch_spectral")
        return a, b

    def energy_parts(self):
        Q, Pn, Pm = C.c_double(), C.c_double(), C.c_double()
        _check(lib().kgoc_energy_parts(self._s, C.byref(Q), C.byref(Pn), C.byref(Pm)), "energy_parts")
        return Q.value, Pn.value, Pm.value

    def energy(self):
        E = C.c_double()
        _check(lib().kgoc_energy(self._s, C.byref(E)), "energy")
        return E.value
