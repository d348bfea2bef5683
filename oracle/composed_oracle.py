"""Plain FP64 CPU oracle of the fourth-order composed time stepping.

TEST INFRASTRUCTURE: only the test suite, the package smoke check and the benchmark's
CPU legs import this module; the CUDA library never does.

Section 3 of Aseeri et al. names higher-order time stepping as future work and gives no
scheme, so the method here is an outside specification, stated in full:

* Eq. (2) written as a one-step map.  Per Fourier mode k, with omega^2 = 1 + k^2 and
  F = R2C(lam u^3) of the field u = C2R(a) (the conventions of kg_oracle.c), the map
  Phi_h of one substep of length h on (a, p) is kick-drift-kick:
      p <- p + (h/2) G_h(a),   a <- a + h p,   p <- p + (h/2) G_h(a),
      G_h(a) = (F(a) - omega^2 a) / (1 + omega^2 h^2 / 4).
  With h = dt throughout and p = v0 at the start this is Eq. (2) exactly (including the
  startup level of kg_oracle.c): a^{n+1} - 2 a^n + a^{n-1} = dt^2 G_dt(a^n) is
  a^{n+1} = 2 c_k a^n - a^{n-1} + 2 beta_k F^n.  G_h is even in h, so Phi_{-h} is the
  inverse of Phi_h: the map is symmetric, hence of even order, and consistent, hence of
  order two.
* The triple jump (Yoshida, Phys. Lett. A 150 (1990) 262; also Suzuki 1990): one step of
  length dt is Phi_{g1 dt} o Phi_{g2 dt} o Phi_{g1 dt} with g1 = 1 / (2 - 2^{1/3}) and
  g2 = 1 - 2 g1, the solution of g1 + g2 + g1 = 1 and g1^3 + g2^3 + g1^3 = 0.  A symmetric
  composition of a symmetric second-order map with these weights is of order four.

The oracle applies every kick with its own evaluation of F (two per substep), in the order
written above; numpy's FFT is the transform step.  Blow-up: before each step, max|u| of
the field at the integer time is compared with the threshold, as for Eq. (2).
"""
import numpy as np

G1 = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
G2 = 1.0 - 2.0 * G1
TRIPLE_JUMP = (G1, G2, G1)


def wavenumbers_sq(N, L):
    """k^2 on the half spectrum [kz][ky][kx] (FFT order, Nyquist index kept)"""
    m = np.fft.fftfreq(N, 1.0 / N)
    m[N // 2] = N // 2                      # the Nyquist index keeps k = pi N / L
    mx = np.arange(N // 2 + 1, dtype=np.float64)
    k = 2.0 * np.pi / L
    return (k * m[:, None, None]) ** 2 + (k * m[None, :, None]) ** 2 + (k * mx[None, None, :]) ** 2


class Composed4Solver:
    """(a, p) = (uh, vh) of a real field on an N^3 grid of side L, stepped by the
    composition `gammas` of the kick-drift-kick map (the triple jump by default;
    gammas = (1,) is Eq. (2))."""

    def __init__(self, N, L, dt, u0, v0=None, lam=1.0, gammas=TRIPLE_JUMP):
        self.N, self.L, self.dt, self.lam = N, float(L), float(dt), float(lam)
        self.gammas = tuple(float(g) for g in gammas)
        self.w2 = 1.0 + wavenumbers_sq(N, L)
        self.a = np.fft.rfftn(np.asarray(u0, dtype=np.float64))
        self.p = np.zeros_like(self.a) if v0 is None else np.fft.rfftn(np.asarray(v0, dtype=np.float64))
        self.level = 0
        self.frozen = False
        self.blowup_level = -1
        self.last_maxabs = 0.0

    def field(self, a=None):
        return np.fft.irfftn(self.a if a is None else a, s=(self.N,) * 3, axes=(0, 1, 2))

    def force(self, a):
        """F(a) = R2C(lam u^3), u = C2R(a)"""
        u = self.field(a)
        return np.fft.rfftn(self.lam * u * u * u)

    def G(self, a, h):
        return (self.force(a) - self.w2 * a) / (1.0 + self.w2 * h * h / 4.0)

    def substep(self, h):
        self.p = self.p + 0.5 * h * self.G(self.a, h)
        self.a = self.a + h * self.p
        self.p = self.p + 0.5 * h * self.G(self.a, h)

    def step(self, n, threshold=0.0):
        """n steps (fewer if the field blows up); returns (blown_up, blowup_level)"""
        for _ in range(int(n)):
            if self.frozen:
                break
            self.last_maxabs = float(np.abs(self.field()).max())
            if threshold > 0.0 and not (self.last_maxabs <= threshold):
                self.frozen = True
                self.blowup_level = self.level
                break
            for g in self.gammas:
                self.substep(g * self.dt)
            self.level += 1
        return self.frozen, self.blowup_level

    def stored_velocity(self):
        """the velocity variable the GPU library keeps between steps:
        P = p - (h1/2) G_{h1}(a), h1 = gammas[0] dt (p before the last closing half kick)"""
        h1 = self.gammas[0] * self.dt
        return self.p - 0.5 * h1 * self.G(self.a, h1)

    def energy(self):
        """continuous energy of section 1.1 at the current (synchronised) level, by Parseval:
        (h^3/N^3) sum_k w_k (|p|^2 + omega^2 |a|^2) / 2 - lam (h^3/4) sum_x u^4"""
        N = self.N
        h3 = (self.L / N) ** 3
        w = np.full(self.a.shape, 2.0)
        w[..., 0] = 1.0
        w[..., N // 2] = 1.0
        quad = 0.5 * np.sum(w * (np.abs(self.p) ** 2 + self.w2 * np.abs(self.a) ** 2)) * h3 / N ** 3
        u = self.field()
        return float(quad - self.lam * h3 / 4.0 * np.sum(u ** 4))
