"""Write constant_field.txt: the spatially constant solution of the scheme, Eq. (2).

For u^n(x) = a_n everywhere the Laplacian term of Eq. (2) vanishes and the scheme
reduces to the scalar recurrence
    (a_{n+1} - 2 a_n + a_{n-1}) / dt^2 + (a_{n+1} + 2 a_n + a_{n-1}) / 4 = lam a_n^3,
solved here for a_{n+1} directly in that form, in 50-digit decimal arithmetic.
The first level uses the symmetric start (a_1 - a_{-1}) / (2 dt) = v0 = 0, i.e.
a_1 = a_{-1}, substituted into the same equation at n = 0.
No code of the oracle or of the GPU library is used.
"""
import os
from decimal import Decimal, getcontext

getcontext().prec = 50

CASES = [  # (a0, dt, lam, steps)
    ("0.3", "0.01", "1", 300),
    ("1.2", "0.005", "1", 200),
    ("0.7", "0.05", "0", 100),
]


def levels(a0, dt, lam, steps):
    a0, dt, lam = Decimal(a0), Decimal(dt), Decimal(lam)
    inv = 1 / (dt * dt)
    q = Decimal(1) / 4
    # n = 0 with a_1 = a_{-1}: 2 (a_1 - a_0) inv + (2 a_1 + 2 a_0) q = lam a_0^3
    a1 = (lam * a0 ** 3 + 2 * a0 * inv - 2 * a0 * q) / (2 * inv + 2 * q)
    seq = [a0, a1]
    prev, cur = a0, a1
    for _ in range(steps - 1):
        nxt = (lam * cur ** 3 + (2 * cur - prev) * inv - (2 * cur + prev) * q) / (inv + q)
        seq.append(nxt)
        prev, cur = cur, nxt
    return seq


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "constant_field.txt")
    with open(out, "w") as f:
        f.write("# constant-field levels a_n of Eq. (2); columns: case a0 dt lam n a_n (50-digit decimal)\n")
        for ci, (a0, dt, lam, steps) in enumerate(CASES):
            for n, a in enumerate(levels(a0, dt, lam, steps)):
                f.write("%d %s %s %s %d %s\n" % (ci, a0, dt, lam, n, format(a, ".25e")))


if __name__ == "__main__":
    main()
