"""Host logic of the ranker driver: Sobol points, AUC, and the bracket/bisection logic
(with a stand-in solver whose blow-up boundary is known)."""
import numpy as np
import pytest

from paper_1501_04552_gb300 import ranker as R


def test_sobol_matches_scipy():
    qmc = pytest.importorskip("scipy.stats").qmc
    assert np.array_equal(R.sobol2(8192), qmc.Sobol(d=2, scramble=False).random(8192))
    assert np.array_equal(R.sobol2(100, skip=7), R.sobol2(107)[7:])


def test_sobol_stratifies():
    u = R.sobol2(1024)
    h, _, _ = np.histogram2d(u[:, 0], u[:, 1], bins=32, range=[[0, 1], [0, 1]])
    assert h.min() == h.max() == 1          # one point in every elementary 1/32 x 1/32 cell


def test_auc_against_pair_counting():
    rng = np.random.default_rng(0)
    s = np.round(rng.uniform(size=300), 2)    # ties included
    y = rng.uniform(size=300) < 0.4
    pos, neg = s[y], s[~y]
    ref = (np.sum(pos[:, None] > neg[None, :]) + 0.5 * np.sum(pos[:, None] == neg[None, :])) / (pos.size * neg.size)
    assert abs(R.auc(s, y) - ref) < 1e-12


def fake_solver(boundary):
    def solve(A, s, T, dt=0.005, N=64, threshold=1e3, chunk=1024, precision="df64"):
        A = np.asarray(A)
        flag = A > boundary(np.asarray(s))
        return {"flag": flag, "tb": np.where(flag, 1.0, np.inf), "features": np.ones((A.size, 4)),
                "seconds": 0.0, "instance_steps": 0}
    return solve


def test_bisection_finds_the_boundary_and_guided_brackets_save_runs(monkeypatch):
    b = lambda s: 1.0 + 1.2 * s
    monkeypatch.setattr(R, "solve", fake_solver(b))
    sv = np.linspace(0.5, 2.0, 16)
    a1, r1 = R.boundary_bisect(sv, 10.0, 0.04)
    assert np.all(np.abs(a1 - b(sv)) <= 0.02)
    a2, r2 = R.boundary_bisect(sv, 10.0, 0.04, lo=b(sv) - 0.05, hi=b(sv) + 0.1)
    assert np.all(np.abs(a2 - b(sv)) <= 0.02) and r2 < r1
    # wrong guesses are detected and widened to the right side of the boundary
    a3, _ = R.boundary_bisect(sv, 10.0, 0.04, lo=b(sv) + 0.3, hi=b(sv) + 0.5)
    a4, _ = R.boundary_bisect(sv, 10.0, 0.04, lo=b(sv) - 0.6, hi=b(sv) - 0.4)
    assert np.all(np.abs(a3 - b(sv)) <= 0.02) and np.all(np.abs(a4 - b(sv)) <= 0.02)
